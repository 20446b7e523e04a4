"""The batch form's CTA schedule (rpca_batch_schedule, the host computation
that rpca_batch_create and rpca_batch_tune use), checked without a GPU: a
hand-worked longest-processing-time assignment, the CTA-split invariants, and
Graham's bound for LPT (makespan <= (4/3 - 1/(3L)) x the optimum) against
brute force on small random batches."""
import itertools

import numpy as np
import pytest

from paper_2506_10257_gb300 import rpca


@pytest.fixture(scope="module", autouse=True)
def lib():
    return rpca.load()


def loads(shapes, lane):
    return sum(shapes[w][0] * shapes[w][1] for w in lane)


def test_hand_worked_lpt_assignment():
    # loads 5,1,4,3,2,3 (x 1000 pixels, T = 1): sorted 5,4,3,3,2,1 (equal loads keep index order);
    # 5->A, 4->B, 3(w3)->B (4 < 5), 3(w5)->A (5 < 7), 2->B (7 < 8), 1->A (8 < 9)
    shapes = [(5000, 1), (1000, 1), (4000, 1), (3000, 1), (2000, 1), (3000, 1)]
    sch = rpca.batch_schedule(shapes, ctas=100, lanes=2, alpha=1.0)
    assert [ws for _, ws in sch] == [[0, 5, 1], [2, 3, 4]]
    assert [loads(shapes, ws) for _, ws in sch] == [9000, 9000]
    assert [c for c, _ in sch] == [50, 50]


def test_cta_split_follows_load_power():
    shapes = [(3000, 10), (1000, 10)]
    c1 = [c for c, _ in rpca.batch_schedule(shapes, ctas=152, lanes=2, alpha=1.0)]
    assert c1 == [114, 38]                                  # 152 x 3/4, 152 x 1/4
    c0 = [c for c, _ in rpca.batch_schedule(shapes, ctas=152, lanes=2, alpha=0.0)]
    assert c0 == [76, 76]                                   # alpha 0: equal shares
    ch = [c for c, _ in rpca.batch_schedule(shapes, ctas=152, lanes=2, alpha=0.5)]
    want = 152 * np.sqrt(3) / (np.sqrt(3) + 1)              # 96.3: the remainder goes to the larger fraction
    assert sum(ch) == 152 and abs(ch[0] - want) < 1


def test_caps_bind_and_the_rest_goes_elsewhere():
    shapes = [(262144, 20), (4096, 20), (4096, 20)]
    # the 149 CTAs beyond one a lane split 144.5 / 2.3 / 2.3: uncapped [146, 3, 3]; with the
    # small windows capped at 2 CTAs the large one takes what they cannot use
    sch = rpca.batch_schedule(shapes, ctas=152, lanes=3, alpha=1.0)
    assert [c for c, _ in sch] == [146, 3, 3]
    sch = rpca.batch_schedule(shapes, ctas=152, lanes=3, alpha=1.0, max_ctas=[152, 2, 2])
    assert [c for c, _ in sch] == [148, 2, 2]
    sch = rpca.batch_schedule(shapes, ctas=152, lanes=3, alpha=1.0, max_ctas=[10, 4, 4])
    assert [c for c, _ in sch] == [10, 4, 4]                # every lane capped: CTAs stay unused


def test_lane_count_is_clamped():
    shapes = [(1000, 5)] * 5
    assert len(rpca.batch_schedule(shapes, ctas=152, lanes=64)) == 5     # at most one lane per window
    assert len(rpca.batch_schedule(shapes, ctas=3, lanes=5)) == 3        # at most one lane per CTA
    one = rpca.batch_schedule(shapes, ctas=152, lanes=1)
    assert one == [(152, [0, 1, 2, 3, 4])]


@pytest.mark.parametrize("seed", range(12))
def test_invariants_and_lpt_bound_against_brute_force(seed):
    rng = np.random.default_rng(seed)
    n = int(rng.integers(2, 8))
    L = int(rng.integers(2, 4))
    shapes = [(int(rng.integers(1, 64)) * 1024, int(rng.integers(5, 33))) for _ in range(n)]
    ctas = int(rng.integers(L, 300))
    alpha = float(rng.choice([0.0, 0.5, 1.0]))
    cap = [int(rng.integers(1, 200)) for _ in range(n)]
    sch = rpca.batch_schedule(shapes, ctas=ctas, lanes=L, alpha=alpha, max_ctas=cap)
    # every window exactly once, each lane in descending load
    assert sorted(w for _, ws in sch for w in ws) == list(range(n))
    for c, ws in sch:
        ld = [shapes[w][0] * shapes[w][1] for w in ws]
        assert ld == sorted(ld, reverse=True)
        assert 1 <= c <= max(1, max(cap[w] for w in ws))
    assert sum(c for c, _ in sch) <= ctas and len(sch) == min(L, n, ctas)
    # LPT makespan within Graham's 4/3 - 1/(3L) of the brute-force optimum
    Ls = len(sch)
    w_load = [m * T for m, T in shapes]
    best = min(max(sum(w_load[w] for w in range(n) if a[w] == l) for l in range(Ls))
               for a in itertools.product(range(Ls), repeat=n))
    got = max(loads(shapes, ws) for _, ws in sch)
    assert got <= (4 / 3 - 1 / (3 * Ls)) * best + 1e-9


def test_bad_arguments():
    with pytest.raises(rpca.RpcaError):
        rpca.batch_schedule([], ctas=10, lanes=1)
    with pytest.raises(rpca.RpcaError):
        rpca.batch_schedule([(0, 5)], ctas=10, lanes=1)
    with pytest.raises(rpca.RpcaError):
        rpca.batch_schedule([(10, 5)], ctas=0, lanes=1)
    with pytest.raises(rpca.RpcaError):
        rpca.batch_schedule([(10, 5)], ctas=10, lanes=1, alpha=float("nan"))
    with pytest.raises(rpca.RpcaError):
        rpca.batch_schedule([(10, 5)], ctas=10, lanes=1, max_ctas=[0])
