"""GPU: the batched persistent form against single solves and the oracle.

Every window of a batch runs the same iteration as its single solve; only the
number of CTAs sharing its pixels (and so the grouping of the FP32 partial
sums) differs, so L and S agree with the single solve and with the oracle
within the FP32 tolerance (relative Frobenius <= 1e-5) and the iteration
counts agree within one.  A window given the same CTA count as its single
solve reproduces it bit for bit.
"""
import numpy as np
import pytest

from oracle import rpca_oracle as O
from paper_2506_10257_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

FP32_TOL = 1e-5

SHAPES = [(64, 64, 20), (32, 48, 12), (40, 40, 7), (16, 16, 32), (20, 17, 13), (63, 64, 20), (8, 8, 3)]


@pytest.fixture(scope="module")
def rp():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2506_10257_gb300 import rpca
    rpca.load()
    return rpca


def rel(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (nb if nb > 0 else 1.0)


def windows(shapes, seed0=100):
    out = []
    for i, (ny, nx, T) in enumerate(shapes):
        out.append(synth.make_window(seed=seed0 + i, ny=ny, nx=nx, T=T, n_bound=4, n_free=6))
    return out


def run_batch(rp, wins, thetas=None, tune=False, schedule=None, **kw):
    shapes = [(w.m, w.T) for w in wins]
    b = rp.Batch(shapes, **kw)
    if schedule is not None:
        b.set_schedule(**schedule)
    X = [torch.from_numpy(np.ascontiguousarray(w.frames, dtype=np.float32)).cuda() for w in wins]
    masks = [torch.zeros(w.m, dtype=torch.uint8, device="cuda") for w in wins] if thetas is not None else None
    if tune:
        b.tune(X, reps=1)
    Ls, Ss, res = b.solve(X, masks=masks, thetas=thetas)
    torch.cuda.synchronize()
    info = b.info()
    b.close()
    out = [dict(L=L.cpu().numpy(), S=S.cpu().numpy(), res=r) for L, S, r in zip(Ls, Ss, res)]
    if masks is not None:
        for o, mk in zip(out, masks):
            o["mask"] = mk.cpu().numpy().astype(bool)
    return out, info


def single(rp, w, **kw):
    X = torch.from_numpy(np.ascontiguousarray(w.frames, dtype=np.float32)).cuda()
    plan = rp.Plan(w.m, w.T, **kw)
    L, S, res = plan.solve(X)
    torch.cuda.synchronize()
    plan.close()
    return dict(L=L.cpu().numpy(), S=S.cpu().numpy(), res=res)


def test_batch_matches_single_solves_and_oracle(rp):
    wins = windows(SHAPES)
    refs = [O.rpca_frames(w.frames) for w in wins]
    thetas = [O.mask_threshold(O.temporal_mean_abs(r.L), w.bound_mask_gt) for r, w in zip(refs, wins)]
    got, info = run_batch(rp, wins, thetas=thetas)
    # default schedule: lanes of two windows, run paired beside an eigen-step CTA
    assert info["grid"] >= len(wins) and info["lanes"] == (len(wins) + 1) // 2 and info["paired"] == 1
    rows = []
    for w, r, g, th in zip(wins, refs, got, thetas):
        s = single(rp, w)
        rows.append((w.m, w.T, g["res"]["status"], g["res"]["iters"], s["res"]["iters"], r.iters,
                     rel(g["L"], s["L"]), rel(g["S"], s["S"]), rel(g["L"], r.L), rel(g["S"], r.S),
                     info["window_ctas"][len(rows)]))
    print("\n(m, T, status, iters batch/single/oracle, dL/dS vs single, dL/dS vs oracle, CTAs)")
    for row in rows:
        print(row)
    for w, r, g, th, row in zip(wins, refs, got, thetas, rows):
        assert g["res"]["status"] == rp.OK, g["res"]
        assert row[6] <= FP32_TOL and row[7] <= FP32_TOL, row
        assert row[8] <= FP32_TOL and row[9] <= FP32_TOL, row
        assert abs(row[3] - row[4]) <= 1 and abs(row[3] - row[5]) <= 1, row
        mref = O.bound_mask(O.temporal_mean_abs(r.L), th)
        if mref.any():
            assert O.dice(g["mask"], mref) >= 0.999


@pytest.mark.parametrize("lanes", [1, 2])
def test_paired_lanes_refill_their_slots(rp, lanes):
    # 9 windows on 1 or 2 paired lanes: each slot runs several windows one
    # after the other, windows finish at different iterations (max_iter caps
    # and sizes differ), so slots are refilled while the other slot's window
    # is mid-solve; every result equals its single solve's within the FP32
    # tolerance and the oracle's
    shapes = [(64, 64, 20), (16, 16, 8), (40, 40, 7), (32, 48, 12), (8, 8, 3), (63, 64, 20), (16, 16, 32),
              (20, 17, 13), (24, 24, 16)]
    wins = windows(shapes, seed0=150)
    params = [dict(max_iter=(5 if i % 3 == 1 else 500)) for i in range(len(wins))]
    got, info = run_batch(rp, wins, params=params, schedule=dict(lanes=lanes, paired=True))
    assert info["paired"] == 1 and info["lanes"] == lanes
    for w, g, p in zip(wins, got, params):
        s = single(rp, w, **p)
        r = O.rpca_frames(w.frames, max_iter=p["max_iter"])
        assert g["res"]["status"] == s["res"]["status"], (g["res"], s["res"])
        assert abs(g["res"]["iters"] - s["res"]["iters"]) <= 1
        assert rel(g["L"], s["L"]) <= FP32_TOL and rel(g["S"], s["S"]) <= FP32_TOL
        assert rel(g["L"], r.L) <= FP32_TOL and rel(g["S"], r.S) <= FP32_TOL


def test_paired_and_unpaired_schedules_agree(rp):
    wins = windows(SHAPES[:6], seed0=170)
    a, ia = run_batch(rp, wins, schedule=dict(lanes=3, paired=True))
    b, ib = run_batch(rp, wins, schedule=dict(lanes=6, paired=False))
    assert ia["paired"] == 1 and ib["paired"] == 0
    for x, y in zip(a, b):
        assert x["res"]["status"] == y["res"]["status"] == rp.OK
        assert rel(x["L"], y["L"]) <= FP32_TOL and rel(x["S"], y["S"]) <= FP32_TOL


def test_batch_is_deterministic(rp):
    wins = windows(SHAPES[:4], seed0=200)
    a, _ = run_batch(rp, wins)
    b, _ = run_batch(rp, wins)
    for x, y in zip(a, b):
        assert np.array_equal(x["L"], y["L"]) and np.array_equal(x["S"], y["S"])


def test_more_windows_than_lanes(rp):
    # 400 small windows: lanes hold several windows each, run one after another
    shapes = [(16, 16, 8 + (i % 5) * 4) for i in range(400)]
    wins = windows(shapes, seed0=300)
    got, info = run_batch(rp, wins)
    assert info["lanes"] <= info["grid"]
    for k in (0, 1, 57, 199, 398, 399):
        r = O.rpca_frames(wins[k].frames)
        assert rel(got[k]["L"], r.L) <= FP32_TOL and rel(got[k]["S"], r.S) <= FP32_TOL
    assert all(g["res"]["status"] == rp.OK for g in got)


def test_tuned_schedule_keeps_results(rp):
    wins = windows([(64, 64, 20), (128, 64, 16), (16, 16, 8), (32, 32, 24)], seed0=400)
    base, _ = run_batch(rp, wins)
    tuned, info = run_batch(rp, wins, tune=True)
    assert info["grid"] >= 1 and info["lanes"] >= 1
    for x, y in zip(base, tuned):
        assert rel(y["L"], x["L"]) <= FP32_TOL and rel(y["S"], x["S"]) <= FP32_TOL


def test_batch_per_window_parameters(rp):
    wins = windows([(32, 32, 10), (32, 32, 10)], seed0=500)
    got, _ = run_batch(rp, wins, params=[dict(max_iter=3), dict(mu_schedule=rp.MU_FIXED_L1, max_iter=60, tol=1e-6)])
    assert got[0]["res"]["status"] == rp.NOT_CONVERGED and got[0]["res"]["iters"] == 3
    r0 = O.rpca_frames(wins[0].frames, max_iter=3)
    assert rel(got[0]["L"], r0.L) <= FP32_TOL and rel(got[0]["S"], r0.S) <= FP32_TOL
    r1 = O.rpca_frames(wins[1].frames, schedule=O.SCHEDULE_FIXED_L1, max_iter=60, tol=1e-6)
    assert got[1]["res"]["iters"] == r1.iters
    assert rel(got[1]["L"], r1.L) <= 1e-4 and rel(got[1]["S"], r1.S) <= 1e-4


def test_batch_rejects_unsupported(rp):
    with pytest.raises(rp.RpcaError):
        rp.Batch([(4096, 20)], precision=rp.PREC_TF32)
    with pytest.raises(rp.RpcaError):
        rp.Batch([(4096, 20), (4096, 20)], params=[dict(), dict(precision=rp.PREC_BF16X3)])
    with pytest.raises(ValueError):
        rp.Batch([])


def oracle_same_iters(frames, iters, **kw):
    """The oracle's iterate with the GPU's iteration count (rerun when the FP32
    and FP64 residuals cross tol one iteration apart)."""
    ref = O.rpca_frames(frames, **kw)
    assert abs(iters - ref.iters) <= 1, (iters, ref.iters)
    if iters != ref.iters:
        ref = O.rpca_frames(frames, **dict(kw, max_iter=iters, tol=1e-30))
    return ref


def test_batch_with_wide_windows(rp):
    # a window of more than 32 frames sends every window of the batch through
    # the tiled bodies (narrow ones included)
    wins = windows([(32, 32, 12), (24, 40, 50), (32, 32, 20), (16, 32, 100), (20, 17, 33)], seed0=600)
    got, info = run_batch(rp, wins)
    for w, g in zip(wins, got):
        assert g["res"]["status"] == rp.OK, g["res"]
        ref = oracle_same_iters(w.frames, g["res"]["iters"])
        eL, eS = rel(g["L"], ref.L), rel(g["S"], ref.S)
        assert eL <= FP32_TOL and eS <= FP32_TOL, (eL, eS, w.m, w.T)


def test_batch_of_complex_windows(rp):
    shapes = [(16, 16, 8), (32, 32, 20), (24, 24, 13)]
    wins = [synth.make_window(seed=700 + i, ny=ny, nx=nx, T=T, n_bound=4, n_free=6, complex_iq=True)
            for i, (ny, nx, T) in enumerate(shapes)]
    b = rp.Batch([(w.m, w.T) for w in wins], dtype=rp.C64)
    X = [torch.from_numpy(np.ascontiguousarray(w.frames, dtype=np.complex64)).cuda() for w in wins]
    Ls, Ss, res = b.solve(X)
    torch.cuda.synchronize()
    b.close()
    for w, L, S, r in zip(wins, Ls, Ss, res):
        assert r["status"] == rp.OK
        ref = oracle_same_iters(w.frames, r["iters"])
        assert r["rank"] == ref.rank
        Lg = L.cpu().numpy().astype(np.complex128)
        Sg = S.cpu().numpy().astype(np.complex128)
        eL = np.linalg.norm(Lg - ref.L) / np.linalg.norm(ref.L)
        eS = np.linalg.norm(Sg - ref.S) / np.linalg.norm(ref.S)
        assert eL <= FP32_TOL and eS <= FP32_TOL, (eL, eS)


def test_batch_rejects_mixed_element_types(rp):
    with pytest.raises(rp.RpcaError):
        rp.Batch([(256, 8), (256, 8)], params=[dict(), dict(dtype=rp.C64)])


@pytest.mark.parametrize("prec", ["TF32X3", "BF16X3"])
@pytest.mark.parametrize("paired", [True, False])
def test_tensor_core_batch_matches_oracle(rp, prec, paired):
    # the mixed-precision batched form: every window's two contractions on the
    # tensor cores inside the persistent launch; each window against the FP64
    # oracle at the precision's tolerance and against its single solve
    tol = {"TF32X3": 1e-5, "BF16X3": 1e-4}[prec]
    wins = windows([(64, 64, 20), (32, 48, 12), (63, 64, 20), (16, 16, 32), (40, 40, 7), (20, 17, 13)], seed0=800)
    lanes = 3 if paired else 6
    got, info = run_batch(rp, wins, precision=getattr(rp, "PREC_" + prec), schedule=dict(lanes=lanes, paired=paired))
    assert info["paired"] == int(paired)
    for w, g in zip(wins, got):
        assert g["res"]["status"] == rp.OK, g["res"]
        r = O.rpca_frames(w.frames)
        eL, eS = rel(g["L"], r.L), rel(g["S"], r.S)
        assert eL <= tol and eS <= tol, (prec, w.m, w.T, eL, eS)
        s = single(rp, w, precision=getattr(rp, "PREC_" + prec))
        assert rel(g["L"], s["L"]) <= tol and rel(g["S"], s["S"]) <= tol


@pytest.mark.slow
def test_tensor_core_batch_full_size(rp):
    # 4 windows of 512 x 512 x 20 in TF32x3: many tiles per CTA in every pass
    wins = [synth.make_preset("w512x512_t20", seed=900 + i) for i in range(4)]
    got, info = run_batch(rp, wins, precision=rp.PREC_TF32X3)
    for w, g in zip(wins[:2], got[:2]):
        r = O.rpca_frames(w.frames)
        assert g["res"]["status"] == rp.OK
        assert rel(g["L"], r.L) <= 1e-5 and rel(g["S"], r.S) <= 1e-5


def test_tensor_core_batch_rejects_wide_windows(rp):
    with pytest.raises(rp.RpcaError) as e:
        rp.Batch([(4096, 20), (4096, 40)], precision=rp.PREC_TF32X3)
    assert e.value.status == rp.ERR_UNSUPPORTED
