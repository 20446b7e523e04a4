"""GPU: the frame pre-filter (rpca_prefilter) against its FP64 oracle.

Kept frames bit-exact, neighbour correlations within 1e-12 (both FP64, the
GPU from shifted raw moments, the oracle from centred frames), averaged frames
within 1e-6 of the largest magnitude (FP64 sliding sums, FP32 output); the
high-pass variant within 1e-6 of its largest output magnitude plus 1e-12 of
the largest input magnitude (the FP64 difference of the centre frame and the
window mean, rounded once to FP32)."""
import numpy as np
import pytest

from oracle import prefilter_oracle as P
from oracle import rpca_oracle as O
from paper_2506_10257_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rp():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2506_10257_gb300 import rpca
    rpca.load()
    return rpca


def smooth_frames(seed, T, m, drift=0.05, offset=1.0):
    rng = np.random.default_rng(seed)
    base = offset + rng.standard_normal(m)
    return (base[None, :] + drift * np.cumsum(rng.standard_normal((T, m)), axis=0)).astype(np.float32)


def check(rp, F, corr_min, window, high_pass=False):
    Y, kept, corr = rp.prefilter(torch.from_numpy(F).cuda(), corr_min=corr_min, window=window, high_pass=high_pass)
    want_Y, want_kept, want_c = P.prefilter(F, corr_min, window, high_pass=high_pass)
    assert kept.cpu().numpy().tolist() == want_kept.tolist()
    if F.shape[0] > 1:
        np.testing.assert_allclose(corr.cpu().numpy(), want_c, rtol=0, atol=1e-12)
    Yh = Y.cpu().numpy().astype(np.float64)
    assert Yh.shape == want_Y.shape
    if want_Y.size:
        tol = 1e-6 * max(np.abs(want_Y).max(), 1e-30) + (1e-12 * np.abs(F).max() if high_pass else 0.0)
        assert np.abs(Yh - want_Y).max() <= tol
    return Yh, kept.cpu().numpy(), corr.cpu().numpy()


@pytest.mark.parametrize("T,m,bad,window", [(30, 5003, [5, 17], 20), (24, 4096, [0, 23], 5), (40, 333, [], 20),
                                            (12, 70000, [6], 3)])
def test_prefilter_matches_oracle(rp, T, m, bad, window):
    F = smooth_frames(T * 7 + m, T, m)
    rng = np.random.default_rng(m)
    for t in bad:
        F[t] = (1.0 + rng.standard_normal(m)).astype(np.float32)   # uncorrelated with its neighbours
    _, kept, _ = check(rp, F, 0.8, window)
    assert set(kept.tolist()) == set(range(T)) - set(bad)


def test_prefilter_edge_cases(rp):
    F = smooth_frames(1, 1, 1000)
    Y, kept, _ = check(rp, F, 0.8, 1)                # one frame: kept, window 1 returns it
    assert kept.tolist() == [0] and np.array_equal(Y, F.astype(np.float64))
    check(rp, F, 0.8, 20)                            # fewer kept frames than the window: no output
    rng = np.random.default_rng(2)
    check(rp, rng.standard_normal((6, 2000)).astype(np.float32), 0.8, 2)   # nothing correlates: none kept
    G = smooth_frames(3, 8, 512)
    G[4] = 2.5                                       # a frame without variance correlates 0
    _, kept, corr = check(rp, G, 0.8, 2)
    assert corr[3] == 0.0 and corr[4] == 0.0 and 4 not in kept.tolist()


def test_prefilter_on_the_paper_reference_shape(rp):
    # 338 x 260 pixels, 132 frames (the in vivo reference's frame count), with
    # three frames displaced by a whole-image shift (motion) that drop out
    w = synth.make_window(seed=55, ny=338, nx=260, T=132, n_bound=200, n_free=400, speed=(0.5, 5.0))
    F = w.frames.copy()
    for t in (40, 41, 90):
        img = F[t].reshape(338, 260)
        F[t] = np.roll(img, (25, 31), axis=(0, 1)).reshape(-1)
    Y, kept, corr = check(rp, F, 0.8, 20)
    assert 90 not in kept.tolist() and Y.shape == (len(kept) - 19, 338 * 260)


def test_prefilter_feeds_a_solve_on_the_same_stream(rp):
    # a 64 x 64 microbubble window of 30 frames with one displaced frame
    # (neighbour correlations 0.80-0.96, the displaced frame's ~0), pre-filtered
    # at 0.5 and solved on one stream without a host round trip between
    w = synth.make_window(seed=31, ny=64, nx=64, T=30, n_bound=15, n_free=30)
    F = w.frames.copy()
    F[11] = np.roll(F[11].reshape(64, 64), (9, 13), axis=(0, 1)).reshape(-1)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        X = torch.from_numpy(F).cuda()
        Yf, kf, cf, count = rp.prefilter(X, 0.5, 10, stream=s, wait=False)
        plan = rp.Plan(4096, 20)                   # 29 kept frames expected: 20 averaged frames
        L, S, _ = plan.solve(Yf[:20], stream=s, wait=False)
    s.synchronize()
    K, n = count.cpu().tolist()
    want_Y, want_kept, _ = P.prefilter(F, 0.5, 10)
    assert kf[:K].cpu().numpy().tolist() == want_kept.tolist() and n == 20
    res = plan.result()
    plan.close()
    ref = O.rpca_frames(Yf[:n].cpu().numpy().astype(np.float64))   # the oracle on the same input
    assert res["status"] == rp.OK and abs(res["iters"] - ref.iters) <= 1
    rel = lambda a, b: np.linalg.norm(a - b) / np.linalg.norm(b)
    assert rel(L.cpu().numpy().astype(np.float64), ref.L) <= 1e-5
    assert rel(S.cpu().numpy().astype(np.float64), ref.S) <= 1e-5


def test_prefilter_rejects_bad_arguments(rp):
    X = torch.zeros((4, 64), dtype=torch.float32, device="cuda")
    with pytest.raises(rp.RpcaError):
        rp.prefilter(X, corr_min=float("nan"))
    with pytest.raises(rp.RpcaError):
        rp.prefilter(X, window=0)
    with pytest.raises(ValueError):
        rp.prefilter(X.double())


@pytest.mark.parametrize("T,m,bad,window", [(30, 5003, [5, 17], 7), (24, 4096, [0, 23], 6), (40, 70000, [9], 20),
                                            (12, 333, [], 1)])
def test_highpass_matches_oracle(rp, T, m, bad, window):
    F = smooth_frames(T * 5 + m, T, m)
    t = np.arange(T, dtype=np.float32)[:, None]
    F += (0.3 * t + 0.2 * np.sin(0.9 * t)).astype(np.float32)   # a slow trend under a faster oscillation
    rng = np.random.default_rng(m + 1)
    for b in bad:
        F[b] = (1.0 + rng.standard_normal(m)).astype(np.float32)
    Y, kept, _ = check(rp, F, 0.8, window, high_pass=True)
    assert set(kept.tolist()) == set(range(T)) - set(bad)
    if window == 1:
        assert not Y.any()                            # a one-frame window removes everything


def test_highpass_removes_a_linear_trend_exactly(rp):
    # frames t*v + c (exact in FP32) with an odd window: every output is 0
    T, m, w = 26, 2048, 5
    rng = np.random.default_rng(9)
    v = rng.integers(-8, 8, m).astype(np.float32)
    c = rng.integers(-100, 100, m).astype(np.float32)
    F = (np.arange(T, dtype=np.float32)[:, None] * v[None, :] + c[None, :]).astype(np.float32)
    Y, kept, _ = rp.prefilter(torch.from_numpy(F).cuda(), corr_min=-2.0, window=w, high_pass=True)
    assert kept.cpu().numpy().tolist() == list(range(T)) and Y.shape == (T - w + 1, m)
    assert float(Y.abs().max()) <= 1e-12 * float(np.abs(F).max())


def test_highpass_feeds_a_solve(rp):
    # a 64 x 64 microbubble window of 26 frames with a slow gain ramp: high-passed
    # over 7 frames, then solved; the oracle runs on the same 20 high-passed frames
    w = synth.make_window(seed=37, ny=64, nx=64, T=26, n_bound=15, n_free=30)
    F = (w.frames * (1.0 + 0.01 * np.arange(26, dtype=np.float32))[:, None]).astype(np.float32)
    X = torch.from_numpy(F).cuda()
    Y, kept, _ = rp.prefilter(X, corr_min=0.5, window=7, high_pass=True)
    assert kept.numel() == 26 and Y.shape[0] == 20
    want_Y, _, _ = P.prefilter(F, 0.5, 7, high_pass=True)
    np.testing.assert_allclose(Y.cpu().numpy(), want_Y, rtol=0, atol=1e-6 * np.abs(want_Y).max() + 1e-9)
    plan = rp.Plan(4096, 20)
    L, S, res = plan.solve(Y.contiguous())
    plan.close()
    ref = O.rpca_frames(Y.cpu().numpy().astype(np.float64))
    assert res["status"] == rp.OK and abs(res["iters"] - ref.iters) <= 1
    rel = lambda a, b: np.linalg.norm(a - b) / np.linalg.norm(b)
    assert rel(L.cpu().numpy().astype(np.float64), ref.L) <= 1e-5
    assert rel(S.cpu().numpy().astype(np.float64), ref.S) <= 1e-5


def test_highpass_rejects_bad_arguments(rp):
    X = torch.zeros((4, 64), dtype=torch.float32, device="cuda")
    with pytest.raises(rp.RpcaError):
        rp.prefilter(X, window=0, high_pass=True)
