"""GPU parity of complex IQ windows (complex64, Hermitian Gram, magnitude
shrink) against the CPU oracle in complex128.

The solver runs the window as its interleaved real embedding (2T columns) on
the tiled path; the tolerance is the FP32 one: relative Frobenius error of L
and S <= 1e-5, iteration counts within one (when they differ by one the
oracle is rerun to the GPU's count), bound-bubble mask Dice >= 0.999.
"""
import numpy as np
import pytest

from oracle import rpca_oracle as O
from paper_2506_10257_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

FP32_TOL = 1e-5


@pytest.fixture(scope="module")
def rp():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2506_10257_gb300 import rpca
    rpca.load()
    return rpca


def rel(a, b):
    a = np.asarray(a, np.complex128)
    b = np.asarray(b, np.complex128)
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (nb if nb > 0 else 1.0)


def cuda(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.complex64)).cuda()


def solve(rp, frames, theta=None, **kw):
    T, m = frames.shape
    plan = rp.Plan(m, T, dtype=rp.C64, **kw)
    mask = torch.zeros(m, dtype=torch.uint8, device="cuda") if theta is not None else None
    L, S, res = plan.solve(cuda(frames), mask=mask, theta=0.0 if theta is None else theta)
    torch.cuda.synchronize()
    plan.close()
    out = dict(L=L.cpu().numpy(), S=S.cpu().numpy(), res=res)
    if mask is not None:
        out["mask"] = mask.cpu().numpy().astype(bool)
    return out


def check(frames, got, tol=FP32_TOL, iters_within=1, **kw):
    ref = O.rpca_frames(frames, **kw)
    if iters_within is not None:
        assert abs(got["res"]["iters"] - ref.iters) <= iters_within, (got["res"]["iters"], ref.iters)
        if got["res"]["iters"] != ref.iters:
            ref = O.rpca_frames(frames, **dict(kw, max_iter=got["res"]["iters"], tol=1e-30))
    eL, eS = rel(got["L"], ref.L), rel(got["S"], ref.S)
    assert eL <= tol and eS <= tol, (eL, eS, got["res"]["iters"], ref.iters)
    return ref


@pytest.mark.parametrize("ny,nx,T", [(16, 16, 8), (64, 64, 20), (31, 45, 13), (40, 40, 50), (64, 64, 100)])
def test_complex_solve_matches_oracle(rp, ny, nx, T):
    w = synth.make_window(seed=ny * nx + T, ny=ny, nx=nx, T=T, n_bound=6, n_free=10, complex_iq=True)
    got = solve(rp, w.frames)
    assert got["res"]["status"] == rp.OK
    ref = check(w.frames, got)
    assert got["res"]["rank"] == ref.rank


@pytest.mark.parametrize("prec", ["TF32X3", "BF16X3"])
@pytest.mark.parametrize("ny,nx,T", [(16, 16, 8), (64, 64, 20), (31, 45, 13), (40, 40, 50), (48, 48, 64)])
def test_complex_tensor_core_matches_oracle(rp, prec, ny, nx, T):
    # the tiled tensor-core pass on the real embedding (Q, Z~ = Z' V and
    # (i Z') V, and the Gram of both row sets on tcgen05): TF32x3 at the FP32
    # tolerance and within one iteration of the oracle; BF16x3 at 1e-4 (its
    # rounding floor near the stopping tolerance can cost iterations)
    w = synth.make_window(seed=3 * ny * nx + T, ny=ny, nx=nx, T=T, n_bound=6, n_free=10, complex_iq=True)
    got = solve(rp, w.frames, precision=getattr(rp, "PREC_" + prec))
    assert got["res"]["status"] == rp.OK
    if prec == "TF32X3":
        check(w.frames, got)
    else:
        check(w.frames, got, tol=1e-4, iters_within=None)


def test_complex_mask(rp):
    w = synth.make_preset("w64x64_t20", seed=3, complex_iq=True)
    ref = O.rpca_frames(w.frames)
    theta = O.mask_threshold(O.temporal_mean_abs(ref.L), w.bound_mask_gt)
    got = solve(rp, w.frames, theta=theta)
    mref = O.bound_mask(O.temporal_mean_abs(ref.L), theta)
    assert O.dice(got["mask"], mref) >= 0.999


@pytest.mark.parametrize("drive", ["HOST", "STREAM"])
def test_complex_other_drives(rp, drive):
    w = synth.make_window(seed=4, ny=24, nx=24, T=12, n_bound=4, n_free=6, complex_iq=True)
    got = solve(rp, w.frames, drive=getattr(rp, "DRIVE_" + drive))
    check(w.frames, got)


def test_complex_fixed_schedule(rp):
    w = synth.make_window(seed=5, ny=32, nx=32, T=10, n_bound=5, n_free=8, complex_iq=True)
    got = solve(rp, w.frames, mu_schedule=rp.MU_FIXED_L1, max_iter=60, tol=1e-6)
    ref = O.rpca_frames(w.frames, schedule=O.SCHEDULE_FIXED_L1, max_iter=60, tol=1e-6)
    assert got["res"]["iters"] == ref.iters
    assert rel(got["L"], ref.L) <= 1e-4 and rel(got["S"], ref.S) <= 1e-4


def test_complex_warm_start(rp):
    w = synth.make_window(seed=6, ny=32, nx=32, T=13, n_bound=4, n_free=6, complex_iq=True)
    F = np.ascontiguousarray(w.frames, dtype=np.complex64)
    prev = O.rpca_frames(F[0:12])
    S0 = np.zeros_like(prev.S); S0[:-1] = prev.S[1:]
    Y0 = np.zeros_like(prev.Y); Y0[:-1] = prev.Y[1:]
    S0, Y0 = S0.astype(np.complex64), Y0.astype(np.complex64)
    ref = O.rpca_frames(F[1:13], S0=S0.astype(np.complex128), Y0=Y0.astype(np.complex128))
    plan = rp.Plan(w.m, 12, dtype=rp.C64, warm_start=1)
    L, S, res = plan.solve(cuda(F[1:13]), L=cuda(Y0), S=cuda(S0))
    torch.cuda.synchronize()
    plan.close()
    assert rel(L.cpu().numpy(), ref.L) <= FP32_TOL and rel(S.cpu().numpy(), ref.S) <= FP32_TOL


def test_complex_served_chain(rp):
    # the server's frame shift of the warm state covers (Re, Im) pairs: a cold
    # policy must equal cold solves, the warm one must stay close to the oracle chain
    w = synth.make_window(seed=7, ny=24, nx=24, T=12, n_bound=4, n_free=6, complex_iq=True)
    F = np.ascontiguousarray(w.frames, dtype=np.complex64)
    wins = [np.ascontiguousarray(F[s:s + 10]) for s in range(3)]
    sv = rp.Server(hbm_budget_bytes=10**9, max_slots=2, warm=True, warm_mu_scale=0.0)
    ids = [sv.submit(cuda(x), key=9) for x in wins]
    outs = []
    for r in ids:
        st, res = sv.wait(r)
        L, S, _ = sv.outputs(r)
        outs.append((st, L.cpu().numpy(), S.cpu().numpy()))
    sv.close()
    prev = None
    for k, x in enumerate(wins):
        kw = {}
        if prev is not None:
            S0 = np.zeros_like(prev.S); S0[:-1] = prev.S[1:]
            Y0 = np.zeros_like(prev.Y); Y0[:-1] = prev.Y[1:]
            kw = dict(S0=S0, Y0=Y0)
        ref = O.rpca_frames(x, **kw)
        st, L, S = outs[k]
        assert st == rp.OK
        tol = FP32_TOL if k == 0 else 2e-3
        assert rel(L, ref.L) <= tol and rel(S, ref.S) <= tol, (k, rel(L, ref.L), rel(S, ref.S))
        prev = ref


def test_complex_limits(rp):
    with pytest.raises(rp.RpcaError):
        rp.Plan(1000, 113, dtype=rp.C64)          # 2T > 224
    with pytest.raises(rp.RpcaError):
        rp.Plan(1000, 65, dtype=rp.C64, precision=rp.PREC_BF16X3)   # 2T > 128: no tensor-core pass
    rp.Plan(1000, 64, dtype=rp.C64, precision=rp.PREC_BF16X3).close()
