"""Pins of the CPU FP64 oracle against facts fixed by the paper and by the mathematics.

None of these compares the oracle with itself: every expected value is a closed
form, a hand-derived iteration, an optimality certificate, a symmetry of the
problem, or a brute-force search.
"""
import math

import numpy as np
import pytest

from conftest import read_golden
from oracle import rpca_oracle as O
from paper_2506_10257_gb300 import synth


# --- Eq. 5: soft-thresholding ------------------------------------------------

def test_shrink_closed_form_table():
    g = 0.75
    x = np.array([-3.0, -g, -g / 2, 0.0, g / 2, g, 3.0, 1.0])
    want = np.array([-2.25, 0.0, 0.0, 0.0, 0.0, 0.0, 2.25, 0.25])
    np.testing.assert_array_equal(O.shrink(x, g), want)


def test_shrink_complex_keeps_phase():
    g = 0.5
    z = np.array([3 + 4j, 0.3 + 0.4j, 0j, -2j])
    want = np.array([(3 + 4j) * (4.5 / 5), 0j, 0j, -1.5j])
    np.testing.assert_allclose(O.shrink(z, g), want, rtol=0, atol=1e-15)


# --- Eq. 4: singular value thresholding -------------------------------------

def test_svt_on_constructed_spectrum():
    rng = np.random.default_rng(0)
    m, T = 50, 7
    U, _ = np.linalg.qr(rng.standard_normal((m, T)))
    V, _ = np.linalg.qr(rng.standard_normal((T, T)))
    sig = np.array([9.0, 5.0, 3.0, 2.0, 1.5, 0.5, 0.1])
    M = (U * sig) @ V.T
    tau = 1.75
    want = (U * np.maximum(sig - tau, 0)) @ V.T
    got, r = O.svt(M, tau)
    assert r == 4
    np.testing.assert_allclose(got, want, rtol=0, atol=1e-13)


def test_svt_tie_at_threshold_is_dropped():
    M = np.diag([3.0, 2.0, 1.0])
    got, r = O.svt(M, 2.0)
    assert r == 1
    np.testing.assert_allclose(got, np.diag([1.0, 0.0, 0.0]), atol=1e-15)


# --- Sec. II-A iteration, hand-derived --------------------------------------

def test_two_iterations_match_hand_derivation():
    g = read_golden("spike_two_iterations.txt")
    a, m, T = g["a"], int(g["m"]), int(g["T"])
    X = np.zeros((m, T))
    X[0, 0] = a
    r1 = O.rpca(X, max_iter=1)
    assert r1.lam == pytest.approx(g["lambda"], rel=1e-15)
    assert r1.mu == pytest.approx(g["mu1"], rel=1e-14)
    assert r1.L[0, 0] == pytest.approx(g["L1"], rel=1e-13)
    assert r1.S[0, 0] == pytest.approx(g["S1"], rel=1e-13)
    assert r1.Y[0, 0] == pytest.approx(g["Y1"], rel=1e-13)
    assert r1.resid == pytest.approx(g["resid1"], rel=1e-13)
    assert not r1.converged
    for A in (r1.L, r1.S, r1.Y):
        B = A.copy()
        B[0, 0] = 0
        assert np.abs(B).max() < 1e-15
    r2 = O.rpca(X, max_iter=2)
    assert r2.iters == 2 and r2.converged
    assert r2.mu == pytest.approx(g["mu2"], rel=1e-14)
    assert r2.L[0, 0] == pytest.approx(g["L2"], rel=1e-12)
    assert r2.S[0, 0] == pytest.approx(g["S2"], rel=1e-12)
    assert r2.Y[0, 0] == pytest.approx(g["Y2"], rel=1e-12)
    assert r2.resid < 1e-15


def test_fixed_l1_schedule_first_iteration():
    # mu = m*T/(4 ||X||_1) (Sec. II-A); for X = a e_00 with m*T = 32: mu = 8/a,
    # tau = a/8 -> L = 7a/8; S = shrink(a/8, lambda*a/8); Y = mu*E = lambda.
    a, m, T = 3.0, 8, 4
    X = np.zeros((m, T))
    X[0, 0] = a
    lam = 1 / math.sqrt(8)
    r = O.rpca(X, schedule=O.SCHEDULE_FIXED_L1, max_iter=1)
    assert r.mu == pytest.approx(8 / a, rel=1e-15)
    assert r.L[0, 0] == pytest.approx(7 * a / 8, rel=1e-13)
    assert r.S[0, 0] == pytest.approx(a * (1 - lam) / 8, rel=1e-13)
    assert r.Y[0, 0] == pytest.approx(lam, rel=1e-12)
    r5 = O.rpca(X, schedule=O.SCHEDULE_FIXED_L1, max_iter=5, tol=0)
    assert all(h[0] == r.mu for h in r5.history)     # mu held constant
    # a negative entry counts with its magnitude in ||X||_1: a e_00 - a e_11
    # has ||X||_1 = 2a, so mu = 32 / (8 a) = 4/a
    X[1, 1] = -a
    assert O.rpca(X, schedule=O.SCHEDULE_FIXED_L1, max_iter=1).mu == pytest.approx(4 / a, rel=1e-15)


def test_ialm_penalty_schedule_and_default_lambda():
    # mu0 = 1.25 / ||X||_2 with the spectral norm: X = diag(3, 4) in a 6 x 3
    # matrix has singular values {4, 3} (Frobenius norm 5), so mu0 = 1.25/4;
    # lambda = 1/sqrt(max(m, T)) = 1/sqrt(6)
    X = np.zeros((6, 3))
    X[0, 0], X[1, 1] = 3.0, 4.0
    r = O.rpca(X, max_iter=1)
    assert r.mu == pytest.approx(1.25 / 4, rel=1e-15)
    assert r.lam == pytest.approx(1 / math.sqrt(6), rel=1e-15)
    # the larger dimension sets lambda whichever it is: 100 x 4 and 4 x 100 both give 1/10
    rng = np.random.default_rng(5)
    for shape in ((100, 4), (4, 100)):
        assert O.rpca(rng.standard_normal(shape), max_iter=1).lam == pytest.approx(0.1, rel=1e-15)
    # mu_k = min(1.5^(k-1), 1e7) mu0: the cap binds from k = 41 (1.5^40 > 1e7)
    G = rng.standard_normal((6, 3))
    h = O.rpca(G, max_iter=45, tol=-1.0).history
    assert len(h) == 45
    for k, (mu, _, _) in enumerate(h):
        assert mu == pytest.approx(min(1.5 ** k, 1e7) * h[0][0], rel=1e-12)
    assert h[44][0] == h[40][0] == pytest.approx(1e7 * h[0][0], rel=1e-12) and h[39][0] < h[40][0]


# --- stopping rule and special cases ----------------------------------------

def test_stopping_invariant_and_max_iter():
    w = synth.make_preset("w64x64_t20", seed=11)
    X = w.frames.T.astype(np.float64)
    r = O.rpca(X, tol=1e-7)
    assert r.converged and r.resid <= 1e-7
    assert np.linalg.norm(X - r.L - r.S) / np.linalg.norm(X) == pytest.approx(r.resid, rel=1e-6)
    assert r.history[-2][2] > 1e-7            # did not stop early
    r3 = O.rpca(X, tol=1e-7, max_iter=3)
    assert not r3.converged and r3.iters == 3


def test_zero_matrix():
    r = O.rpca(np.zeros((16, 4)))
    assert r.converged and r.iters == 0
    assert not r.L.any() and not r.S.any()


def test_trivial_solution_all_sparse():
    # Spikes in distinct rows and columns: lambda*sgn(X) has spectral norm
    # lambda < 1, which certifies (L, S) = (0, X) as the PCP optimum.
    m, T = 60, 6
    X = np.zeros((m, T))
    for j, (row, v) in enumerate([(3, 5.0), (17, -2.0), (22, 7.0), (40, -1.0), (51, 3.0), (59, 4.0)]):
        X[row, j] = v
    r = O.rpca(X, rho=1.05, tol=1e-12, max_iter=3000)
    assert np.linalg.norm(r.L) <= 1e-6 * np.linalg.norm(X)
    np.testing.assert_allclose(r.S, X, atol=1e-6)


def test_trivial_solution_all_low_rank():
    # X = s u v^T with +-1/sqrt(m), +-1/sqrt(T) entries: u v^T has entries
    # 1/sqrt(mT) < lambda, a certificate that (L, S) = (X, 0) is optimal.
    rng = np.random.default_rng(5)
    m, T = 64, 8
    u = rng.choice([-1.0, 1.0], m) / math.sqrt(m)
    v = rng.choice([-1.0, 1.0], T) / math.sqrt(T)
    X = 10.0 * np.outer(u, v)
    r = O.rpca(X, rho=1.05, tol=1e-12, max_iter=3000)
    assert np.linalg.norm(r.S) <= 1e-6 * np.linalg.norm(X)
    np.testing.assert_allclose(r.L, X, atol=1e-6)


# --- exact recovery and optimality certificate ------------------------------

def _kkt(r):
    """Residuals of the PCP optimality conditions at (L, S) with dual Y."""
    Y, lam = r.Y, r.lam
    supp = r.S != 0
    U, s, Vh = np.linalg.svd(r.L, full_matrices=False)
    k = int(np.sum(s > 1e-9 * s[0]))
    U, V = U[:, :k], Vh[:k].T
    W = Y - U @ V.T
    return dict(
        sign=np.max(np.abs(Y[supp] - lam * np.sign(r.S[supp]))) if supp.any() else 0.0,
        off=np.max(np.abs(Y[~supp])) / lam,
        UtW=np.linalg.norm(U.T @ W), WV=np.linalg.norm(W @ V), W2=np.linalg.norm(W, 2), rank=k)


def test_planted_exact_recovery():
    F, L0, S0 = synth.planted(7, m=400, T=40, rank=2, density=0.05)
    r = O.rpca_frames(F, rho=1.2, tol=1e-10, max_iter=2000)
    assert np.linalg.norm(r.L - L0) / np.linalg.norm(L0) <= 1e-8
    assert np.linalg.norm(r.S - S0) / np.linalg.norm(S0) <= 1e-8
    assert r.rank == 2


def test_kkt_certificate_on_synthetic_window():
    F, _, _ = synth.planted(8, m=400, T=40, rank=2, density=0.05)
    r = O.rpca(F.T, rho=1.05, tol=1e-11, max_iter=3000)
    k = _kkt(r)
    assert k["sign"] < 1e-9 and k["off"] <= 1 + 1e-9
    assert k["UtW"] < 1e-7 and k["WV"] < 1e-7 and k["W2"] < 1.0


def test_bruteforce_8x4_optimality():
    rng = np.random.default_rng(3)
    X = rng.standard_normal((8, 4))
    X[:, 1] = X[:, 0] + 0.01 * rng.standard_normal(8)
    X[2, 3] += 6.0
    r = O.rpca(X, rho=1.05, tol=1e-13, max_iter=5000)
    lam = r.lam

    def f(L, S):
        return np.linalg.svd(L, compute_uv=False).sum() + lam * np.abs(S).sum()

    f0 = f(r.L, r.S)
    for scale in (1e-1, 1e-2, 1e-3):
        D = scale * rng.standard_normal((20000, 8, 4))
        vals = np.array([f(r.L + d, r.S - d) for d in D])
        assert vals.min() >= f0 - 1e-9


# --- symmetries -------------------------------------------------------------

def test_scale_equivariance():
    w = synth.make_preset("w64x64_t20", seed=2)
    X = w.frames.T.astype(np.float64)
    r1 = O.rpca(X)
    r2 = O.rpca(4.0 * X)
    assert r1.iters == r2.iters
    np.testing.assert_allclose(r2.L, 4.0 * r1.L, rtol=0, atol=1e-9 * np.abs(X).max())
    np.testing.assert_allclose(r2.S, 4.0 * r1.S, rtol=0, atol=1e-9 * np.abs(X).max())


def test_frame_permutation_equivariance():
    w = synth.make_preset("w64x64_t20", seed=4)
    X = w.frames.T.astype(np.float64)
    perm = np.random.default_rng(1).permutation(X.shape[1])
    r1 = O.rpca(X)
    r2 = O.rpca(X[:, perm])
    assert r1.iters == r2.iters
    np.testing.assert_allclose(r2.L, r1.L[:, perm], atol=1e-9)
    np.testing.assert_allclose(r2.S, r1.S[:, perm], atol=1e-9)


def test_complex_global_phase_equivariance_and_real_case():
    w = synth.make_window(seed=5, ny=32, nx=32, T=12, n_bound=5, n_free=8, complex_iq=True)
    X = w.frames.T.astype(np.complex128)
    ph = np.exp(0.7j)
    r1 = O.rpca(X)
    r2 = O.rpca(ph * X)
    np.testing.assert_allclose(r2.L, ph * r1.L, atol=1e-9)
    np.testing.assert_allclose(r2.S, ph * r1.S, atol=1e-9)
    Xr = np.real(X)
    rr = O.rpca(Xr)
    rc = O.rpca(Xr.astype(np.complex128))
    np.testing.assert_allclose(rc.L, rr.L, atol=1e-10)
    np.testing.assert_allclose(rc.S, rr.S, atol=1e-10)


# --- Sec. II-F metrics ------------------------------------------------------

def test_rmse_and_dice_hand_values():
    assert O.rmse(np.array([[1.0, 2.0], [3.0, 4.0]]), np.array([[1.0, 0.0], [3.0, 0.0]])) == \
        pytest.approx(math.sqrt((4 + 16) / 4))
    a = np.array([1, 1, 0, 0, 1], bool)
    b = np.array([1, 0, 0, 1, 1], bool)
    assert O.dice(a, b) == pytest.approx(2 * 2 / 6)
    assert O.dice(np.zeros(3, bool), np.zeros(3, bool)) == 1.0
    img = np.array([0.2, 3.0, 1.0, 4.0])
    th = O.mask_threshold(img, np.array([0, 1, 0, 1], bool))
    assert th == pytest.approx(1.75)
    np.testing.assert_array_equal(O.bound_mask(img, th), [False, True, False, True])
    # "at least theta": a pixel exactly at the threshold is in the mask
    np.testing.assert_array_equal(O.bound_mask(np.array([1.0, 0.999, 2.0]), 1.0), [True, False, True])


def test_temporal_mean_abs_hand_values():
    # the image that is binarised (Sec. II-F): per pixel, the mean over frames
    # of the magnitude.  Input (T, m) frame rows, output one value per pixel.
    # Signs cancel in a mean of values (pixel 0 would give 1), not in a mean
    # of magnitudes; a mean over pixels instead of frames gives 3 values.
    real = np.array([[1.0, -2.0], [-3.0, 4.0], [5.0, 0.0]])
    img = O.temporal_mean_abs(real)
    assert img.shape == (2,)
    np.testing.assert_array_equal(img, [3.0, 2.0])
    # complex IQ entries count with their modulus: |3+4i| = 5, |-6-8i| = 10
    cplx = np.array([[3 + 4j, 1j], [-6 - 8j, 0.0]])
    img = O.temporal_mean_abs(cplx)
    assert img.shape == (2,) and img.dtype == np.float64
    np.testing.assert_array_equal(img, [7.5, 0.5])
    # one frame: the magnitudes themselves
    np.testing.assert_array_equal(O.temporal_mean_abs(np.array([[-2.5, 0.0, 7.0]])), [2.5, 0.0, 7.0])


def test_warm_start_from_converged_state_is_a_fixed_point():
    # The ALM iteration is at a fixed point at its own converged (S, Y, mu): one
    # more iteration from there meets the stopping test at once and returns the
    # same L and S (to the tolerance the cold solve stopped at).  A warm start
    # that ignored S0 or Y0 would need more iterations or land elsewhere.
    w = synth.make_window(seed=11, ny=24, nx=24, T=12, n_bound=4, n_free=6)
    X = w.frames.T.astype(np.float64)
    cold = O.rpca(X)
    warm = O.rpca(X, S0=cold.S, Y0=cold.Y, mu_init=cold.mu)
    assert cold.converged and warm.converged and warm.iters == 1
    assert np.linalg.norm(warm.L - cold.L) <= 1e-5 * np.linalg.norm(cold.L)
    assert np.linalg.norm(warm.S - cold.S) <= 1e-5 * np.linalg.norm(cold.S)


def test_warm_start_with_zero_state_is_the_cold_start():
    w = synth.make_window(seed=12, ny=16, nx=16, T=8, n_bound=3, n_free=4)
    X = w.frames.T.astype(np.float64)
    a = O.rpca(X)
    b = O.rpca(X, S0=np.zeros_like(X), Y0=np.zeros_like(X), mu_init=O.initial_mu(X, O.SCHEDULE_IALM))
    assert a.iters == b.iters and np.array_equal(a.L, b.L) and np.array_equal(a.S, b.S)


def test_warm_start_keeps_the_cold_cap():
    # mu_max = 1e7 * mu0 of the cold schedule, whatever mu_init is: started at
    # mu_init = mu0 * 1e7 * 10 the first step uses mu_init, the second the cap.
    w = synth.make_window(seed=13, ny=16, nx=16, T=8, n_bound=3, n_free=4)
    X = w.frames.T.astype(np.float64)
    mu0 = O.initial_mu(X, O.SCHEDULE_IALM)
    r = O.rpca(X, mu_init=mu0 * 1e8, max_iter=2, tol=1e-30)
    assert r.history[0][0] == mu0 * 1e8 and r.history[1][0] == 1e7 * mu0


def test_frames_wrapper_transposes_the_warm_state():
    w = synth.make_window(seed=14, ny=8, nx=8, T=6, n_bound=2, n_free=2)
    X = w.frames.T.astype(np.float64)
    cold = O.rpca(X)
    a = O.rpca(X, S0=cold.S, Y0=cold.Y, mu_init=cold.mu)
    b = O.rpca_frames(w.frames, S0=cold.S.T, Y0=cold.Y.T, mu_init=cold.mu)
    assert np.array_equal(a.L.T, b.L) and np.array_equal(a.S.T, b.S)

