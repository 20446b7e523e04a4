"""CPU FP64 oracle for robust PCA by principal component pursuit (test infrastructure).

TEST INFRASTRUCTURE ONLY.  This module is the slow, plainly written reference
the CUDA solver is checked against.  Only the test-suite, the smoke check and
the benchmark's CPU-baseline leg may import it; the product path never does.
It shares no code with the CUDA path.

Everything follows Sec. II-A of the paper (arXiv 2506.10257), written out
step by step in float64 (complex128 for IQ data) with a full thin SVD from
LAPACK for the singular value thresholding.  The matrix convention is the
paper's: the Casorati matrix ``X`` is (pixels x frames) = (m x T).

Readings taken where the paper is silent or ambiguous (each listed with its
reason in the design notes of the repository):

* lambda defaults to 1/sqrt(max(m, T)) (PCP's standard weight; the paper says
  only that it is "set as explained earlier").
* two penalty schedules: ``"ialm"`` (mu0 = 1.25/||X||_2, mu <- min(rho*mu,
  mu_max), mu_max = 1e7*mu0, rho = 1.5) and ``"fixed_l1"`` (the paper's
  mu = m*T/(4 ||X||_1), held constant, Sec. II-A and II-B).
* L = S = Y = 0 at the start; the steps run in the order L, S, Y, each using
  the newest values (Eq. 4, Eq. 5, Eq. 6 with the freshly updated L and S).
* the stopping test ||X - L - S||_F <= tol*||X||_F (Sec. II-A) is made after
  the Y update with that iteration's residual; ``iters`` counts completed Y
  updates; mu is updated only when the loop goes on.
* shrink maps |x| == gamma to 0; complex entries shrink in magnitude and keep
  their phase (0 stays 0).
"""
from __future__ import annotations

import dataclasses

import numpy as np

SCHEDULE_IALM = "ialm"
SCHEDULE_FIXED_L1 = "fixed_l1"


def shrink(x: np.ndarray, gamma: float) -> np.ndarray:
    """Soft-thresholding operator of Eq. 5: sgn(x) * max(|x| - gamma, 0).

    For complex x, sgn(x) = x/|x| (and 0 at x = 0), so the magnitude shrinks
    and the phase is kept.
    """
    x = np.asarray(x)
    mag = np.abs(x)
    keep = np.maximum(mag - gamma, 0.0)
    if np.iscomplexobj(x):
        out = np.zeros_like(x)
        nz = mag > 0
        out[nz] = x[nz] / mag[nz] * keep[nz]
        return out
    return np.sign(x) * keep


def svt(M: np.ndarray, tau: float) -> tuple[np.ndarray, int]:
    """Singular value thresholding D_tau(M) = U max(Lambda - tau, 0) V^* (Eq. 4).

    Uses the full thin SVD of M.  Returns (D_tau(M), number of singular values
    above tau).
    """
    U, sig, Vh = np.linalg.svd(M, full_matrices=False)
    kept = np.maximum(sig - tau, 0.0)
    r = int(np.count_nonzero(kept > 0))
    return (U[:, :r] * kept[:r]) @ Vh[:r, :], r


def spectral_norm(X: np.ndarray) -> float:
    """||X||_2, the largest singular value (LAPACK SVD)."""
    return float(np.linalg.svd(X, compute_uv=False)[0])


def default_lambda(m: int, T: int) -> float:
    """lambda = 1/sqrt(max(m, T)), the PCP weight the paper inherits from Candes et al."""
    return 1.0 / np.sqrt(max(m, T))


@dataclasses.dataclass
class Result:
    L: np.ndarray
    S: np.ndarray
    Y: np.ndarray
    iters: int
    resid: float        # ||X - L - S||_F / ||X||_F at the last iteration
    converged: bool
    rank: int           # singular values kept by the last SVT step
    mu: float           # penalty used by the last iteration
    lam: float
    history: list       # per-iteration (mu, rank, relative residual)


def initial_mu(X: np.ndarray, schedule: str, mu0_scale: float = 1.25) -> float:
    """Starting penalty.

    ``ialm``: mu0 = mu0_scale / ||X||_2.
    ``fixed_l1``: mu = n1*n2 / (4 ||X||_1) with n1 x n2 the size of X and
    ||X||_1 the entrywise l1 norm (Sec. II-A).
    """
    if schedule == SCHEDULE_IALM:
        return mu0_scale / spectral_norm(X)
    if schedule == SCHEDULE_FIXED_L1:
        m, T = X.shape
        return m * T / (4.0 * float(np.sum(np.abs(X))))
    raise ValueError(f"unknown schedule {schedule!r}")


def rpca(
    X: np.ndarray,
    lam: float | None = None,
    schedule: str = SCHEDULE_IALM,
    mu0_scale: float = 1.25,
    rho: float = 1.5,
    mu_max_factor: float = 1e7,
    tol: float = 1e-7,
    max_iter: int = 500,
    S0: np.ndarray | None = None,
    Y0: np.ndarray | None = None,
    mu_init: float | None = None,
) -> Result:
    """Principal component pursuit (Eq. 2) by the augmented-Lagrangian iteration.

    Per iteration k (Sec. II-A, steps 1-3):
      Eq. 4:  L = D_{1/mu}(X - S + Y/mu)
      Eq. 5:  S = shrink_{lam/mu}(X - L + Y/mu)
      Eq. 6:  Y = Y + mu (X - L - S)
      stop when ||X - L - S||_F <= tol ||X||_F (tested after Eq. 6);
      else, under ``ialm``, mu = min(rho*mu, mu_max).

    ``S0``, ``Y0`` and ``mu_init`` give a warm start (all three default to the
    cold start S = Y = 0 and the schedule's first mu).  The paper has no warm
    start; the reading taken: the cap mu_max = mu_max_factor * mu0 stays the
    cold schedule's (mu0 from this X) whatever mu_init is.
    """
    X = np.asarray(X)
    X = X.astype(np.complex128 if np.iscomplexobj(X) else np.float64)
    m, T = X.shape
    if lam is None or lam <= 0:
        lam = default_lambda(m, T)
    normX = float(np.linalg.norm(X))
    S = np.zeros_like(X) if S0 is None else np.array(S0, dtype=X.dtype)
    Y = np.zeros_like(X) if Y0 is None else np.array(Y0, dtype=X.dtype)
    L = np.zeros_like(X)
    if normX == 0.0:
        return Result(L, S, Y, 0, 0.0, True, 0, 0.0, lam, [])
    mu0 = initial_mu(X, schedule, mu0_scale)
    mu = mu0 if mu_init is None else float(mu_init)
    mu_max = mu_max_factor * mu0
    history = []
    resid = np.inf
    rank = 0
    for k in range(1, max_iter + 1):
        if k > 1 and schedule == SCHEDULE_IALM:
            mu = min(rho * mu, mu_max)                     # penalty growth
        L, rank = svt(X - S + Y / mu, 1.0 / mu)           # Eq. 4
        S = shrink(X - L + Y / mu, lam / mu)               # Eq. 5
        E = X - L - S
        Y = Y + mu * E                                     # Eq. 6
        resid = float(np.linalg.norm(E)) / normX
        history.append((mu, rank, resid))
        if resid <= tol:                                   # stopping rule, Sec. II-A
            return Result(L, S, Y, k, resid, True, rank, mu, lam, history)
    return Result(L, S, Y, max_iter, resid, False, rank, mu, lam, history)


def rpca_frames(frames: np.ndarray, **kw) -> Result:
    """Same as ``rpca`` on the Casorati matrix X = frames.T of a (T, m) window.

    The returned L, S, Y are transposed back to (T, m) frame rows; a warm
    start's S0 and Y0 are given as (T, m) frame rows too.
    """
    for k in ("S0", "Y0"):
        if kw.get(k) is not None:
            kw[k] = np.asarray(kw[k]).T
    r = rpca(np.asarray(frames).T, **kw)
    r.L, r.S, r.Y = r.L.T, r.S.T, r.Y.T
    return r


# --- evaluation (Sec. II-F) -------------------------------------------------

def rmse(est: np.ndarray, gt: np.ndarray) -> float:
    """Eq. 7: root-mean-square difference over every pixel of every frame."""
    d = np.asarray(est) - np.asarray(gt)
    return float(np.sqrt(np.mean(np.abs(d) ** 2)))


def dice(a: np.ndarray, b: np.ndarray) -> float:
    """Eq. 8: 2|A n B| / (|A| + |B|) of two binary images (1.0 when both are empty)."""
    a = np.asarray(a, dtype=bool)
    b = np.asarray(b, dtype=bool)
    den = int(a.sum()) + int(b.sum())
    if den == 0:
        return 1.0
    return 2.0 * int(np.logical_and(a, b).sum()) / den


def temporal_mean_abs(frames_like: np.ndarray) -> np.ndarray:
    """Per-pixel mean over frames of |value|: the image that is binarised.

    Input (T, m); output (m,).
    """
    return np.mean(np.abs(np.asarray(frames_like, dtype=np.complex128
                                     if np.iscomplexobj(frames_like) else np.float64)), axis=0)


def mask_threshold(image: np.ndarray, gt_core: np.ndarray) -> float:
    """Binarisation threshold (Sec. II-F): based on the mean intensity at the
    ground-truth bubble pixels; this build takes half of that mean."""
    gt_core = np.asarray(gt_core, dtype=bool)
    if not gt_core.any():
        raise ValueError("ground-truth mask is empty")
    return 0.5 * float(np.mean(np.asarray(image)[gt_core]))


def bound_mask(image: np.ndarray, theta: float) -> np.ndarray:
    """Binary image: pixels whose intensity is at least theta."""
    return np.asarray(image) >= theta
