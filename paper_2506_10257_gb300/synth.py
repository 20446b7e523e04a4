"""Seeded synthetic microbubble frame windows (stand-ins for the paper's data).

The paper's inputs are Field II simulations (Sec. II-C, Table I), an agar
phantom (Sec. II-D) and in vivo mouse acquisitions (Sec. II-E); none of them is
available here.  This module draws windows with the same structure the method
relies on (Sec. II-A, Eq. 1): a spatiotemporally coherent background plus
stationary (bound) bubbles that the low-rank part should keep, and moving
(free) bubbles plus thermal noise that the sparse part should take.

Recipe (one window of ``T`` frames of ``ny x nx`` pixels, ``m = ny*nx``):

* background, rank 2: ``B(p,t) = R1(p)*(1 + drift*t/(T-1)) +
  0.01*R2(p)*cos(pi*t/(T-1))`` with R1, R2 Rayleigh(1) magnitudes and
  ``drift = 0.02`` (a slow global gain drift of at most 2 %);
* bound bubbles: ``n_bound`` static isotropic Gaussian blobs, sigma 1.5 px,
  amplitude U[3, 6], uniform centres, rendered out to 4 sigma;
* free bubbles: ``n_free`` blobs of the same shape on straight tracks with
  speed U[vmin, vmax] px/frame and direction U[-pi, pi]; a blob whose centre
  leaves the grid is no longer drawn;
* curved tracks (``accel`` given; the motion model of Sec. II-C): every frame
  each free bubble gets a random acceleration of magnitude U[amin, amax]
  px/frame^2 in a direction U[-pi, pi], and v(t) = v(t-1) + a, x(t) = x(t-1)
  + v(t) (dt = one frame), so tracks bend gradually;
* additive N(0, noise^2) noise, noise = 0.1.

For the complex (IQ) variant every pixel of the background carries one fixed
random phase, every bubble one fixed random phase, and the noise is circular
complex Gaussian with the same per-component standard deviation.

Ground truth: ``L_gt = background + bound blobs``, ``S_gt = free blobs``
(noise belongs to neither), and the bound mask marks pixels where a bound
blob reaches at least half of its own amplitude.

This module holds no step of the decomposition itself; it only draws inputs.
All randomness comes from ``numpy.random.Generator(PCG64(seed))``.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

BLOB_SIGMA = 1.5
BLOB_RADIUS = int(math.ceil(4 * BLOB_SIGMA))  # truncate blobs at 4 sigma


@dataclasses.dataclass
class Window:
    """One synthetic frame window.

    ``frames`` is (T, m): frame t is row t, pixels in row-major image order.
    The Casorati matrix of Sec. II-A is ``X = frames.T`` (m x T).
    """

    frames: np.ndarray          # (T, m) float32 or complex64
    L_gt: np.ndarray            # (T, m) float64 / complex128
    S_gt: np.ndarray            # (T, m) float64 / complex128
    bound_mask_gt: np.ndarray   # (m,) bool
    ny: int
    nx: int
    seed: int

    @property
    def m(self) -> int:
        return self.ny * self.nx

    @property
    def T(self) -> int:
        return self.frames.shape[0]


def _splat(img: np.ndarray, cy: float, cx: float, amp: complex, ny: int, nx: int) -> None:
    """Add one truncated Gaussian blob centred at (cy, cx) into img (ny, nx)."""
    iy0 = int(math.floor(cy)) - BLOB_RADIUS
    ix0 = int(math.floor(cx)) - BLOB_RADIUS
    n = 2 * BLOB_RADIUS + 2
    ys = np.arange(iy0, iy0 + n)
    xs = np.arange(ix0, ix0 + n)
    ys = ys[(ys >= 0) & (ys < ny)]
    xs = xs[(xs >= 0) & (xs < nx)]
    if ys.size == 0 or xs.size == 0:
        return
    dy2 = (ys - cy) ** 2
    dx2 = (xs - cx) ** 2
    r2 = dy2[:, None] + dx2[None, :]
    w = np.exp(-r2 / (2 * BLOB_SIGMA**2))
    w[r2 > (4 * BLOB_SIGMA) ** 2] = 0.0
    img[ys[0]:ys[-1] + 1, xs[0]:xs[-1] + 1] += amp * w


def make_window(
    seed: int,
    ny: int = 64,
    nx: int = 64,
    T: int = 20,
    n_bound: int = 15,
    n_free: int = 30,
    speed: tuple[float, float] = (1.0, 3.0),
    amp: tuple[float, float] = (3.0, 6.0),
    noise: float = 0.1,
    drift: float = 0.02,
    complex_iq: bool = False,
    accel: tuple[float, float] | None = None,
) -> Window:
    """Draw one window; every argument is a recipe parameter (module docstring)."""
    if ny <= 0 or nx <= 0 or T <= 0:
        raise ValueError("ny, nx and T must be positive")
    rng = np.random.Generator(np.random.PCG64(seed))
    m = ny * nx
    cdt = np.complex128 if complex_iq else np.float64
    tn = np.arange(T, dtype=np.float64) / (T - 1) if T > 1 else np.zeros(1)

    r1 = rng.rayleigh(1.0, m)
    r2 = rng.rayleigh(1.0, m)
    bg = (r1[None, :] * (1.0 + drift * tn[:, None])
          + 0.01 * r2[None, :] * np.cos(np.pi * tn)[:, None])
    if complex_iq:
        bg = bg * np.exp(1j * rng.uniform(-np.pi, np.pi, m))[None, :]

    bound_img = np.zeros((ny, nx), dtype=cdt)
    mask = np.zeros((ny, nx), dtype=bool)
    half_r2 = 2 * BLOB_SIGMA**2 * math.log(2.0)   # r^2 where a blob falls to 1/2
    yy, xx = np.mgrid[0:ny, 0:nx]
    for _ in range(n_bound):
        cy = rng.uniform(0, ny)
        cx = rng.uniform(0, nx)
        a = rng.uniform(*amp)
        if complex_iq:
            a = a * np.exp(1j * rng.uniform(-np.pi, np.pi))
        _splat(bound_img, cy, cx, a, ny, nx)
        mask |= ((yy - cy) ** 2 + (xx - cx) ** 2) <= half_r2

    free = np.zeros((T, ny, nx), dtype=cdt)
    for _ in range(n_free):
        cy = rng.uniform(0, ny)
        cx = rng.uniform(0, nx)
        v = rng.uniform(*speed)
        th = rng.uniform(-np.pi, np.pi)
        a = rng.uniform(*amp)
        if complex_iq:
            a = a * np.exp(1j * rng.uniform(-np.pi, np.pi))
        vy, vx = v * math.sin(th), v * math.cos(th)
        if accel is None:
            for t in range(T):
                py, px = cy + vy * t, cx + vx * t
                if not (0 <= py < ny and 0 <= px < nx):
                    break          # left the grid: dropped from here on
                _splat(free[t], py, px, a, ny, nx)
        else:
            py, px = cy, cx
            gone = False
            for t in range(T):
                if t > 0:
                    am = rng.uniform(*accel)
                    ath = rng.uniform(-np.pi, np.pi)
                    vy, vx = vy + am * math.sin(ath), vx + am * math.cos(ath)
                    py, px = py + vy, px + vx
                if gone or not (0 <= py < ny and 0 <= px < nx):
                    gone = True    # left the grid: dropped from here on (draws continue)
                    continue
                _splat(free[t], py, px, a, ny, nx)

    L_gt = bg + bound_img.reshape(1, m)
    S_gt = free.reshape(T, m)
    if complex_iq:
        nz = noise * (rng.standard_normal((T, m)) + 1j * rng.standard_normal((T, m)))
        dt = np.complex64
    else:
        nz = noise * rng.standard_normal((T, m))
        dt = np.float32
    frames = (L_gt + S_gt + nz).astype(dt)
    return Window(frames=frames, L_gt=L_gt, S_gt=S_gt,
                  bound_mask_gt=mask.reshape(m), ny=ny, nx=nx, seed=seed)


# Workload presets: (ny, nx, T, n_bound, n_free, speed) per named workload.
PRESETS = {
    # one 64x64-pixel x 20-frame window (Casorati 4096 x 20)
    "w64x64_t20": dict(ny=64, nx=64, T=20, n_bound=15, n_free=30, speed=(1.0, 3.0)),
    # 512x512-pixel windows (Casorati 262144 x T) with 400 bound / 800 free blobs
    "w512x512_t10": dict(ny=512, nx=512, T=10, n_bound=400, n_free=800, speed=(0.5, 5.0)),
    "w512x512_t20": dict(ny=512, nx=512, T=20, n_bound=400, n_free=800, speed=(0.5, 5.0)),
    "w512x512_t50": dict(ny=512, nx=512, T=50, n_bound=400, n_free=800, speed=(0.5, 5.0)),
    "w512x512_t100": dict(ny=512, nx=512, T=100, n_bound=400, n_free=800, speed=(0.5, 5.0)),
    # a quarter of the 512x512 field (blob counts scaled with the area)
    "w256x256_t50": dict(ny=256, nx=256, T=50, n_bound=100, n_free=200, speed=(0.5, 5.0)),
    "w256x256_t100": dict(ny=256, nx=256, T=100, n_bound=100, n_free=200, speed=(0.5, 5.0)),
    # the paper's own execution-time shape, 338 x 260 pixels (Sec. III-D)
    "w338x260_t20": dict(ny=338, nx=260, T=20, n_bound=200, n_free=400, speed=(0.5, 5.0)),
    "w338x260_t60": dict(ny=338, nx=260, T=60, n_bound=200, n_free=400, speed=(0.5, 5.0)),
    "w338x260_t132": dict(ny=338, nx=260, T=132, n_bound=200, n_free=400, speed=(0.5, 5.0)),
    # curved free-bubble tracks (random per-frame accelerations, Sec. II-C)
    "w64x64_t20_curved": dict(ny=64, nx=64, T=20, n_bound=15, n_free=30, speed=(1.0, 3.0), accel=(0.05, 0.5)),
    "w512x512_t20_curved": dict(ny=512, nx=512, T=20, n_bound=400, n_free=800, speed=(0.5, 5.0),
                                accel=(0.05, 0.5)),
}


def make_preset(name: str, seed: int, complex_iq: bool = False) -> Window:
    return make_window(seed=seed, complex_iq=complex_iq, **PRESETS[name])


def random_dense(seed: int, m: int, T: int, complex_iq: bool = False) -> np.ndarray:
    """Plain N(0,1) frames (T, m) for kernel-level tests with no structure."""
    rng = np.random.Generator(np.random.PCG64(seed))
    if complex_iq:
        return (rng.standard_normal((T, m)) + 1j * rng.standard_normal((T, m))).astype(np.complex64)
    return rng.standard_normal((T, m)).astype(np.float32)


def planted(seed: int, m: int, T: int, rank: int = 2, density: float = 0.05,
            spike: float = 10.0) -> tuple[np.ndarray, np.ndarray, np.ndarray]:
    """Planted low-rank + sparse frames in the exact-recovery regime.

    Returns (frames (T, m) float64, L0 (T, m), S0 (T, m)): L0 = U V^T with
    Gaussian factors scaled to unit-order entries, S0 with a Bernoulli(density)
    support and random-sign entries of magnitude ``spike``.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    U = rng.standard_normal((m, rank))
    V = rng.standard_normal((T, rank))
    L0 = (U @ V.T) / math.sqrt(rank)
    supp = rng.random((m, T)) < density
    S0 = np.where(supp, spike * rng.choice([-1.0, 1.0], size=(m, T)), 0.0)
    return (L0 + S0).T.copy(), L0.T.copy(), S0.T.copy()
