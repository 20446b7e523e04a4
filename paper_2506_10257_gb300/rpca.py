"""Python binding of librpca.so (ctypes; argument marshalling only).

Every step of the solve runs in the CUDA library.  PyTorch provides device
memory (the workspace, outputs) and streams.  There is no CPU fallback: if
the library is missing or no GPU is present, these calls raise.

Layout convention: a window is a (T, m) tensor of frames (frame t is row t,
pixels contiguous), which is the frame-major Casorati matrix X (m x T) of the
C ABI.
"""
from __future__ import annotations

import ctypes
import os

from . import build as _build

# ---- C ABI mirrors (include/rpca.h) ----------------------------------------
OK, NOT_CONVERGED, PENDING = 0, 1, 2
ERR_ARG, ERR_CUDA, ERR_NOMEM, ERR_BUDGET, ERR_TIMEOUT, ERR_NONFINITE, ERR_UNSUPPORTED, ERR_NOTFOUND = \
    -1, -2, -3, -4, -5, -6, -7, -8
R32, C64 = 0, 1
PREC_FP32, PREC_TF32X3, PREC_BF16X3, PREC_TF32 = 0, 1, 2, 3
MU_IALM, MU_FIXED_L1 = 0, 1
DRIVE_GRAPH, DRIVE_HOST, DRIVE_STREAM = 0, 1, 2
MAX_T = 224
MAX_T_NARROW = 32

EXPORTED = ["rpca_params_default", "rpca_workspace_size", "rpca_plan_create", "rpca_solve", "rpca_solve_host",
            "rpca_plan_result", "rpca_plan_destroy", "rpca_status_str", "rpca_gram", "rpca_eig",
            "rpca_gram_noalloc", "rpca_plan_timings", "rpca_batch_create", "rpca_batch_solve",
            "rpca_batch_solve_host", "rpca_batch_tune", "rpca_batch_set_schedule", "rpca_batch_info", "rpca_batch_window_ctas", "rpca_batch_destroy", "rpca_batch_schedule",
            "rpca_server_create", "rpca_server_set_warm", "rpca_submit", "rpca_poll", "rpca_server_wait",
            "rpca_server_stats", "rpca_server_destroy", "rpca_prefilter_scratch_bytes", "rpca_prefilter",
            "rpca_prefilter_highpass", "rpca_step_begin", "rpca_step_run", "rpca_step_sums", "rpca_step_done"]


class Params(ctypes.Structure):
    _fields_ = [("m", ctypes.c_int64), ("T", ctypes.c_int32), ("dtype", ctypes.c_int32),
                ("precision", ctypes.c_int32), ("mu_schedule", ctypes.c_int32),
                ("drive", ctypes.c_int32), ("max_iter", ctypes.c_int32),
                ("lambda_", ctypes.c_double), ("mu0_scale", ctypes.c_double),
                ("rho", ctypes.c_double), ("mu_max_factor", ctypes.c_double),
                ("tol", ctypes.c_double), ("warm_start", ctypes.c_int32), ("sharded", ctypes.c_int32),
                ("mu_init", ctypes.c_double), ("mu_prev_scale", ctypes.c_double)]


class Result(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int32), ("iters", ctypes.c_int32), ("rank", ctypes.c_int32),
                ("sweeps", ctypes.c_int32), ("resid", ctypes.c_double), ("mu", ctypes.c_double),
                ("normX", ctypes.c_double), ("lambda_", ctypes.c_double), ("pass_us", ctypes.c_double),
                ("eig_us", ctypes.c_double), ("init_us", ctypes.c_double), ("passes_timed", ctypes.c_int32),
                ("eigs_timed", ctypes.c_int32)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class Window(ctypes.Structure):
    _fields_ = [("X", ctypes.c_void_p), ("L", ctypes.c_void_p), ("S", ctypes.c_void_p),
                ("mask", ctypes.c_void_p), ("theta", ctypes.c_float), ("pad_", ctypes.c_int32)]


class RpcaError(RuntimeError):
    def __init__(self, status, what=""):
        self.status = status
        super().__init__(f"{what}: {status_str(status)} ({status})")


_lib = None


def lib_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Load librpca.so (building it first if asked); raise if it cannot be loaded."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.LIB
    if not os.path.exists(path):
        if not build_if_missing:
            raise RuntimeError(f"CUDA library not built: {path}")
        _build.build()
    lib = ctypes.CDLL(path)
    vp, i32, i64, f32 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_float
    lib.rpca_params_default.argtypes = [ctypes.POINTER(Params), i64, i32]
    lib.rpca_workspace_size.argtypes = [ctypes.POINTER(Params), ctypes.POINTER(ctypes.c_size_t)]
    lib.rpca_plan_create.argtypes = [ctypes.POINTER(Params), vp, ctypes.c_size_t, ctypes.POINTER(vp)]
    lib.rpca_solve.argtypes = [vp, vp, vp, vp, vp, f32, vp, ctypes.POINTER(Result)]
    lib.rpca_solve_host.argtypes = [vp, vp, vp, vp, vp, f32, vp, ctypes.POINTER(Result)]
    lib.rpca_plan_result.argtypes = [vp, ctypes.POINTER(Result)]
    lib.rpca_plan_destroy.argtypes = [vp]
    lib.rpca_plan_destroy.restype = None
    lib.rpca_status_str.argtypes = [i32]
    lib.rpca_status_str.restype = ctypes.c_char_p
    lib.rpca_gram.argtypes = [vp, i64, i32, vp, vp, i32, vp]
    lib.rpca_eig.argtypes = [vp, i32, vp, vp, vp]
    lib.rpca_gram_noalloc.argtypes = [vp, i64, i32, vp, vp, vp]
    lib.rpca_step_begin.argtypes = [vp, vp, vp, vp, vp, f32, vp]
    lib.rpca_step_run.argtypes = [vp, i32, vp]
    lib.rpca_step_sums.argtypes = [vp, ctypes.POINTER(ctypes.POINTER(ctypes.c_double)),
                                   ctypes.POINTER(ctypes.POINTER(ctypes.c_double))]
    lib.rpca_step_done.argtypes = [vp, ctypes.POINTER(i32), ctypes.POINTER(Result), vp]
    lib.rpca_prefilter_scratch_bytes.argtypes = [i64, i32]
    lib.rpca_prefilter_scratch_bytes.restype = ctypes.c_size_t
    lib.rpca_prefilter.argtypes = [vp, i64, i32, ctypes.c_double, i32, vp, vp, vp, vp, vp, vp]
    lib.rpca_prefilter_highpass.argtypes = [vp, i64, i32, ctypes.c_double, i32, vp, vp, vp, vp, vp, vp]
    lib.rpca_plan_timings.argtypes = [vp, ctypes.POINTER(ctypes.c_double), i32]
    lib.rpca_batch_create.argtypes = [ctypes.POINTER(Params), i32, ctypes.POINTER(vp)]
    lib.rpca_batch_solve.argtypes = [vp, ctypes.POINTER(Window), vp, ctypes.POINTER(Result)]
    lib.rpca_batch_solve_host.argtypes = [vp, ctypes.POINTER(Window), vp, ctypes.POINTER(Result)]
    lib.rpca_batch_tune.argtypes = [vp, ctypes.POINTER(Window), vp, i32, ctypes.POINTER(ctypes.c_double)]
    lib.rpca_batch_set_schedule.argtypes = [vp, i32, ctypes.c_double, i32, i32]
    lib.rpca_batch_info.argtypes = [vp, ctypes.POINTER(i32), i32]
    lib.rpca_batch_window_ctas.argtypes = [vp, ctypes.POINTER(i32), i32]
    lib.rpca_batch_schedule.argtypes = [i32, vp, vp, vp, i32, i32, ctypes.c_double, ctypes.POINTER(i32), vp, vp, vp]
    lib.rpca_batch_destroy.argtypes = [vp]
    lib.rpca_batch_destroy.restype = None
    lib.rpca_server_create.argtypes = [ctypes.c_size_t, i32, ctypes.POINTER(vp)]
    lib.rpca_server_set_warm.argtypes = [vp, i32, ctypes.c_double, i32]
    lib.rpca_submit.argtypes = [vp, ctypes.POINTER(Params), vp, vp, vp, vp, f32, i32, ctypes.POINTER(ctypes.c_uint64)]
    lib.rpca_poll.argtypes = [vp, ctypes.c_uint64, ctypes.POINTER(Result)]
    lib.rpca_server_wait.argtypes = [vp, ctypes.c_uint64, ctypes.POINTER(Result)]
    lib.rpca_server_stats.argtypes = [vp, ctypes.POINTER(i64), i32]
    lib.rpca_server_destroy.argtypes = [vp]
    lib.rpca_server_destroy.restype = None
    _lib = lib
    return lib


def status_str(st: int) -> str:
    return load().rpca_status_str(st).decode()


def default_params(m: int, T: int, **kw) -> Params:
    p = Params()
    load().rpca_params_default(ctypes.byref(p), int(m), int(T))
    for k, v in kw.items():
        if k == "lam":
            k = "lambda_"
        if not hasattr(p, k):
            raise TypeError(f"unknown parameter {k}")
        setattr(p, k, v)
    return p


def _torch():
    import torch
    if not torch.cuda.is_available():
        raise RuntimeError("rpca needs a CUDA device (no CPU fallback)")
    return torch


def _check_like(frames, **bufs):
    """Output (and warm-state) buffers must be contiguous CUDA tensors of the frames' dtype and shape."""
    _torch()
    for name, t in bufs.items():
        if (t.dtype != frames.dtype or not t.is_cuda or not t.is_contiguous()
                or tuple(t.shape) != tuple(frames.shape)):
            raise ValueError(f"{name} must be a contiguous {frames.dtype} CUDA tensor of shape {tuple(frames.shape)}")


def _stream_handle(stream):
    torch = _torch()
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


class Plan:
    """A solver plan for windows of shape (T, m); owns a torch workspace."""

    def __init__(self, m: int, T: int, **kw):
        torch = _torch()
        self.lib = load()
        self.params = default_params(m, T, **kw)
        nbytes = ctypes.c_size_t()
        st = self.lib.rpca_workspace_size(ctypes.byref(self.params), ctypes.byref(nbytes))
        if st != OK:
            raise RpcaError(st, "rpca_workspace_size")
        self.workspace = torch.empty(max(nbytes.value, 256), dtype=torch.uint8, device="cuda")
        h = ctypes.c_void_p()
        st = self.lib.rpca_plan_create(ctypes.byref(self.params), ctypes.c_void_p(self.workspace.data_ptr()),
                                       nbytes.value, ctypes.byref(h))
        if st != OK:
            raise RpcaError(st, "rpca_plan_create")
        self.handle = h
        self.m, self.T = int(m), int(T)

    def close(self):
        if getattr(self, "handle", None):
            self.lib.rpca_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def solve(self, frames, L=None, S=None, mask=None, theta: float = 0.0, stream=None, wait: bool = True):
        """Solve one window.  frames: (T, m) float32 CUDA tensor.

        Returns (L, S, result) where result is a dict (None when wait=False).
        """
        torch = _torch()
        want = torch.complex64 if self.params.dtype == C64 else torch.float32
        if frames.dtype != want or not frames.is_cuda or not frames.is_contiguous():
            raise ValueError(f"frames must be a contiguous {want} CUDA tensor")
        if tuple(frames.shape) != (self.T, self.m):
            raise ValueError(f"frames shape {tuple(frames.shape)} != {(self.T, self.m)}")
        if L is None:
            L = torch.empty_like(frames)
        if S is None:
            S = torch.empty_like(frames)
        _check_like(frames, L=L, S=S)
        res = Result()
        st = self.lib.rpca_solve(self.handle, ctypes.c_void_p(frames.data_ptr()), ctypes.c_void_p(L.data_ptr()),
                                 ctypes.c_void_p(S.data_ptr()),
                                 ctypes.c_void_p(mask.data_ptr() if mask is not None else 0),
                                 ctypes.c_float(theta), _stream_handle(stream),
                                 ctypes.byref(res) if wait else None)
        if st < 0:
            raise RpcaError(st, "rpca_solve")
        return L, S, (res.as_dict() if wait else None)

    def solve_host(self, frames, L=None, S=None, mask=None, theta: float = 0.0, stream=None):
        """Solve a window held in HOST memory (numpy arrays or CPU tensors, (T, m) float32).

        The C library copies it to the device, solves, and copies L, S (and the
        mask) back into the given host buffers.  Returns (L, S, result)."""
        import numpy as np
        F = np.ascontiguousarray(np.asarray(frames), dtype=np.complex64 if self.params.dtype == C64 else np.float32)
        if F.shape != (self.T, self.m):
            raise ValueError(f"frames shape {F.shape} != {(self.T, self.m)}")
        if L is None:
            L = np.empty_like(F)
        if S is None:
            S = np.empty_like(F)
        res = Result()
        st = self.lib.rpca_solve_host(self.handle, ctypes.c_void_p(F.ctypes.data), ctypes.c_void_p(L.ctypes.data),
                                      ctypes.c_void_p(S.ctypes.data),
                                      ctypes.c_void_p(mask.ctypes.data if mask is not None else 0),
                                      ctypes.c_float(theta), _stream_handle(stream), ctypes.byref(res))
        if st < 0:
            raise RpcaError(st, "rpca_solve_host")
        return L, S, res.as_dict()

    def timings(self) -> dict:
        """Device-timer breakdown of the eigen-steps of the last solve (microseconds)."""
        buf = (ctypes.c_double * 9)()
        st = self.lib.rpca_plan_timings(self.handle, buf, 9)
        if st != OK:
            raise RpcaError(st, "rpca_plan_timings")
        keys = ["eig_load_us", "eig_sweeps_us", "eig_rotprod_us", "eig_basis_us", "eig_rounds", "eigs_timed",
                "pass_work_us", "pass_red1_us", "pass_red2_us"]
        return dict(zip(keys, list(buf)))

    def result(self) -> dict:
        res = Result()
        st = self.lib.rpca_plan_result(self.handle, ctypes.byref(res))
        if st != OK:
            raise RpcaError(st, "rpca_plan_result")
        return res.as_dict()


def solve(frames, **kw):
    """One-shot solve of a (T, m) CUDA window; returns (L, S, result)."""
    T, m = frames.shape
    mask = kw.pop("mask", None)
    theta = kw.pop("theta", 0.0)
    if str(frames.dtype) == "torch.complex64":
        kw.setdefault("dtype", C64)
    plan = Plan(m, T, **kw)
    try:
        return plan.solve(frames, mask=mask, theta=theta)
    finally:
        plan.close()


def gram(frames, V=None, precision: int = PREC_FP32):
    """G = (Z V)^T (Z V) with Z = frames.T; returns a (T, T) float64 CUDA tensor."""
    torch = _torch()
    T, m = frames.shape
    G = torch.empty((T, T), dtype=torch.float64, device="cuda")
    vptr = 0
    if V is not None:
        V = V.to(device="cuda", dtype=torch.float32).contiguous()
        vptr = V.data_ptr()
    st = load().rpca_gram(ctypes.c_void_p(frames.data_ptr()), m, T, ctypes.c_void_p(vptr),
                          ctypes.c_void_p(G.data_ptr()), precision, _stream_handle(None))
    if st != OK:
        raise RpcaError(st, "rpca_gram")
    return G


def eig(G):
    """Eigen-decomposition of a symmetric (T, T) float64 CUDA tensor (FP64 Jacobi).

    Returns (evals descending, evecs as columns)."""
    torch = _torch()
    G = G.to(device="cuda", dtype=torch.float64).contiguous()
    T = G.shape[0]
    ev = torch.empty(T, dtype=torch.float64, device="cuda")
    V = torch.empty((T, T), dtype=torch.float64, device="cuda")
    st = load().rpca_eig(ctypes.c_void_p(G.data_ptr()), T, ctypes.c_void_p(ev.data_ptr()),
                         ctypes.c_void_p(V.data_ptr()), _stream_handle(None))
    if st != OK:
        raise RpcaError(st, "rpca_eig")
    return ev, V


def gram_noalloc(frames, V=None, G=None, stream=None):
    """Same Gram as ``gram`` through rpca_gram_noalloc, which allocates no device
    memory (its scratch is a fixed array inside the library).  The output G
    (T, T) float64 is allocated here by the caller side unless given.  The call
    is asynchronous on `stream` (default: the current stream)."""
    torch = _torch()
    T, m = frames.shape
    s = stream if stream is not None else torch.cuda.current_stream()
    if G is None:
        G = torch.empty((T, T), dtype=torch.float64, device="cuda")
    vptr = 0
    if V is not None:
        V2 = V.to(device="cuda", dtype=torch.float32).contiguous()
        if V2.data_ptr() != V.data_ptr() and s != torch.cuda.current_stream():
            # a converted copy lives in the current stream's pool: keep it from
            # being reused before the kernels on `s` have read it
            V2.record_stream(s)
        V = V2
        vptr = V.data_ptr()
    st = load().rpca_gram_noalloc(ctypes.c_void_p(frames.data_ptr()), m, T, ctypes.c_void_p(vptr),
                                  ctypes.c_void_p(G.data_ptr()), ctypes.c_void_p(s.cuda_stream))
    if st != OK:
        raise RpcaError(st, "rpca_gram_noalloc")
    return G


def prefilter_buffers(frames, window: int = 20):
    """Device buffers of a prefilter call on (T, m) frames: (Y, kept, count, corr, scratch)."""
    torch = _torch()
    T, m = frames.shape
    Y = torch.empty((max(T - window + 1, 0), m), dtype=torch.float32, device=frames.device)
    kept = torch.empty(T, dtype=torch.int32, device=frames.device)
    count = torch.zeros(2, dtype=torch.int32, device=frames.device)
    corr = torch.zeros(max(T - 1, 0), dtype=torch.float64, device=frames.device)
    scratch = torch.empty(max(int(load().rpca_prefilter_scratch_bytes(m, T)), 8), dtype=torch.uint8,
                          device=frames.device)
    return Y, kept, count, corr, scratch


def prefilter(frames, corr_min: float = 0.8, window: int = 20, stream=None, wait: bool = True, out=None,
              high_pass: bool = False):
    """Frame pre-filter of the in vivo reference (rpca_prefilter): frames that
    correlate below corr_min with every neighbour are dropped, then a whole-window
    moving average of `window` frames runs over the kept frames (with high_pass,
    rpca_prefilter_highpass: the window's centre frame minus that average).  frames: (T, m)
    float32 CUDA tensor.  Returns (Y, kept, corr): Y (n, m) float32 with
    n = max(K - window + 1, 0), kept (K,) int32 indices, corr (T - 1,) float64.
    With wait=False the full-size buffers and the device counts are returned
    instead: (Y_full, kept_full, corr, count).  out: buffers from an earlier
    call's prefilter_buffers(frames, window), reused (no allocation)."""
    torch = _torch()
    if frames.dim() != 2 or frames.dtype != torch.float32 or not frames.is_cuda or not frames.is_contiguous():
        raise ValueError("frames must be a contiguous (T, m) float32 CUDA tensor")
    T, m = frames.shape
    lib = load()
    Y, kept, count, corr, scratch = out if out is not None else prefilter_buffers(frames, window)
    fn = lib.rpca_prefilter_highpass if high_pass else lib.rpca_prefilter
    st = fn(ctypes.c_void_p(frames.data_ptr()), m, T, float(corr_min), int(window),
                            ctypes.c_void_p(Y.data_ptr() if Y.numel() else frames.data_ptr()),
                            ctypes.c_void_p(kept.data_ptr()), ctypes.c_void_p(count.data_ptr()),
                            ctypes.c_void_p(corr.data_ptr() if corr.numel() else 0),
                            ctypes.c_void_p(scratch.data_ptr()), _stream_handle(stream))
    if st != OK:
        raise RpcaError(st, "rpca_prefilter_highpass" if high_pass else "rpca_prefilter")
    if not wait:
        return Y, kept, corr, count
    torch.cuda.current_stream().synchronize() if stream is None else stream.synchronize()
    K, n = (int(v) for v in count.cpu().tolist())
    return Y[:n], kept[:K], corr


def batch_schedule(shapes, ctas: int, lanes: int, alpha: float = 1.0, max_ctas=None):
    """The batch form's CTA schedule (rpca_batch_schedule, host only) for
    windows of shapes [(m, T), ...] on `ctas` resident CTAs: a list of
    (lane CTAs, [window indices in run order]) per lane."""
    import numpy as np
    n = len(shapes)
    m = np.ascontiguousarray([s[0] for s in shapes], dtype=np.int64)
    T = np.ascontiguousarray([s[1] for s in shapes], dtype=np.int32)
    cap = None if max_ctas is None else np.ascontiguousarray(max_ctas, dtype=np.int32)
    nl = ctypes.c_int32()
    lc, order, end = (np.zeros(max(n, 1), dtype=np.int32) for _ in range(3))
    st = load().rpca_batch_schedule(n, m.ctypes.data if n else None, T.ctypes.data if n else None,
                                    cap.ctypes.data if cap is not None else None, int(ctas), int(lanes),
                                    float(alpha), ctypes.byref(nl), lc.ctypes.data, order.ctypes.data,
                                    end.ctypes.data)
    if st != OK:
        raise RpcaError(st, "rpca_batch_schedule")
    out, k = [], 0
    for l in range(nl.value):
        out.append((int(lc[l]), [int(w) for w in order[k:end[l]]]))
        k = int(end[l])
    return out


class Batch:
    """Many windows of uneven (T, m) shapes solved by one persistent launch.

    shapes: list of (m, T); kw: parameters applied to every window, or
    params: a list of per-window keyword dicts."""

    def __init__(self, shapes, params=None, **kw):
        _torch()
        self.lib = load()
        self.shapes = [(int(m), int(T)) for m, T in shapes]
        n = len(self.shapes)
        if n < 1:
            raise ValueError("a batch needs at least one window")
        arr = (Params * n)()
        for i, (m, T) in enumerate(self.shapes):
            extra = dict(kw)
            if params is not None:
                extra.update(params[i])
            arr[i] = default_params(m, T, **extra)
        h = ctypes.c_void_p()
        st = self.lib.rpca_batch_create(arr, n, ctypes.byref(h))
        if st != OK:
            raise RpcaError(st, "rpca_batch_create")
        self.handle = h
        self.n = n

    def close(self):
        if getattr(self, "handle", None):
            self.lib.rpca_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _windows(self, frames, Ls, Ss, masks, thetas):
        torch = _torch()
        if len(frames) != self.n:
            raise ValueError(f"expected {self.n} windows, got {len(frames)}")
        w = (Window * self.n)()
        for i, F in enumerate(frames):
            m, T = self.shapes[i]
            if (F.dtype not in (torch.float32, torch.complex64) or not F.is_cuda or not F.is_contiguous()
                    or tuple(F.shape) != (T, m)):
                raise ValueError(f"window {i}: need a contiguous float32 or complex64 CUDA tensor of shape {(T, m)}")
            _check_like(F, L=Ls[i], S=Ss[i])
            w[i].X = F.data_ptr()
            w[i].L = Ls[i].data_ptr()
            w[i].S = Ss[i].data_ptr()
            w[i].mask = masks[i].data_ptr() if masks is not None and masks[i] is not None else 0
            w[i].theta = float(thetas[i]) if thetas is not None else 0.0
        return w

    def solve(self, frames, Ls=None, Ss=None, masks=None, thetas=None, stream=None, wait: bool = True):
        """Solve every window; returns (Ls, Ss, results) (results None when wait=False)."""
        torch = _torch()
        if Ls is None:
            Ls = [torch.empty_like(F) for F in frames]
        if Ss is None:
            Ss = [torch.empty_like(F) for F in frames]
        w = self._windows(frames, Ls, Ss, masks, thetas)
        res = (Result * self.n)()
        st = self.lib.rpca_batch_solve(self.handle, w, _stream_handle(stream), res if wait else None)
        if st < 0:
            raise RpcaError(st, "rpca_batch_solve")
        self._keep = (frames, Ls, Ss, masks)
        return Ls, Ss, ([r.as_dict() for r in res] if wait else None)

    def solve_host(self, frames, Ls, Ss, masks=None, thetas=None, stream=None, wait: bool = True):
        """Solve windows held in HOST memory through rpca_batch_solve_host.

        frames, Ls, Ss (and masks): per window a contiguous CPU tensor (pinned
        for full copy speed) of the window's shape, (T, m) float32 or complex64
        (masks: (m,) uint8).  The library uploads, solves in one persistent
        launch and downloads into Ls, Ss, masks.  With wait=False the call
        returns once enqueued (the buffers must stay untouched until a later
        call with wait=True returns) and results is None."""
        import torch
        if len(frames) != self.n:
            raise ValueError(f"expected {self.n} windows, got {len(frames)}")
        w = (Window * self.n)()
        for i, F in enumerate(frames):
            m, T = self.shapes[i]
            for name, t in (("frames", F), ("L", Ls[i]), ("S", Ss[i])):
                if (t.device.type != "cpu" or not t.is_contiguous() or tuple(t.shape) != (T, m)
                        or t.dtype not in (torch.float32, torch.complex64) or t.dtype != F.dtype):
                    raise ValueError(f"window {i}: {name} must be a contiguous CPU tensor of shape {(T, m)}")
            w[i].X = F.data_ptr()
            w[i].L = Ls[i].data_ptr()
            w[i].S = Ss[i].data_ptr()
            if masks is not None and masks[i] is not None:
                if masks[i].device.type != "cpu" or masks[i].numel() != m or masks[i].dtype != torch.uint8:
                    raise ValueError(f"window {i}: mask must be a ({m},) uint8 CPU tensor")
                w[i].mask = masks[i].data_ptr()
            w[i].theta = float(thetas[i]) if thetas is not None else 0.0
        res = (Result * self.n)()
        st = self.lib.rpca_batch_solve_host(self.handle, w, _stream_handle(stream), res if wait else None)
        if st < 0:
            raise RpcaError(st, "rpca_batch_solve_host")
        return [r.as_dict() for r in res] if wait else None

    def tune(self, frames, reps: int = 3, stream=None) -> float:
        """Autotune the CTA schedule on these windows; returns the best median ms per batch solve."""
        torch = _torch()
        Ls = [torch.empty_like(F) for F in frames]
        Ss = [torch.empty_like(F) for F in frames]
        w = self._windows(frames, Ls, Ss, None, None)
        best = ctypes.c_double()
        st = self.lib.rpca_batch_tune(self.handle, w, _stream_handle(stream), int(reps), ctypes.byref(best))
        if st != OK:
            raise RpcaError(st, "rpca_batch_tune")
        return best.value

    def set_schedule(self, lanes: int, alpha: float = 1.0, ctas_per_sm: int = 1, paired: bool = True):
        """Set the CTA schedule by hand (rpca_batch_set_schedule)."""
        st = self.lib.rpca_batch_set_schedule(self.handle, int(lanes), float(alpha), int(ctas_per_sm), int(bool(paired)))
        if st != OK:
            raise RpcaError(st, "rpca_batch_set_schedule")

    def info(self) -> dict:
        buf = (ctypes.c_int32 * 7)()
        st = self.lib.rpca_batch_info(self.handle, buf, 7)
        if st != OK:
            raise RpcaError(st, "rpca_batch_info")
        keys = ["grid", "lanes", "ctas_per_sm", "alpha_milli", "occ_max", "graph", "paired"]
        out = dict(zip(keys, list(buf)))
        ctas = (ctypes.c_int32 * self.n)()
        if self.lib.rpca_batch_window_ctas(self.handle, ctas, self.n) == OK:
            out["window_ctas"] = list(ctas)
        return out


class Server:
    """Served form: sliding windows of several probes, continuous batching over
    CUDA streams, per-probe warm-start state on the device, HBM admission."""

    STATS = ["bytes", "peak_bytes", "budget", "queued", "running", "peak_running", "started", "finished",
             "evicted", "refused"]

    def __init__(self, hbm_budget_bytes: int = 120 * 10**9, max_slots: int = 8, warm: bool = False,
                 warm_mu_scale: float = 0.1, cold_every: int = 0):
        _torch()
        self.lib = load()
        h = ctypes.c_void_p()
        st = self.lib.rpca_server_create(int(hbm_budget_bytes), int(max_slots), ctypes.byref(h))
        if st != OK:
            raise RpcaError(st, "rpca_server_create")
        self.handle = h
        self.set_warm(warm, warm_mu_scale, cold_every)
        self._keep = {}

    def set_warm(self, warm: bool, warm_mu_scale: float = 0.1, cold_every: int = 0):
        st = self.lib.rpca_server_set_warm(self.handle, int(bool(warm)), float(warm_mu_scale), int(cold_every))
        if st != OK:
            raise RpcaError(st, "rpca_server_set_warm")

    def close(self):
        if getattr(self, "handle", None):
            self.lib.rpca_server_destroy(self.handle)
            self.handle = None
            self._keep = {}

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def submit(self, frames, key: int, L=None, S=None, mask=None, theta: float = 0.0, **kw) -> int:
        """Queue one (T, m) float32 CUDA window of probe `key`; returns the request id.

        L and S (allocated here unless given) receive the result; keep them
        until the request is reported done."""
        torch = _torch()
        if frames.dtype not in (torch.float32, torch.complex64) or not frames.is_cuda or not frames.is_contiguous():
            raise ValueError("frames must be a contiguous float32 or complex64 CUDA tensor")
        T, m = frames.shape
        if frames.dtype == torch.complex64:
            kw = dict(kw, dtype=C64)
        p = default_params(m, T, **kw)
        if L is None:
            L = torch.empty_like(frames)
        if S is None:
            S = torch.empty_like(frames)
        _check_like(frames, L=L, S=S)
        rid = ctypes.c_uint64()
        st = self.lib.rpca_submit(self.handle, ctypes.byref(p), ctypes.c_void_p(frames.data_ptr()),
                                  ctypes.c_void_p(L.data_ptr()), ctypes.c_void_p(S.data_ptr()),
                                  ctypes.c_void_p(mask.data_ptr() if mask is not None else 0), ctypes.c_float(theta),
                                  int(key), ctypes.byref(rid))
        if st != OK:
            raise RpcaError(st, "rpca_submit")
        self._keep[rid.value] = (frames, L, S, mask)
        return rid.value

    def outputs(self, rid: int):
        """(L, S, mask) tensors of a request."""
        f, L, S, mk = self._keep[rid]
        return L, S, mk

    def poll(self, rid: int):
        """None while pending, else (status, result dict)."""
        res = Result()
        st = self.lib.rpca_poll(self.handle, ctypes.c_uint64(rid), ctypes.byref(res))
        if st == PENDING:
            return None
        if st in (ERR_NOTFOUND, ERR_ARG):
            raise RpcaError(st, "rpca_poll")
        return st, res.as_dict()

    def wait(self, rid: int):
        """Block until done; (status, result dict)."""
        res = Result()
        st = self.lib.rpca_server_wait(self.handle, ctypes.c_uint64(rid), ctypes.byref(res))
        if st in (ERR_NOTFOUND, ERR_ARG, ERR_BUDGET):
            raise RpcaError(st, "rpca_server_wait")
        return st, res.as_dict()

    def stats(self) -> dict:
        buf = (ctypes.c_int64 * 10)()
        st = self.lib.rpca_server_stats(self.handle, buf, 10)
        if st != OK:
            raise RpcaError(st, "rpca_server_stats")
        return dict(zip(self.STATS, list(buf)))
