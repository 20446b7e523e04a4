"""One window split by pixel rows across processes (one GPU each).

The iteration of Sec. II-A touches the whole window only through the T x T
Gram Z^T Z (the SVD of Eq. 4 is taken through its eigen-decomposition) and
through the residual and norm sums of the stopping test.  With the pixel rows
of one window spread over the processes of a torch.distributed group, every
process runs the fused pass over its own rows, the processes sum the Gram and
the two scalar sums (one all-reduce of T*32 + 2 doubles per iteration), and every process runs the same eigen-step on the same sums, so
all of them follow the iteration of the whole window and stop together.

``solve_sharded`` drives any engine with the step interface below;
``PlanSteps`` is the GPU engine over the library's step-wise C ABI
(rpca_step_begin / rpca_step_run / rpca_step_sums / rpca_step_done).
"""
from __future__ import annotations

import ctypes
import math

from . import rpca

STEP_INIT, STEP_EIG_INIT, STEP_PASS, STEP_EIG, STEP_FINAL = 0, 1, 2, 3, 4


class _DeviceArray:
    """A device buffer of the library exposed to torch without a copy."""

    def __init__(self, ptr: int, shape, typestr: str):
        self.__cuda_array_interface__ = {"shape": tuple(shape), "typestr": typestr, "data": (ptr, False),
                                         "version": 3, "strides": None}


class PlanSteps:
    """GPU engine: a sharded plan over this process's m_local pixel rows of a
    window of m_total rows and T frames (lambda from the whole window)."""

    def __init__(self, m_local: int, T: int, m_total: int, **kw):
        torch = rpca._torch()
        lam = kw.pop("lambda_", None) or 1.0 / math.sqrt(max(int(m_total), int(T)))
        self.plan = rpca.Plan(m_local, T, sharded=1, lambda_=lam, **kw)
        self.lib = self.plan.lib
        g, s = ctypes.POINTER(ctypes.c_double)(), ctypes.POINTER(ctypes.c_double)()
        st = self.lib.rpca_step_sums(self.plan.handle, ctypes.byref(g), ctypes.byref(s))
        if st != rpca.OK:
            raise rpca.RpcaError(st, "rpca_step_sums")
        gp = ctypes.cast(g, ctypes.c_void_p).value
        sp = ctypes.cast(s, ctypes.c_void_p).value
        self._gram = torch.as_tensor(_DeviceArray(gp, (T, 32), "<f8"), device="cuda")
        self._sums = torch.as_tensor(_DeviceArray(sp, (2,), "<f8"), device="cuda")
        self.m, self.T = int(m_local), int(T)

    def begin(self, X, L, S, mask=None, theta: float = 0.0):
        rpca._check_like(X, L=L, S=S)
        st = self.lib.rpca_step_begin(self.plan.handle, ctypes.c_void_p(X.data_ptr()), ctypes.c_void_p(L.data_ptr()),
                                      ctypes.c_void_p(S.data_ptr()),
                                      ctypes.c_void_p(mask.data_ptr() if mask is not None else 0),
                                      ctypes.c_float(theta), rpca._stream_handle(None))
        if st != rpca.OK:
            raise rpca.RpcaError(st, "rpca_step_begin")

    def run(self, step: int):
        st = self.lib.rpca_step_run(self.plan.handle, int(step), rpca._stream_handle(None))
        if st != rpca.OK:
            raise rpca.RpcaError(st, "rpca_step_run")

    def sums(self):
        """The buffers to sum across the processes: the Gram (T x 32 float64;
        columns >= T unused) and (e2, l1) float64, both on the device."""
        return [self._gram, self._sums]

    def done(self):
        d = ctypes.c_int32()
        res = rpca.Result()
        st = self.lib.rpca_step_done(self.plan.handle, ctypes.byref(d), ctypes.byref(res), rpca._stream_handle(None))
        if st != rpca.OK:
            raise rpca.RpcaError(st, "rpca_step_done")
        return bool(d.value), res.as_dict()

    def close(self):
        self.plan.close()


def _all_reduce(tensors, group, host_stage: bool):
    import torch.distributed as dist
    if group is None and (not dist.is_available() or not dist.is_initialized()):
        return
    if dist.get_world_size(group) == 1:
        return
    for t in tensors:
        if host_stage:
            c = t.cpu()
            dist.all_reduce(c, group=group)
            t.copy_(c)
        else:
            dist.all_reduce(t, group=group)


def solve_sharded(engine, X, L, S, mask=None, theta: float = 0.0, group=None, host_stage: bool = False,
                  max_iter: int = 500):
    """Solve this process's rows X (T x m_local) of a window whose other rows
    the other processes of `group` hold, through `engine` (``PlanSteps`` or any
    object with begin/run/sums/done).  host_stage: reduce through host memory
    (backends without device tensors, e.g. gloo).  Returns the result dict;
    L, S (and the mask) receive this process's rows."""
    engine.begin(X, L, S, mask, theta)
    engine.run(STEP_INIT)
    _all_reduce(engine.sums(), group, host_stage)
    engine.run(STEP_EIG_INIT)
    done, res = engine.done()
    it = 0
    while not done and it <= max_iter + 1:
        engine.run(STEP_PASS)
        _all_reduce(engine.sums(), group, host_stage)
        engine.run(STEP_EIG)
        done, res = engine.done()
        it += 1
    engine.run(STEP_FINAL)
    _, res = engine.done()
    return res
