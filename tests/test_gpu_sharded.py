"""GPU: one window split by pixel rows, through the step-wise C ABI.

One process: the sharded plan driven step by step equals the whole-window
plan and the oracle.  Two processes on the one GPU (gloo, sums reduced through
host memory; no kernel waits on another process): the halves solved
separately equal the oracle's solve of the whole window."""
import os
import socket

import numpy as np
import pytest

from oracle import rpca_oracle as O
from paper_2506_10257_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

FP32_TOL = 1e-5


def rel(a, b):
    return np.linalg.norm(np.asarray(a, np.float64) - b) / np.linalg.norm(b)


@pytest.fixture(scope="module")
def rp():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2506_10257_gb300 import rpca
    rpca.load()
    return rpca


def test_one_process_steps_equal_the_plan(rp):
    from paper_2506_10257_gb300.sharded import PlanSteps, solve_sharded
    w = synth.make_preset("w64x64_t20", seed=21)
    X = torch.from_numpy(w.frames).cuda()
    T, m = X.shape
    L, S = torch.empty_like(X), torch.empty_like(X)
    mask = torch.zeros(m, dtype=torch.uint8, device="cuda")
    eng = PlanSteps(m, T, m)
    res = solve_sharded(eng, X, L, S, mask=mask, theta=2.0)
    eng.close()
    L0, S0, res0 = rp.Plan(m, T).solve(X, mask=torch.zeros_like(mask), theta=2.0)
    ref = O.rpca_frames(w.frames)
    assert res["status"] == rp.OK and res["iters"] == res0["iters"]
    assert rel(L.cpu().numpy(), L0.cpu().numpy()) <= 1e-6 and rel(S.cpu().numpy(), S0.cpu().numpy()) <= 1e-6
    assert rel(L.cpu().numpy(), ref.L) <= FP32_TOL and rel(S.cpu().numpy(), ref.S) <= FP32_TOL
    assert abs(res["iters"] - ref.iters) <= 1


def test_step_api_rejects_a_plan_without_sharding(rp):
    import ctypes
    plan = rp.Plan(256, 8)
    g, s = ctypes.POINTER(ctypes.c_double)(), ctypes.POINTER(ctypes.c_double)()
    assert plan.lib.rpca_step_sums(plan.handle, ctypes.byref(g), ctypes.byref(s)) == rp.ERR_ARG
    assert plan.lib.rpca_step_run(plan.handle, 2, None) == rp.ERR_ARG
    plan.close()
    with pytest.raises(rp.RpcaError):
        rp.Plan(256, 40, sharded=1)             # the tiled path is not sharded
    with pytest.raises(rp.RpcaError):
        rp.Plan(256, 8, sharded=1, mu_schedule=rp.MU_FIXED_L1)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, frames, out):
    import torch.distributed as dist
    from paper_2506_10257_gb300.sharded import PlanSteps, solve_sharded
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    T, m = frames.shape
    bounds = [0, 2000, m] if world == 2 else [0, m]     # uneven halves, multiples of 4 not required
    lo, hi = bounds[rank], bounds[rank + 1]
    X = torch.from_numpy(np.ascontiguousarray(frames[:, lo:hi])).cuda()
    L, S = torch.empty_like(X), torch.empty_like(X)
    eng = PlanSteps(hi - lo, T, m)
    res = solve_sharded(eng, X, L, S, host_stage=True)
    out[rank] = (lo, hi, L.cpu().numpy(), S.cpu().numpy(), res["iters"], res["status"])
    eng.close()
    dist.destroy_process_group()


def test_two_processes_split_one_window(rp):
    import torch.multiprocessing as mp
    w = synth.make_preset("w64x64_t20", seed=22)
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.spawn(_rank_main, args=(2, _free_port(), w.frames, out), nprocs=2, join=True)
    T, m = w.frames.shape
    L, S = np.zeros((T, m)), np.zeros((T, m))
    its = set()
    for r in range(2):
        lo, hi, Lr, Sr, it, st = out[r]
        assert st == rp.OK
        L[:, lo:hi], S[:, lo:hi] = Lr, Sr
        its.add(it)
    ref = O.rpca_frames(w.frames)
    assert len(its) == 1 and abs(its.pop() - ref.iters) <= 1
    assert rel(L, ref.L) <= FP32_TOL and rel(S, ref.S) <= FP32_TOL
