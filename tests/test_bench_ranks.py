"""The benchmark's multi-rank host logic with 2 gloo ranks on CPU: rank
discovery from the launcher's environment, the barrier, and the max over the
ranks' times from which the whole-job throughput is formed.  No GPU."""
import importlib.util
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    argv = sys.argv
    sys.argv = ["bench.py"]
    try:
        spec.loader.exec_module(mod)
    finally:
        sys.argv = argv
    return mod


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    import torch.distributed as dist
    os.environ.update(RANK=str(rank), LOCAL_RANK=str(rank), WORLD_SIZE=str(world),
                      MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    b = _bench()
    r, lr, w = b.dist_env()
    dist.init_process_group("gloo", rank=r, world_size=w)
    b._barrier(w)
    t = b._max_over_ranks(1.0 + 2.0 * r, w)          # rank times 1.0 and 3.0 s
    out[r] = (r, lr, w, t, w * 8 * 10 / t)             # whole-job solves/s of 8 windows x 10 steps per rank
    dist.destroy_process_group()


def test_two_ranks_take_the_slowest_time():
    import torch.multiprocessing as mp
    out = mp.Manager().dict()
    mp.spawn(_rank_main, args=(2, _free_port(), out), nprocs=2, join=True)
    assert sorted(out.keys()) == [0, 1]
    for r in (0, 1):
        rank, lrank, world, t, value = out[r]
        assert (rank, lrank, world) == (r, r, 2)
        assert t == 3.0                                 # max over the ranks
        assert value == pytest.approx(2 * 80 / 3.0)     # all ranks' work over the slowest rank's time
