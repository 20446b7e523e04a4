"""One window split by pixel rows across two processes (gloo, CPU).

The driver (paper_2506_10257_gb300.sharded.solve_sharded) is run by two gloo
ranks, each holding half of the window's pixel rows, over a test-side FP64
NumPy engine with the step semantics of the library's step-wise C ABI (local
pass over the rows, Gram and scalar sums handed to the driver for the
all-reduce, eigen-step on the summed Gram).  The result must equal the
unsharded oracle's: the only exchange of the iteration is the Gram and the two
scalar sums.  No GPU."""
import math
import os
import socket

import numpy as np
import pytest

from oracle import rpca_oracle as O
from paper_2506_10257_gb300 import synth

torch = pytest.importorskip("torch")


class NumpySteps:
    """FP64 engine with the step semantics of rpca_step_* (Gram route)."""

    def __init__(self, m_total, T, tol=1e-7, max_iter=500, rho=1.5):
        self.lam = 1.0 / math.sqrt(max(m_total, T))
        self.tol, self.max_iter, self.rho = tol, max_iter, rho
        self.G = torch.zeros((T, T), dtype=torch.float64)
        self.s = torch.zeros(2, dtype=torch.float64)

    @staticmethod
    def _weights(G, tau):
        lam, V = np.linalg.eigh(G)
        sig = np.sqrt(np.maximum(lam, 0.0))
        f = np.where(sig > tau, tau / np.where(sig > 0, sig, 1.0), 1.0)
        return (V * f) @ V.T

    def begin(self, X, L, S, mask=None, theta=0.0):
        self.X = np.asarray(X, dtype=np.float64).T          # (m_local, T)
        self.Lout, self.Sout = L, S
        self.S = np.zeros_like(self.X)
        self.Y = np.zeros_like(self.X)
        self.k, self.is_done, self.resid = 0, False, 0.0

    def run(self, step):
        if step == 0:      # INIT: Gram of X, ||X||_F^2, ||X||_1
            self.G.copy_(torch.from_numpy(self.X.T @ self.X))
            self.s.copy_(torch.tensor([np.sum(self.X ** 2), np.sum(np.abs(self.X))]))
        elif step == 1:    # EIG_INIT
            G = self.G.numpy()
            self.normX = math.sqrt(self.s[0].item())
            self.mu = 1.25 / math.sqrt(np.linalg.eigvalsh(G).max())
            self.mu_max = 1e7 * self.mu
            self.mu_nxt = min(self.rho * self.mu, self.mu_max)
            self.W = self._weights(G, 1.0 / self.mu)
        elif step == 2:    # PASS: Eq. 4-6 on the local rows, next Gram
            Z = self.X - self.S + self.Y / self.mu
            Q = Z @ self.W
            R = self.S + Q
            Sn = O.shrink(R, self.lam / self.mu)
            C = R - Sn
            E = C - self.Y / self.mu
            self.L = Z - Q
            self.S, self.Y = Sn, self.mu * C
            Zn = self.X - self.S + self.Y / self.mu_nxt
            self.G.copy_(torch.from_numpy(Zn.T @ Zn))
            self.s.copy_(torch.tensor([np.sum(E ** 2), 0.0]))
        elif step == 3:    # EIG: residual test, mu update, eigen-step
            self.k += 1
            self.resid = math.sqrt(self.s[0].item()) / self.normX
            if self.resid <= self.tol or self.k >= self.max_iter:
                self.is_done = True
            else:
                self.mu = self.mu_nxt
                self.mu_nxt = min(self.rho * self.mu, self.mu_max)
                self.W = self._weights(self.G.numpy(), 1.0 / self.mu)
        elif step == 4:    # FINAL
            self.Lout[...] = self.L.T
            self.Sout[...] = self.S.T

    def sums(self):
        return [self.G, self.s]

    def done(self):
        return self.is_done, {"iters": self.k, "resid": self.resid}


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, frames, out):
    import torch.distributed as dist
    from paper_2506_10257_gb300.sharded import solve_sharded
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    T, m = frames.shape
    bounds = np.linspace(0, m, world + 1).astype(int)
    lo, hi = bounds[rank], bounds[rank + 1]
    X = frames[:, lo:hi]
    L = np.zeros_like(X, dtype=np.float64)
    S = np.zeros_like(X, dtype=np.float64)
    res = solve_sharded(NumpySteps(m, T), X, L, S, group=None)
    out[rank] = (lo, hi, L, S, res["iters"], res["resid"])
    dist.destroy_process_group()


def run_world(frames, world):
    import torch.multiprocessing as mp
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_rank_main, args=(world, _free_port(), frames, out), nprocs=world, join=True)
    T, m = frames.shape
    L, S = np.zeros((T, m)), np.zeros((T, m))
    iters = set()
    for r in range(world):
        lo, hi, Lr, Sr, it, _ = out[r]
        L[:, lo:hi], S[:, lo:hi] = Lr, Sr
        iters.add(it)
    return L, S, iters


def test_two_ranks_reproduce_the_whole_window():
    w = synth.make_window(seed=81, ny=32, nx=32, T=16, n_bound=8, n_free=12)
    L2, S2, it2 = run_world(w.frames, 2)
    L1, S1, it1 = run_world(w.frames, 1)
    ref = O.rpca_frames(w.frames)
    assert it2 == it1 == {ref.iters}            # every rank stops at the oracle's iteration
    rel = lambda a, b: np.linalg.norm(a - b) / np.linalg.norm(b)
    assert rel(L2, L1) <= 1e-10 and rel(S2, S1) <= 1e-10   # only the Gram's summation order differs
    assert rel(L2, ref.L) <= 1e-8 and rel(S2, ref.S) <= 1e-8


def test_uneven_split_with_three_ranks():
    w = synth.make_window(seed=82, ny=20, nx=17, T=9, n_bound=4, n_free=6)
    L3, S3, it3 = run_world(w.frames, 3)
    ref = O.rpca_frames(w.frames)
    assert it3 == {ref.iters}
    rel = lambda a, b: np.linalg.norm(a - b) / np.linalg.norm(b)
    assert rel(L3, ref.L) <= 1e-8 and rel(S3, ref.S) <= 1e-8
