"""rpca_gram_noalloc through the C ABI, against the Gram written out in FP64.

rpca_gram_noalloc serves callers that may not allocate device memory while
they run (a scanner pipeline that reserves its memory at start-up and must
not stall on the allocator, a process whose device memory belongs to another
framework's pool); it keeps its scratch in a fixed array inside the library.
Its result must equal G = (Z V)^T (Z V), formed here in float64 from the same
float32 inputs, within the Gram tolerance of the kernel-level tests, on two
calls in a row (the second runs on the scratch the first left behind), on the
current stream and on a stream of its own, and it must agree with the
allocating rpca_gram.  This file is collected last.
"""
import numpy as np
import pytest

from paper_2506_10257_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def fp64_gram(F, V32):
    Z = F.T.astype(np.float64)
    if V32 is not None:
        Z = Z @ V32.astype(np.float64)
    return Z.T @ Z


@pytest.mark.parametrize("m,T,rotate", [(4096, 20, True), (70000, 32, False), (300, 7, True), (200000, 12, True)])
@pytest.mark.parametrize("own_stream", [False, True])
def test_gram_noalloc_matches_fp64_twice(m, T, rotate, own_stream):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2506_10257_gb300 import rpca
    F = synth.random_dense(100 + m + T, m, T)
    X = torch.from_numpy(F).cuda()
    V32 = None
    V = None
    if rotate:
        Q, _ = np.linalg.qr(np.random.default_rng(T).standard_normal((T, T)))
        V32 = Q.astype(np.float32)
        # given as float64 on the host, so the binding converts it (a temporary
        # that must outlive the kernels on a stream of their own)
        V = torch.from_numpy(V32.astype(np.float64))
    want = fp64_gram(F, V32)
    tol = 2e-6 * np.abs(want).max()
    stream = torch.cuda.Stream() if own_stream else None
    for _ in range(2):
        G = rpca.gram_noalloc(X, V=V, stream=stream)
        torch.cuda.synchronize()
        assert np.abs(G.cpu().numpy() - want).max() <= tol
    # and the allocating entry point gives the same Gram
    Ga = rpca.gram(X, V=V).cpu().numpy()
    assert np.abs(Ga - G.cpu().numpy()).max() <= tol
