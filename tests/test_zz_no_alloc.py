"""rpca_gram_noalloc against rpca_gram, through the C ABI.

rpca_gram_noalloc serves callers that may not allocate device memory while
they run (a scanner pipeline that reserves its memory at start-up, a process
whose memory belongs to another pool); it keeps its scratch in a fixed array
inside the library.  Its result must equal the allocating rpca_gram within the
Gram tolerance of the other tests, on two calls in a row (the second call runs
on the scratch the first one left behind).  This file is collected last.
"""
import numpy as np
import pytest

from paper_2506_10257_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("m,T,rotate", [(4096, 20, True), (70000, 32, False), (300, 7, True), (200000, 12, True)])
def test_gram_noalloc_matches_gram_twice(m, T, rotate):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2506_10257_gb300 import rpca
    X = torch.from_numpy(synth.random_dense(100 + m + T, m, T)).cuda()
    V = None
    if rotate:
        Q, _ = np.linalg.qr(np.random.default_rng(T).standard_normal((T, T)))
        V = torch.from_numpy(Q.astype(np.float32)).cuda()
    want = rpca.gram(X, V=V).cpu().numpy()
    tol = 2e-6 * np.abs(want).max()
    for _ in range(2):
        G = rpca.gram_noalloc(X, V=V)
        torch.cuda.synchronize()
        assert np.abs(G.cpu().numpy() - want).max() <= tol
