"""The allocation-free Gram entry point (pod_cg_gram_noalloc) against pod_cg_gram.

For callers that cannot allocate device memory where they need the product (device-wide
synchronisation of cudaMalloc in latency-bound loops, or a host that owns the whole
device-memory budget): the variant keeps its scratch in a fixed array inside the library.
Two calls in a row with different shapes must match the workspace-taking entry point
within the Gram tolerance the other tests use. This file is collected last so a failure
here cannot hide any other test's result.
"""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def test_gram_noalloc_matches_gram():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1512_05820_gb300 import _lib, solver
    L = _lib.load()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    for n, p, q in [(50000, 32, 33), (10007, 13, 7)]:
        rng = np.random.default_rng(n + q)
        X = torch.as_tensor(rng.normal(size=(n, p)), device="cuda")
        Y = torch.as_tensor(rng.normal(size=(n, q)), device="cuda")
        G_ref = solver.gram(X, Y)
        Xc, Yc = X.t().contiguous(), Y.t().contiguous()
        G = torch.full((p, q), float("nan"), dtype=torch.float64, device="cuda")
        rc = L.pod_cg_gram_noalloc(n, Xc.data_ptr(), p, Yc.data_ptr(), q, G.data_ptr(), stream)
        torch.cuda.synchronize()
        assert rc == 0, L.pod_cg_last_error(None)
        Xn = np.linalg.norm(X.cpu().numpy(), axis=0)
        Yn = np.linalg.norm(Y.cpu().numpy(), axis=0)
        bound = 1e-15 * n * np.outer(Xn, Yn)
        assert np.all(np.abs(G.cpu().numpy() - G_ref.cpu().numpy()) <= bound)


def test_gram_noalloc_rejects_oversize():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1512_05820_gb300 import _lib
    L = _lib.load()
    X = torch.zeros((66, 100), dtype=torch.float64, device="cuda")
    G = torch.zeros((66, 66), dtype=torch.float64, device="cuda")
    rc = L.pod_cg_gram_noalloc(100, X.data_ptr(), 66, X.data_ptr(), 66, G.data_ptr(), None)
    assert rc == 1 and b"65" in L.pod_cg_last_error(None)
