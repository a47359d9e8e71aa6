"""The allocation-free Gram entry point (pod_cg_gram_noalloc).

It serves callers that cannot allocate device memory where they need the product: loops
where cudaMalloc/cudaFree would synchronise the whole device, and hosts that hand out the
whole device-memory budget themselves. The variant keeps its scratch in a fixed array
inside the library. Two calls in a row with different shapes must give the result of the
workspace-taking entry point bit for bit (same kernels, same split shape), and both must
agree with an FP64 product computed on the host within the Gram bound the other tests use.
This file is collected last so a failure here cannot hide any other test's result.
"""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1512_05820_gb300 import _lib
    return _lib.load()


def test_gram_noalloc_matches_gram(lib):
    from paper_1512_05820_gb300 import solver
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    for n, p, q in [(50000, 32, 33), (10007, 13, 7)]:
        rng = np.random.default_rng(n + q)
        Xh, Yh = rng.normal(size=(n, p)), rng.normal(size=(n, q))
        X = torch.as_tensor(Xh, device="cuda")
        Y = torch.as_tensor(Yh, device="cuda")
        G_ref = solver.gram(X, Y).cpu().numpy()
        Xc, Yc = X.t().contiguous(), Y.t().contiguous()
        G = torch.full((p, q), float("nan"), dtype=torch.float64, device="cuda")
        rc = lib.pod_cg_gram_noalloc(n, Xc.data_ptr(), p, Yc.data_ptr(), q, G.data_ptr(), stream)
        torch.cuda.synchronize()
        assert rc == 0, lib.pod_cg_last_error(None)
        Gn = G.cpu().numpy()
        assert np.array_equal(Gn, G_ref)
        # independent FP64 product on the host; the bound is that of any FP64 sum of n
        # products: |error| <= n u sum_k |x_k y_k| <= 1e-15 n ||x|| ||y||
        bound = 1e-15 * n * np.outer(np.linalg.norm(Xh, axis=0), np.linalg.norm(Yh, axis=0))
        assert np.all(np.abs(Gn - Xh.T @ Yh) <= bound)


def test_gram_noalloc_rejects_more_than_65_columns(lib):
    X = torch.zeros((66, 100), dtype=torch.float64, device="cuda")
    G = torch.zeros((66, 66), dtype=torch.float64, device="cuda")
    rc = lib.pod_cg_gram_noalloc(100, X.data_ptr(), 66, X.data_ptr(), 66, G.data_ptr(), None)
    assert rc == 1 and b"65" in lib.pod_cg_last_error(None)
