"""Output-oriented POD (Section 3.3, metric C^T C) on the GPU against the oracle's
Algorithm 5, through the C ABI. The GPU forms the Gram (C S)^T (C S) of the snapshots'
output images and eigensolves it; the oracle takes the thin SVD of C S by one-sided
Jacobi rotations (equal in exact arithmetic). FP64 tolerances as the identity-metric
parity tests: same w, iterations within 1, 1e-10 in the A-norm at equal counts; the GPU
basis is C^T C-orthonormal to 1e-10."""
import numpy as np
import pytest

from oracle import Oracle, OracleSequence
from paper_1512_05820_gb300 import workloads as wl

from test_gpu_parity import a_err, to_dev

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1512_05820_gb300 import _lib
    _lib.load()
    return torch.device("cuda:0")


def _functionals(n, q=100, seed=11):
    """q random linear functionals with U[0, 1] entries (the paper's output experiment)."""
    return np.random.default_rng(seed).uniform(0.0, 1.0, size=(q, n))


@pytest.mark.parametrize("three_stage", [0, 1])
def test_output_pod_sequence(dev, three_stage):
    from paper_1512_05820_gb300.solver import DeviceCSR, PodCG
    seq = wl.diffusion3d_moving(m=16, p=8, s_max=8, w_max=8, period=10)
    C = _functionals(seq.n)
    orc = Oracle()
    extra = dict(three_stage=True, y_max=8, energy_y=1 - 1e-10, tol_stage2=1e-4) if three_stage else {}
    oseq = OracleSequence(seq.n, s_max=seq.s_max, w_max=seq.w_max, energy=seq.energy, oracle=orc, C=C, **extra)
    solver = PodCG(seq.n, w_max=seq.w_max, s_max=seq.s_max, energy=seq.energy, three_stage=three_stage,
                   **({k: v for k, v in extra.items() if k != "three_stage"}))
    solver.set_output_functionals(to_dev(C, dev))
    A0 = DeviceCSR.from_numpy(seq.row_ptr, seq.col, np.zeros(seq.nnz), device=dev)
    for j, val, b in seq.systems():
        A = (seq.row_ptr, seq.col, val)
        x, st = solver.solve(A0.with_values(to_dev(val, dev)), to_dev(b, dev), seq.tol)
        xo, info = oseq.solve(A, b, seq.tol)
        if st["w"] > 0 and not three_stage:
            W = solver.basis().cpu().numpy()
            CW = C @ W
            assert np.max(np.abs(CW.T @ CW - np.eye(W.shape[1]))) <= 1e-10
        solver.add_snapshots(to_dev(xo, dev))
        x = x.cpu().numpy()
        assert st["status"] == "ok", st
        assert st["w"] == info["w"], (j, st["w"], info["w"])
        assert abs(st["iters"] - info["iters"]) <= 1, (j, st["iters"], info["iters"])
        assert np.linalg.norm(b - orc.spmv(A, x)) / np.linalg.norm(b) <= seq.tol
        if st["iters"] == info["iters"]:
            assert a_err(orc, A, x, xo) <= 1e-10, (j, a_err(orc, A, x, xo))
    solver.close()


def test_output_pod_set_after_snapshots_and_reset(dev):
    """Functionals set after the snapshots give the same solve, bit for bit, as set
    before them; q = 0 returns to the identity-metric POD (bitwise equal to a handle that
    never had functionals)."""
    from paper_1512_05820_gb300.solver import DeviceCSR, PodCG
    seq = wl.diffusion3d_moving(m=14, p=4, s_max=6, w_max=6, period=8)
    systems = seq.all_systems()
    C = to_dev(_functionals(seq.n, q=37, seed=3), dev)
    A0 = DeviceCSR.from_numpy(seq.row_ptr, seq.col, np.zeros(seq.nnz), device=dev)
    snaps = to_dev(np.random.default_rng(4).normal(size=(seq.n, 5)), dev)
    j, val, b = systems[-1]
    A, bt = A0.with_values(to_dev(val, dev)), to_dev(b, dev)
    s1 = PodCG(seq.n, w_max=6, s_max=6)
    s1.set_output_functionals(C)
    s1.add_snapshots(snaps)
    x1, st1 = s1.solve(A, bt, seq.tol)
    s2 = PodCG(seq.n, w_max=6, s_max=6)
    s2.add_snapshots(snaps)
    s2.set_output_functionals(C)
    x2, st2 = s2.solve(A, bt, seq.tol)
    assert torch.equal(x1, x2) and st1["w"] == st2["w"]
    s2.set_output_functionals(None)
    x3, st3 = s2.solve(A, bt, seq.tol)
    s3 = PodCG(seq.n, w_max=6, s_max=6)
    s3.add_snapshots(snaps)
    x4, st4 = s3.solve(A, bt, seq.tol)
    assert torch.equal(x3, x4) and st3["w"] == st4["w"]
