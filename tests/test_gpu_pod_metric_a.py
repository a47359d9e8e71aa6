"""POD with the metric A of the system being solved (pod_metric = 1; Algorithm 4 with
Theta = A) on the GPU against the oracle, through the C ABI: w equal, iterations within
1, 1e-10 in the A-norm at equal counts, and the basis A-orthonormal to 1e-10; with the
three-stage algorithm the augmenting basis makes Y^T A Y = I, so stage two needs at most
one iteration per system."""
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


@pytest.mark.parametrize("three_stage", [0, 1])
def test_pod_metric_a_sequence(dev, three_stage):
    from paper_1512_05820_gb300.solver import DeviceCSR, PodCG
    seq = wl.diffusion3d_moving(m=16, p=8, s_max=8, w_max=8, period=10)
    orc = Oracle()
    extra = dict(three_stage=True, y_max=8, energy_y=1 - 1e-10, tol_stage2=1e-4) if three_stage else {}
    oseq = OracleSequence(seq.n, s_max=seq.s_max, w_max=seq.w_max, energy=seq.energy, oracle=orc, metric_a=True,
                          **extra)
    solver = PodCG(seq.n, w_max=seq.w_max, s_max=seq.s_max, energy=seq.energy, pod_metric=1,
                   three_stage=three_stage, **({k: v for k, v in extra.items() if k != "three_stage"}))
    A0 = DeviceCSR.from_numpy(seq.row_ptr, seq.col, np.zeros(seq.nnz), device=dev)
    for j, val, b in seq.systems():
        A = (seq.row_ptr, seq.col, val)
        x, st = solver.solve(A0.with_values(to_dev(val, dev)), to_dev(b, dev), seq.tol)
        xo, info = oseq.solve(A, b, seq.tol)
        if st["w"] > 0 and not three_stage:
            W = solver.basis().cpu().numpy()
            AW = np.stack([orc.spmv(A, W[:, k]) for k in range(W.shape[1])], axis=1)
            assert np.max(np.abs(W.T @ AW - np.eye(W.shape[1]))) <= 1e-10
        if three_stage and st["y"] > 0:
            assert st["stage2_iters"] <= 1, st["stage2_iters"]
        solver.add_snapshots(to_dev(xo, dev))
        x = x.cpu().numpy()
        assert st["status"] == "ok", st
        assert st["w"] == info["w"], (j, st["w"], info["w"])
        assert abs(st["iters"] - info["iters"]) <= 1, (j, st["iters"], info["iters"])
        assert np.linalg.norm(b - orc.spmv(A, x)) / np.linalg.norm(b) <= seq.tol
        if st["iters"] == info["iters"]:
            assert a_err(orc, A, x, xo) <= 1e-10, (j, a_err(orc, A, x, xo))
    solver.close()


def test_pod_metric_a_excludes_output_functionals(dev):
    from paper_1512_05820_gb300.solver import PodCG, PodCGError
    s = PodCG(100, pod_metric=1)
    with pytest.raises(PodCGError) as e:
        s.set_output_functionals(torch.ones((3, 100), dtype=torch.float64, device=dev))
    assert e.value.status == 9
