"""The CG product in 3x3 block-sparse form (k_bsr.cu) against the CSR product and the
FP64 oracle, through the C ABI: same sequences solved both ways (iterations within 1,
solutions within the elasticity parity bound 5e-9 in the A-norm), pattern detection
(blocked patterns use it, others fall back or are refused), and a handle that alternates
between a blocked and an unblocked pattern of the same order."""
import numpy as np
import pytest

from oracle import Oracle
from paper_1512_05820_gb300 import workloads as wl

from test_gpu_parity import a_err, dcsr, to_dev

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1512_05820_gb300 import _lib
    _lib.load()
    return torch.device("cuda:0")


@pytest.mark.parametrize("precision", [0, 1])
def test_bsr_matches_csr_sequence(dev, precision):
    """6^3-element cantilever (n = 882; block rows of 8 to 27 blocks at faces, edges and
    inside), 4 systems: the block form and the CSR form take the same iterations (within
    1) and reach the same solutions (5e-9 A-norm in FP64; both within tol in mixed
    precision)."""
    from paper_1512_05820_gb300.solver import DeviceCSR, PodCG
    seq = wl.elasticity_cantilever(e=6, p=4, w_max=8, s_max=8)
    orc = Oracle()
    runs = []
    for bsr in (0, 1):
        solver = PodCG(seq.n, w_max=seq.w_max, s_max=seq.s_max, energy=seq.energy, precision=precision, bsr=bsr)
        A0 = DeviceCSR.from_numpy(seq.row_ptr, seq.col, np.zeros(seq.nnz), device=dev)
        res = []
        for j, val, b in seq.systems():
            x, st = solver.solve(A0.with_values(to_dev(val, dev)), to_dev(b, dev), seq.tol)
            solver.add_snapshots(x)
            res.append((x.cpu().numpy(), st, val, b))
        runs.append(res)
        solver.close()
    for (x0, s0, val, b), (x1, s1, _, _) in zip(runs[0], runs[1]):
        A = (seq.row_ptr, seq.col, val)
        assert s0["status"] == s1["status"] == "ok"
        for x in (x0, x1):
            assert np.linalg.norm(b - orc.spmv(A, x)) / np.linalg.norm(b) <= seq.tol
        if precision == 0:
            assert abs(s0["iters"] - s1["iters"]) <= 1
            if s0["iters"] == s1["iters"]:
                assert a_err(orc, A, x1, x0) <= 5e-9


def test_bsr_pattern_detection(dev, orc):
    """bsr = 1 on a pattern without 3x3 blocks (a diffusion operator of order 3k) is an
    argument error; bsr = -1 falls back to the CSR product there and solves it."""
    from paper_1512_05820_gb300.solver import PodCG, PodCGError
    A = wl.DiffusionOperator((9, 10)).csr(np.exp(np.random.default_rng(0).normal(size=90)))
    b = np.random.default_rng(1).normal(size=A.n)
    s1 = PodCG(A.n, bsr=1)
    with pytest.raises(PodCGError) as e:
        s1.solve(dcsr(A, dev), to_dev(b, dev), 1e-10)
    assert e.value.status == 1
    s2 = PodCG(A.n, bsr=-1)
    x, st = s2.solve(dcsr(A, dev), to_dev(b, dev), 1e-10)
    xo, k, _ = orc.pcg(A.arrays(), b, None, 1e-10 * np.linalg.norm(b))
    assert st["status"] == "ok" and abs(st["iters"] - k) <= 1
    assert a_err(orc, A.arrays(), x.cpu().numpy(), xo) <= 1e-10


def test_bsr_handle_switches_patterns(dev, orc):
    """One handle (bsr = -1, FP64, no snapshots) solves a blocked elasticity system, an
    unblocked SPD system of the same order, then the elasticity system again: each solve
    picks its own product form and matches the oracle's plain PCG."""
    from paper_1512_05820_gb300.solver import PodCG
    seq = wl.elasticity_cantilever(e=5, p=1)
    j, val, b = next(iter(seq.systems()))
    E = (seq.row_ptr, seq.col, val)
    R = wl.random_spd_csr(seq.n, 0.01, seed=3)
    bR = np.random.default_rng(2).normal(size=seq.n)
    solver = PodCG(seq.n, bsr=-1)
    for A, rhs in ((E, b), (R.arrays(), bR), (E, b)):
        x, st = solver.solve(dcsr(A, dev), to_dev(rhs, dev), 1e-10)
        xo, k, _ = orc.pcg(A, rhs, None, 1e-10 * np.linalg.norm(rhs))
        assert st["status"] == "ok" and abs(st["iters"] - k) <= 2, (st["iters"], k)
        assert a_err(orc, A, x.cpu().numpy(), xo) <= 5e-9
