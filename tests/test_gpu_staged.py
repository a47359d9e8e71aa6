"""Both forms of the FP32 update and direction passes (row-parallel float4, and tiles staged
in shared memory by the TMA engine) across every basis-width bucket, against the FP64 oracle
with the same snapshots.

n = 23^3 = 12,167 is not a multiple of the 256-row tile, so every solve ends on a ragged
tile; nsnap seeded random snapshots with energy 1 give w = nsnap (up to the cap).
Tolerance as for the other mixed-precision tests: the FP64 true residual reaches tol,
w equals the oracle's, and the A-norm difference to the oracle's solution is within what
two solutions of residual <= tol can differ by (1e-5 here)."""
import numpy as np
import pytest

from oracle import Oracle, OracleSequence
from paper_1512_05820_gb300 import workloads as wl

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1512_05820_gb300 import _lib
    _lib.load()
    return torch.device("cuda:0")


def _a_err(orc, A, x, xo):
    dx = x - xo
    return float(np.sqrt(dx @ orc.spmv(A, dx)) / np.sqrt(xo @ orc.spmv(A, xo)))


@pytest.mark.parametrize("form", [0, 1])
@pytest.mark.parametrize("nsnap,w_max", [(6, 8), (14, 16), (22, 32), (40, 48), (64, 64)])
def test_mixed_staged_widths(dev, nsnap, w_max, form):
    from paper_1512_05820_gb300.solver import DeviceCSR, PodCG
    seq = wl.diffusion3d_moving(m=23, p=2, s_max=64, w_max=w_max, period=10)
    systems = list(seq.systems())
    j, val, b = systems[1]
    A = (seq.row_ptr, seq.col, val)
    S = np.random.default_rng(nsnap).normal(size=(seq.n, nsnap))
    orc = Oracle()
    oseq = OracleSequence(seq.n, s_max=64, w_max=w_max, energy=1.0, oracle=orc)
    for k in range(nsnap):
        oseq.add_snapshot(S[:, k])
    xo, info = oseq.solve(A, b, seq.tol)
    solver = PodCG(seq.n, w_max=w_max, s_max=64, energy=1.0, precision=1, proj_form=form)
    solver.add_snapshots(torch.as_tensor(S, device=dev))
    x, st = solver.solve(DeviceCSR.from_numpy(seq.row_ptr, seq.col, val, device=dev), torch.as_tensor(b, device=dev),
                         seq.tol)
    solver.close()
    x = x.cpu().numpy()
    assert st["status"] == "ok", st
    assert st["w"] == info["w"] == min(nsnap, w_max)
    true_rel = np.linalg.norm(b - orc.spmv(A, x)) / np.linalg.norm(b)
    assert true_rel <= seq.tol and st["final_relres"] <= seq.tol
    assert _a_err(orc, A, x, xo) <= 1e-5


@pytest.mark.parametrize("form,lanes,graph_mode", [(0, 1, 0), (1, 1, 0), (0, 1, 2), (1, 2, 2)])
def test_mixed_loop_modes_bitwise_equal(dev, form, lanes, graph_mode):
    """Mixed precision: the conditional-graph loop and the chunked loop agree bit for bit.
    Loop mode 0 launches the same three kernels per iteration as the chunked loop. Loop mode
    2 with one lane per CSR row (bases up to 8 wide) runs the whole inner loop as one
    persistent launch while the chunked loop launches the row-parallel kernels: the
    persistent kernel repeats their arithmetic and reduction order, so the iterates are the
    same (with 2 lanes it falls back to the three kernels)."""
    from paper_1512_05820_gb300.solver import DeviceCSR, PodCG
    seq = wl.diffusion3d_moving(m=19, p=5, s_max=6, w_max=8, period=10)
    outs, loop_ms = [], []
    for mode in (graph_mode, 1):
        solver = PodCG(seq.n, w_max=seq.w_max, s_max=seq.s_max, energy=seq.energy, precision=1, loop_mode=mode,
                       proj_form=form, spmv_lanes=lanes)
        A0 = DeviceCSR.from_numpy(seq.row_ptr, seq.col, np.zeros(seq.nnz), device=dev)
        xs, its = [], []
        for j, val, b in seq.systems():
            x, st = solver.solve(A0.with_values(torch.as_tensor(val, device=dev)), torch.as_tensor(b, device=dev),
                                 seq.tol)
            solver.add_snapshots(x)
            xs.append(x.clone())
            its.append((st["iters"], st["w"]))
            if mode != 1:
                loop_ms.append(st["ms_loop"])
        solver.close()
        outs.append((xs, its))
    assert outs[0][1] == outs[1][1]
    for a, c in zip(outs[0][0], outs[1][0]):
        assert torch.equal(a, c)
    # the graph-mode solves ran the persistent loop exactly in loop mode 2 with one lane per row
    persistent = graph_mode == 2 and lanes == 1
    assert all((t > 0.0) == persistent for t in loop_ms), loop_ms


def test_projection_form_is_timed(dev):
    """Default configuration on a system of >= 65,536 rows: the handle times both forms of each
    pass for the bucket, keeps the faster for each, and the solve reaches tol."""
    from paper_1512_05820_gb300.solver import DeviceCSR, PodCG
    seq = wl.diffusion3d_moving(m=42, p=2, s_max=8, w_max=8, period=10)
    assert seq.n >= 65536
    solver = PodCG(seq.n, w_max=8, s_max=8, energy=1.0, precision=1)
    solver.add_snapshots(torch.as_tensor(np.random.default_rng(3).normal(size=(seq.n, 6)), device=dev))
    j, val, b = list(seq.systems())[1]
    x, st = solver.solve(DeviceCSR.from_numpy(seq.row_ptr, seq.col, val, device=dev), torch.as_tensor(b, device=dev),
                         seq.tol)
    tun = solver.tuning()["projection"]
    solver.close()
    assert st["status"] == "ok" and st["final_relres"] <= seq.tol
    rec = tun["w<=8"]
    for p in ("update", "direction"):
        direct, staged = rec[f"ms_{p}_direct"], rec[f"ms_{p}_staged"]
        assert direct > 0 and staged > 0
        assert rec[p] == ("staged" if staged < direct else "direct")


@pytest.mark.parametrize("lanes", [1, 4, 32])
def test_forced_spmv_lanes(dev, lanes):
    """A forced CSR SpMV width is used as given (FP64 and mixed) and the solves still reach
    tol with the oracle's basis width."""
    from paper_1512_05820_gb300.solver import DeviceCSR, PodCG
    seq = wl.diffusion3d_moving(m=20, p=3, s_max=4, w_max=8, period=10)
    for prec in (0, 1):
        solver = PodCG(seq.n, w_max=8, s_max=4, energy=seq.energy, precision=prec, spmv_lanes=lanes)
        A0 = DeviceCSR.from_numpy(seq.row_ptr, seq.col, np.zeros(seq.nnz), device=dev)
        for j, val, b in seq.systems():
            x, st = solver.solve(A0.with_values(torch.as_tensor(val, device=dev)), torch.as_tensor(b, device=dev),
                                 seq.tol)
            assert st["status"] == "ok" and st["final_relres"] <= seq.tol
            solver.add_snapshots(x)
        assert solver.tuning()["spmv_lanes"] == lanes
        solver.close()
