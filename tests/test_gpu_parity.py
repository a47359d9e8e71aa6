"""GPU path against the FP64 oracle, through the C ABI.

Tolerances (FP64 mode): per system ||x - x_orc||_A / ||x_orc||_A <= 1e-10 with the same
snapshots (the oracle's previous solutions are fed to the GPU handle, so rounding
differences cannot compound along the sequence), iteration counts within 1 (summation
order differs), final true residual <= tol. When the counts differ by one, the exit test
(Eq. (sequenceInexact)) met its threshold within rounding on one side only; the GPU
iterate is then compared with the oracle's iterate after the same number of steps (two
FP64 CG runs that differ only in summation order stop one step apart on the elasticity
test matrix, and their final iterates differ by one CG step, 7e-10 in the A-norm).
Step-level kernels: element-wise relative errors at rounding level of the contraction
(bounds stated per test).
"""
import numpy as np
import pytest

import pins
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


def to_dev(a, dev):
    return torch.as_tensor(np.ascontiguousarray(a), device=dev)


def dcsr(A, dev):
    from paper_1512_05820_gb300.solver import DeviceCSR
    rp, col, val = A if isinstance(A, tuple) else A.arrays()
    return DeviceCSR.from_numpy(rp, col, val, device=dev)


def a_err(orc, A, x, xo):
    dx = x - xo
    num = dx @ orc.spmv(A, dx)
    den = xo @ orc.spmv(A, xo)
    return float(np.sqrt(max(num, 0.0) / den))


# ------------------------------------------------------------------ step kernels


@pytest.mark.parametrize("case", ["ragged", "diffusion3d", "tiny"])
def test_spmv(dev, orc, case):
    from paper_1512_05820_gb300.solver import spmv
    if case == "ragged":
        A = wl.random_spd_csr(3001, 0.01, seed=4, empty_rows=17)
    elif case == "diffusion3d":
        A = wl.DiffusionOperator((13, 17, 19)).csr(np.exp(np.random.default_rng(0).normal(size=13 * 17 * 19)))
    else:
        A = wl.DiffusionOperator((1, 1)).csr(np.ones(1))
    x = np.random.default_rng(1).normal(size=A.n)
    y = spmv(dcsr(A, dev), to_dev(x, dev)).cpu().numpy()
    yo = orc.spmv(A.arrays(), x)
    scale = orc.spmv((A.row_ptr, A.col, np.abs(A.val)), np.abs(x)) + 1e-300
    assert np.max(np.abs(y - yo) / scale) <= 4e-16 * 80


@pytest.mark.parametrize("w", [1, 7, 32, 48])
def test_spmm(dev, orc, w):
    from paper_1512_05820_gb300.solver import spmm
    A = wl.DiffusionOperator((21, 23, 11)).csr(np.exp(np.random.default_rng(2).normal(size=21 * 23 * 11)))
    W = np.asfortranarray(np.random.default_rng(3).normal(size=(A.n, w)))
    AW = spmm(dcsr(A, dev), to_dev(W, dev)).cpu().numpy()
    AWo = orc.spmm(A.arrays(), W)
    assert np.max(np.abs(AW - AWo)) <= 1e-13 * np.max(np.abs(AWo))


@pytest.mark.parametrize("n,p,q", [(10007, 13, 7), (257, 1, 40), (50000, 32, 33), (1, 3, 3)])
def test_gram(dev, orc, n, p, q):
    from paper_1512_05820_gb300.solver import gram
    rng = np.random.default_rng(n + p)
    X = np.asfortranarray(rng.normal(size=(n, p)))
    Y = np.asfortranarray(rng.normal(size=(n, q)))
    G = gram(to_dev(X, dev), to_dev(Y, dev)).cpu().numpy()
    Go = orc.gram(X, Y)
    bound = 1e-15 * n * np.outer(np.linalg.norm(X, axis=0), np.linalg.norm(Y, axis=0))
    assert np.all(np.abs(G - Go) <= bound + 1e-300)


@pytest.mark.parametrize("s", [1, 5, 12, 40])
def test_pod(dev, orc, s):
    from paper_1512_05820_gb300.solver import pod
    S, _ = pins._snapshots(n=3000, s=max(s, 1), seed=s)
    S = np.asfortranarray(S[:, :s])
    W, w, sig2 = pod(to_dev(S, dev), 0.9999, 32)
    Wo, wo, sig2o = orc.pod_evd(S, 0.9999, 32)
    assert w == wo
    assert np.max(np.abs(sig2.cpu().numpy() - sig2o)) <= 1e-13 * sig2o[0]
    W = W.cpu().numpy()
    assert np.max(np.abs(W.T @ W - np.eye(w))) <= 1e-10
    cos = np.linalg.svd(W.T @ Wo, compute_uv=False)
    assert cos.min() >= 1 - 1e-10


# ------------------------------------------------------------------ whole solves


def run_parity(dev, seq, n_systems=None, tol_a=1e-10, **cfg):
    from paper_1512_05820_gb300.solver import DeviceCSR, PodCG
    orc = Oracle()
    oseq = OracleSequence(seq.n, s_max=seq.s_max, w_max=seq.w_max, energy=seq.energy, oracle=orc)
    solver = PodCG(seq.n, w_max=seq.w_max, s_max=seq.s_max, energy=seq.energy, cond_diag=1, **cfg)
    A0 = DeviceCSR.from_numpy(seq.row_ptr, seq.col, np.zeros(seq.nnz), device=dev)
    out = []
    for j, val, b in seq.systems():
        if n_systems and j > n_systems:
            break
        A = (seq.row_ptr, seq.col, val)
        x, st = solver.solve(A0.with_values(to_dev(val, dev)), to_dev(b, dev), seq.tol)
        W_j = oseq.basis()[0]
        xo, info = oseq.solve(A, b, seq.tol)
        solver.add_snapshots(to_dev(xo, dev))
        x = x.cpu().numpy()
        assert st["status"] == "ok", st
        assert st["w"] == info["w"], (j, st["w"], info["w"])
        assert abs(st["iters"] - info["iters"]) <= 1, (j, st["iters"], info["iters"])
        if st["iters"] != info["iters"] and st["refinements"] == 0 and info["refinements"] == 0:
            # The exit test ||r_k|| <= tol ||b|| landed within rounding of the threshold, so
            # one side stopped one step later; compare the iterates at the GPU's count.
            xo_k, info_k, _, _ = orc.solve_system(A, b, W_j, 0.0, kmax=st["iters"], max_refine=0)
            assert info_k["iters"] == st["iters"]
            err = a_err(orc, A, x, xo_k)
        else:
            err = a_err(orc, A, x, xo)
        true_rel = np.linalg.norm(b - orc.spmv(A, x)) / np.linalg.norm(b)
        out.append((j, st, info, err))
        assert err <= tol_a, f"system {j}: A-norm diff {err:.2e}"
        assert true_rel <= seq.tol and st["final_relres"] <= seq.tol
        if info["w"] > 0:
            assert abs(st["stage1_relres"] - info["stage1_relres"]) <= 1e-8 * info["stage1_relres"]
            assert abs(st["cond_gram"] - info["cond_gram"]) <= 1e-8 * info["cond_gram"]
    solver.close()
    return out


def test_sequence_2d_64(dev):
    """The 64x64 five-point sequence (10 systems, w <= 8) system by system."""
    out = run_parity(dev, wl.diffusion2d_drift())
    assert out[-1][1]["w"] > 0


def test_sequence_2d_ragged(dev):
    """A 37x41-like ragged grid size (n not a multiple of the block) with a wider basis."""
    seq = wl.diffusion2d_drift(m=37, p=8, w_max=16)
    run_parity(dev, seq)


def test_sequence_3d_small(dev):
    """The moving-source 3D sequence on a 20^3 grid (n = 8000), window 12, w <= 32."""
    seq = wl.diffusion3d_moving(m=20, p=14, s_max=12, w_max=32, period=14)
    run_parity(dev, seq)


def test_plain_pcg(dev, orc):
    """No snapshots: the GPU runs plain Jacobi PCG; same iterate as the oracle's PCG."""
    from paper_1512_05820_gb300.solver import PodCG
    seq = wl.diffusion3d_moving(m=16, p=1)
    j, val, b = next(iter(seq.systems()))
    A = (seq.row_ptr, seq.col, val)
    solver = PodCG(seq.n)
    x, st = solver.solve(dcsr(A, dev), to_dev(b, dev), 1e-10)
    xo, k, stat = orc.pcg(A, b, None, 1e-10 * np.linalg.norm(b))
    assert st["w"] == 0 and abs(st["iters"] - k) <= 1
    assert a_err(orc, A, x.cpu().numpy(), xo) <= 1e-10


def test_stage_one_exact(dev, orc):
    """x* in the span of the snapshots: stage one returns it and no iteration runs."""
    from paper_1512_05820_gb300.solver import PodCG
    A = pins.small_diffusion(30, seed=4)
    rng = np.random.default_rng(5)
    xs = rng.normal(size=A.n)
    b = orc.spmv(A.arrays(), xs)
    solver = PodCG(A.n, w_max=8)
    solver.add_snapshots(to_dev(np.stack([xs + rng.normal(size=A.n), xs - 0.5 * rng.normal(size=A.n), xs], 1), dev))
    x, st = solver.solve(dcsr(A, dev), to_dev(b, dev), 1e-9)
    assert st["iters"] == 0 and st["w"] == 3
    assert np.linalg.norm(x.cpu().numpy() - xs) <= 1e-11 * np.linalg.norm(xs)


# ------------------------------------------------------------------ edge and error cases


def test_edge_single_row_and_zero_rhs(dev):
    from paper_1512_05820_gb300.solver import PodCG
    A = wl.DiffusionOperator((1, 1)).csr(np.array([2.0]))
    s = PodCG(1)
    x, st = s.solve(dcsr(A, dev), to_dev(np.array([3.0]), dev), 1e-12)
    assert abs(x.item() - 3.0 / A.val[0]) <= 1e-15 and st["iters"] <= 1
    B = wl.DiffusionOperator((9, 9)).csr(np.ones(81))
    s2 = PodCG(81)
    x, st = s2.solve(dcsr(B, dev), to_dev(np.zeros(81), dev), 1e-8)
    assert st["iters"] == 0 and float(x.abs().max()) == 0.0


def test_edge_ragged_rows(dev, orc):
    """Heavy-tailed row lengths and diagonal-only rows."""
    from paper_1512_05820_gb300.solver import PodCG
    A = wl.random_spd_csr(4099, 0.004, seed=9, empty_rows=33)
    b = np.random.default_rng(2).normal(size=A.n)
    s = PodCG(A.n)
    x, st = s.solve(dcsr(A, dev), to_dev(b, dev), 1e-10)
    xo, k, _ = orc.pcg(A.arrays(), b, None, 1e-10 * np.linalg.norm(b))
    assert st["status"] == "ok" and abs(st["iters"] - k) <= 1
    assert a_err(orc, A.arrays(), x.cpu().numpy(), xo) <= 1e-10


def test_error_not_spd(dev):
    from paper_1512_05820_gb300.solver import PodCG, PodCGError
    A = wl.DiffusionOperator((8, 8)).csr(np.ones(64))
    val = A.val.copy()
    diag_idx = [k for i in range(64) for k in range(A.row_ptr[i], A.row_ptr[i + 1]) if A.col[k] == i]
    val[diag_idx[5]] = -1.0
    s = PodCG(64)
    with pytest.raises(PodCGError) as e:
        s.solve(dcsr((A.row_ptr, A.col, val), dev), to_dev(np.ones(64), dev), 1e-8)
    assert e.value.status == 2
    # the handle stays usable
    x, st = s.solve(dcsr(A, dev), to_dev(np.ones(64), dev), 1e-8)
    assert st["status"] == "ok"


def test_error_breakdown(dev):
    """Positive diagonal but indefinite: (A p, p) <= 0 is detected."""
    from paper_1512_05820_gb300.solver import PodCG, PodCGError
    D = np.array([[1.0, 3.0], [3.0, 1.0]])
    A = pins.dense_to_csr(D)
    s = PodCG(2)
    with pytest.raises(PodCGError) as e:
        s.solve(dcsr(A, dev), to_dev(np.array([1.0, -1.0]), dev), 1e-12)
    assert e.value.status == 3


def test_error_maxit_and_nonfinite(dev):
    from paper_1512_05820_gb300.solver import PodCG, PodCGError
    A = wl.DiffusionOperator((16, 16)).csr(np.ones(256))
    s = PodCG(256, k_max=3, max_refine=0)
    x, st = s.solve(dcsr(A, dev), to_dev(np.ones(256), dev), 1e-12, raise_on_error=False)
    assert st["status"] == "maxit" and st["iters"] == 3
    b = np.ones(256)
    b[7] = np.nan
    s2 = PodCG(256)
    with pytest.raises(PodCGError) as e:
        s2.solve(dcsr(A, dev), to_dev(b, dev), 1e-8)
    assert e.value.status == 5


def test_arg_errors(dev):
    from paper_1512_05820_gb300.solver import PodCG, PodCGError
    with pytest.raises(PodCGError):
        PodCG(0)
    with pytest.raises(PodCGError):
        PodCG(10, w_max=65)
    s = PodCG(10)
    A = wl.DiffusionOperator((3, 3)).csr(np.ones(9))
    with pytest.raises(PodCGError) as e:
        s.solve(dcsr(A, dev), to_dev(np.ones(10), dev), 1e-8)   # A of order 9, handle of order 10
    assert e.value.status == 1
    with pytest.raises(PodCGError) as e:
        s.solve(dcsr(wl.DiffusionOperator((2, 5)).csr(np.ones(10)), dev), to_dev(np.ones(10), dev), -1.0)
    assert e.value.status == 1


# ------------------------------------------------------------------ loop forms, precision, adjoint


def _gpu_sequence(dev, seq, n_systems, **cfg):
    from paper_1512_05820_gb300.solver import DeviceCSR, PodCG
    solver = PodCG(seq.n, w_max=seq.w_max, s_max=seq.s_max, energy=seq.energy, **cfg)
    A0 = DeviceCSR.from_numpy(seq.row_ptr, seq.col, np.zeros(seq.nnz), device=dev)
    xs, sts = [], []
    for j, val, b in seq.systems():
        if j > n_systems:
            break
        x, st = solver.solve(A0.with_values(to_dev(val, dev)), to_dev(b, dev), seq.tol)
        solver.add_snapshots(x)
        xs.append(x.clone())
        sts.append(st)
    solver.close()
    return xs, sts


def test_loop_modes_bitwise_equal(dev):
    """The conditional-graph loop and the chunked plain-graph loop run the same kernels
    with the same launch shapes, so the iterates are identical bit for bit."""
    seq = wl.diffusion3d_moving(m=18, p=5, s_max=6, w_max=8, period=10)
    xa, sa = _gpu_sequence(dev, seq, 5, loop_mode=0)
    xb, sb = _gpu_sequence(dev, seq, 5, loop_mode=1)
    for a, b, s1, s2 in zip(xa, xb, sa, sb):
        assert torch.equal(a, b)
        assert s1["iters"] == s2["iters"] and s1["w"] == s2["w"]


@pytest.mark.parametrize("loop_mode", [0, 1])
def test_sequence_mixed_precision(dev, loop_mode):
    """FP32 inner CG inside FP64 refinement: the FP64 true residual reaches tol for every
    system, w matches the oracle's, and the solution is within the accuracy that two
    solutions of residual <= tol can differ by (reported, bounded loosely here)."""
    from paper_1512_05820_gb300.solver import DeviceCSR, PodCG
    seq = wl.diffusion3d_moving(m=20, p=10, s_max=10, w_max=16, period=12)
    orc = Oracle()
    oseq = OracleSequence(seq.n, s_max=seq.s_max, w_max=seq.w_max, energy=seq.energy, oracle=orc)
    solver = PodCG(seq.n, w_max=seq.w_max, s_max=seq.s_max, energy=seq.energy, precision=1, loop_mode=loop_mode)
    A0 = DeviceCSR.from_numpy(seq.row_ptr, seq.col, np.zeros(seq.nnz), device=dev)
    for j, val, b in seq.systems():
        A = (seq.row_ptr, seq.col, val)
        x, st = solver.solve(A0.with_values(to_dev(val, dev)), to_dev(b, dev), seq.tol)
        xo, info = oseq.solve(A, b, seq.tol)
        solver.add_snapshots(to_dev(xo, dev))
        x = x.cpu().numpy()
        true_rel = np.linalg.norm(b - orc.spmv(A, x)) / np.linalg.norm(b)
        assert st["status"] == "ok", st
        assert true_rel <= seq.tol and st["final_relres"] <= seq.tol
        assert st["w"] == info["w"]
        assert a_err(orc, A, x, xo) <= 1e-5
        assert st["refinements"] >= 1


def test_adjoint_reuses_forward_factors(dev, orc):
    """lambda = A_j^{-1} g with the basis of forward system j (A_j symmetric): same
    iterate as the oracle's solve with that basis, to the FP64 parity tolerance."""
    from paper_1512_05820_gb300.solver import DeviceCSR, PodCG
    seq = wl.diffusion3d_moving(m=16, p=6, s_max=6, w_max=8, period=10)
    oseq = OracleSequence(seq.n, s_max=seq.s_max, w_max=seq.w_max, energy=seq.energy, oracle=orc)
    solver = PodCG(seq.n, w_max=seq.w_max, s_max=seq.s_max, energy=seq.energy, keep_factors=3)
    A0 = DeviceCSR.from_numpy(seq.row_ptr, seq.col, np.zeros(seq.nnz), device=dev)
    g = np.random.default_rng(3).normal(size=seq.n)
    kept = []
    for j, val, b in seq.systems():
        Wo, wo, _ = oseq.basis()
        x, st = solver.solve(A0.with_values(to_dev(val, dev)), to_dev(b, dev), seq.tol)
        xo, info = oseq.solve((seq.row_ptr, seq.col, val), b, seq.tol)
        solver.add_snapshots(to_dev(xo, dev))
        kept.append((st["system_id"], val, Wo))
    for sysid, val, Wo in kept[-3:]:
        A = (seq.row_ptr, seq.col, val)
        lam, st = solver.solve_adjoint(sysid, A0.with_values(to_dev(val, dev)), to_dev(g, dev), 1e-10)
        lo, info, _, _ = orc.solve_system(A, g, Wo, 1e-10)
        assert st["w"] == Wo.shape[1] and abs(st["iters"] - info["iters"]) <= 1
        assert a_err(orc, A, lam.cpu().numpy(), lo) <= 1e-10
    # evicted system
    from paper_1512_05820_gb300.solver import PodCGError
    with pytest.raises(PodCGError) as e:
        solver.solve_adjoint(kept[0][0], A0.with_values(to_dev(kept[0][1], dev)), to_dev(g, dev), 1e-8)
    assert e.value.status == 9
