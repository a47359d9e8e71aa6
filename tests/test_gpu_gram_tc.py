"""Tensor-core split-bf16 Gram (pod_cg_gram_tc) against the FP64 oracle Gram, and solves
that use it for the stage-one reduced matrix.

Reference: the oracle's FP64 X^T [Y, e] of the inputs rounded to FP32 (the kernel rounds
every input to FP32 first; exact for FP32 inputs). Error bound per entry, from the
arithmetic: the bf16 part products are exact in FP32; per 128-row window the FP32 TMEM
accumulator takes at most 32 MMA additions (8 K-steps x 4 part products), each adding at
most a couple of FP32 roundings (2^-23 relative to the running sum and the 16 added
products); windows are summed Kahan-compensated in FP32 and CTAs in FP64; the dropped part
products (lo*mid, lo*lo when p > 42) weigh <= 2^-24. Altogether
|G - G_ref| <= 2^-16 * sum_i |x_ia| |y_ic|, with the FP32 rounding of FP64 inputs
(2 * 2^-24 * the same sum) on top for FP64 inputs.
"""
import numpy as np
import pytest

from paper_1512_05820_gb300 import workloads as wl

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

BOUND = 2.0 ** -16


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1512_05820_gb300 import _lib
    _lib.load()
    return torch.device("cuda:0")


def _inputs(n, p, qy, extra, dtype, seed):
    rng = np.random.default_rng(seed)
    X = rng.normal(size=(n, p)) * np.exp(rng.normal(size=p))        # column scales vary
    Y = rng.normal(size=(n, qy)) * np.exp(rng.normal(size=qy))
    e = rng.normal(size=n) if extra else None
    return X.astype(dtype), Y.astype(dtype), e


def _check(dev, orc, X, Y, e, rounding):
    from paper_1512_05820_gb300.solver import gram_tc
    n, p = X.shape
    qy = Y.shape[1]
    Xd = torch.as_tensor(X, device=dev)
    Yd = torch.as_tensor(Y, device=dev) if qy > 0 else None
    ed = torch.as_tensor(e, device=dev) if e is not None else None
    G = gram_tc(Xd, Yd, ed).cpu().numpy()
    # reference: FP64 oracle Gram of the values the kernel multiplies
    cols = [Y.astype(np.float64)] if qy > 0 else []
    if e is not None:
        cols.append(e.astype(np.float32).astype(np.float64)[:, None])
    Yr = np.hstack(cols)
    Xr = X.astype(np.float32).astype(np.float64)
    Yr32 = Yr.astype(np.float32).astype(np.float64)
    G_ref = orc.gram(Xr, Yr32) if rounding else orc.gram(X.astype(np.float64), Yr)
    absum = np.abs(Xr).T @ np.abs(Yr32)
    bound = BOUND * absum + (2.0 * 2.0 ** -24 * absum if rounding is False else 0.0)
    err = np.abs(G - G_ref)
    assert G.shape == (p, Yr.shape[1])
    assert np.all(np.isfinite(G))
    assert np.all(err <= bound + 1e-300), f"max err/absum {np.max(err / (absum + 1e-300)):.3e}"
    G2 = gram_tc(Xd, Yd, ed).cpu().numpy()
    assert np.array_equal(G, G2), "not deterministic"
    return float(np.max(err / (absum + 1e-300)))


@pytest.mark.parametrize("n,p,qy,extra", [
    (5004, 22, 22, True),     # the stage-one shape W^T [AW, b], three stacked parts
    (5004, 42, 42, False),    # 3p = 126: last width with all nine part products
    (5004, 43, 43, True),     # 3p > 128: [hi; mid] + [lo; 0], seven products
    (5004, 64, 64, True),     # q = 65: widest tile, N = 80
    (5004, 1, 0, True),       # one column against b only
    (32, 8, 8, False),        # a single chunk
    (100, 5, 3, True),        # fewer chunks than SMs, ragged tail
    (300_000, 32, 32, True),  # several chunks per CTA, several flush windows
])
def test_gram_tc_fp32(dev, orc, n, p, qy, extra):
    X, Y, e = _inputs(n, p, qy, extra, np.float32, n + p)
    _check(dev, orc, X, Y, e, rounding=True)


@pytest.mark.parametrize("n,p,qy,extra", [(5002, 22, 22, True), (5002, 48, 48, True), (70, 3, 2, False)])
def test_gram_tc_fp64(dev, orc, n, p, qy, extra):
    X, Y, e = _inputs(n, p, qy, extra, np.float64, n + 7 * p)
    _check(dev, orc, X, Y, e, rounding=False)


def test_gram_tc_full_size(dev, orc):
    """The stage-one shape of the 128^3 workload: n = 2,097,152, W (n x 22) FP32 against
    [AW (n x 22), b], every entry checked against the oracle."""
    X, Y, e = _inputs(2_097_152, 22, 22, True, np.float32, 2097)
    r = _check(dev, orc, X, Y, e, rounding=True)
    assert r <= BOUND


def test_gram_tc_arg_errors(dev):
    from paper_1512_05820_gb300.solver import gram_tc, PodCGError
    X = torch.zeros((5001, 4), dtype=torch.float32, device=dev)    # 5001 * 4 bytes: not 16-aligned
    with pytest.raises(PodCGError):
        gram_tc(X, X)
    X = torch.zeros((64, 65), dtype=torch.float32, device=dev)     # p > 64
    with pytest.raises(PodCGError):
        gram_tc(X, X[:, :2])


def test_tc_gram_needs_mixed_precision(dev):
    from paper_1512_05820_gb300.solver import PodCG, PodCGError
    with pytest.raises(PodCGError):
        PodCG(1000, precision=0, use_tc_gram=1)


@pytest.mark.parametrize("precision", [1])
def test_solves_with_tc_gram(dev, precision):
    """Mixed precision with the tensor-core reduced matrix: every system reaches tol with the
    same basis width as with the CUDA-core FP32 Gram, in a comparable number of iterations."""
    from paper_1512_05820_gb300.solver import DeviceCSR, PodCG
    seq = wl.diffusion3d_moving(m=24, p=8, s_max=8, w_max=16, period=10)
    res = {}
    for tc in (0, 1):
        solver = PodCG(seq.n, w_max=seq.w_max, s_max=seq.s_max, energy=seq.energy, precision=precision,
                       use_tc_gram=tc)
        A0 = DeviceCSR.from_numpy(seq.row_ptr, seq.col, np.zeros(seq.nnz), device=dev)
        sts = []
        for j, val, b in seq.systems():
            x, st = solver.solve(A0.with_values(torch.as_tensor(val, device=dev)), torch.as_tensor(b, device=dev),
                                 seq.tol)
            assert st["status"] == "ok", st
            assert st["final_relres"] <= seq.tol
            solver.add_snapshots(x)
            sts.append(st)
        solver.close()
        res[tc] = sts
    for s0, s1 in zip(res[0], res[1]):
        assert s0["w"] == s1["w"]
        assert s1["iters"] <= 1.05 * s0["iters"] + 3, (s0["iters"], s1["iters"])
        if s0["w"] > 0:
            assert abs(s1["stage1_relres"] - s0["stage1_relres"]) <= 1e-3 * s0["stage1_relres"]


def test_auto_gram_choice(dev):
    """use_tc_gram = -1 (the default): on a system of >= 65,536 rows the handle times both
    stage-one Grams once per basis width and reports which ran (stats gram_tc); the solve
    matches the forced CUDA-core and tensor-core runs' basis width and accuracy. Below 65,536
    rows the CUDA-core Gram runs without timing."""
    from paper_1512_05820_gb300.solver import DeviceCSR, PodCG
    seq = wl.diffusion3d_moving(m=42, p=4, s_max=4, w_max=8, period=10)   # n = 74,088
    assert seq.n >= 65536
    systems = seq.all_systems()
    A0 = DeviceCSR.from_numpy(seq.row_ptr, seq.col, np.zeros(seq.nnz), device=dev)
    runs = {}
    for tc in (-1, 0, 1):
        solver = PodCG(seq.n, w_max=seq.w_max, s_max=seq.s_max, energy=seq.energy, precision=1, use_tc_gram=tc)
        sts = []
        for j, val, b in systems:
            x, st = solver.solve(A0.with_values(torch.as_tensor(val, device=dev)), torch.as_tensor(b, device=dev),
                                 seq.tol)
            assert st["status"] == "ok" and st["final_relres"] <= seq.tol, st
            solver.add_snapshots(x)
            sts.append(st)
        solver.close()
        runs[tc] = sts
    for k, st in enumerate(runs[-1]):
        if st["w"] == 0:
            assert st["gram_tc"] == 0
        assert st["gram_tc"] in (0, 1)
        assert st["w"] == runs[0][k]["w"] == runs[1][k]["w"]
    assert all(st["gram_tc"] == 1 for st in runs[1] if st["w"] > 0)
    assert all(st["gram_tc"] == 0 for st in runs[0])
    small = wl.diffusion2d_drift(m=40, p=3)
    solver = PodCG(small.n, w_max=small.w_max, s_max=small.s_max, energy=small.energy, precision=1)
    A0 = DeviceCSR.from_numpy(small.row_ptr, small.col, np.zeros(small.nnz), device=dev)
    for j, val, b in small.systems():
        x, st = solver.solve(A0.with_values(torch.as_tensor(val, device=dev)), torch.as_tensor(b, device=dev),
                             small.tol)
        solver.add_snapshots(x)
        assert st["gram_tc"] == 0
    solver.close()
