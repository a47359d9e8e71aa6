"""Differentiation through a sequence of solves: GPU assembly, adjoint solves reusing the
forward bases, and the fused edge-wise dL/dtheta kernel, against independent references:
dense solves with dA/dtheta from complex-step differentiation of the generator, and
central finite differences of the loss."""
import numpy as np
import pytest

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


@pytest.mark.parametrize("shape", [(7, 13), (4, 5, 6), (1, 1), (3, 1, 2)])
def test_assemble_matches_generator(dev, shape):
    from paper_1512_05820_gb300.adjoint import DiffusionProblem, assemble
    op = wl.DiffusionOperator(shape)
    rng = np.random.default_rng(len(shape))
    theta = rng.normal(0, 0.5, op.n)
    u = rng.uniform(size=op.n)
    prob = DiffusionProblem.from_operator(op, shifts=np.stack([0.01 * u, 0.02 * u]), device=dev)
    for j in range(2):
        v = assemble(prob, torch.as_tensor(theta, device=dev), j).cpu().numpy()
        ref = op.values(np.exp(theta), (j + 1) * 0.01 * u)
        assert np.max(np.abs(v - ref) / np.abs(ref)) <= 4e-15


def _problem(m, p, seed, dev):
    from paper_1512_05820_gb300.adjoint import DiffusionProblem
    op = wl.DiffusionOperator((m, m, m))
    rng = np.random.default_rng(seed)
    theta = rng.normal(0, 0.5, op.n)
    u = rng.uniform(size=op.n)
    shifts = np.stack([0.01 * (j + 1) * u for j in range(p)])
    B = np.stack([op.gaussian((m / 2 + m / 4 * np.cos(j), m / 2 + m / 4 * np.sin(j), m / 2), 1.5) for j in range(p)])
    c = rng.normal(size=op.n)
    prob = DiffusionProblem.from_operator(op, shifts=shifts, device=dev, tol=1e-13, w_max=8, s_max=8)
    return op, theta, shifts, B, c, prob


def _gpu_loss_grad(theta, B, c, prob, dev):
    from paper_1512_05820_gb300.adjoint import solve_sequence
    th = torch.as_tensor(theta, device=dev).requires_grad_(True)
    Bt = torch.as_tensor(B, device=dev).requires_grad_(True)
    X = solve_sequence(th, Bt, prob)
    loss = (X * torch.as_tensor(c, device=dev)).sum()
    loss.backward()
    return float(loss), th.grad.cpu().numpy(), Bt.grad.cpu().numpy(), X.detach().cpu().numpy()


def test_gradient_vs_dense_complex_step(dev):
    """8^3 grid, 3 systems: dL/dtheta and dL/dB against dense solves, with dA/dtheta_c from
    complex-step differentiation of the generator (no formula shared with the kernel)."""
    op, theta, shifts, B, c, prob = _problem(8, 3, 1, dev)
    loss, g_theta, g_B, X = _gpu_loss_grad(theta, B, c, prob, dev)
    rows = np.repeat(np.arange(op.n), np.diff(op.row_ptr))
    m = np.zeros(op.nnz)
    loss_ref = 0.0
    for j in range(3):
        A = op.csr(np.exp(theta), shifts[j]).todense()
        x = np.linalg.solve(A, B[j])
        lam = np.linalg.solve(A, c)
        loss_ref += c @ x
        assert np.linalg.norm(X[j] - x) <= 1e-10 * np.linalg.norm(x)
        assert np.linalg.norm(g_B[j] - lam) <= 1e-10 * np.linalg.norm(lam)
        m += lam[rows] * x[op.col]
    h = 1e-30
    g_ref = np.empty(op.n)
    for cc in range(op.n):
        th = theta.astype(np.complex128)
        th[cc] += 1j * h
        dval = op.values(np.exp(th)).imag / h
        g_ref[cc] = -(dval * m).sum()
    assert abs(loss - loss_ref) <= 1e-11 * abs(loss_ref)
    assert np.max(np.abs(g_theta - g_ref)) <= 1e-8 * np.max(np.abs(g_ref))


def test_gradient_vs_central_differences(dev):
    """24^3 grid, 4 systems: dL/dtheta at 6 random cells against the fourth-order central
    difference of the loss (h = 1e-3), each loss from GPU solves at tol 1e-13."""
    op, theta, shifts, B, c, prob = _problem(24, 4, 2, dev)
    loss, g_theta, _, _ = _gpu_loss_grad(theta, B, c, prob, dev)
    from paper_1512_05820_gb300.adjoint import solve_sequence

    def L(th):
        with torch.no_grad():
            X = solve_sequence(torch.as_tensor(th, device=dev), torch.as_tensor(B, device=dev), prob)
            return float((X * torch.as_tensor(c, device=dev)).sum())

    rng = np.random.default_rng(7)
    cells = rng.choice(op.n, size=6, replace=False)
    h = 1e-3
    scale = np.max(np.abs(g_theta))
    for cc in cells:
        e = np.zeros(op.n)
        e[cc] = h
        fd = (-L(theta + 2 * e) + 8 * L(theta + e) - 8 * L(theta - e) + L(theta - 2 * e)) / (12 * h)
        assert abs(fd - g_theta[cc]) <= 1e-6 * max(abs(g_theta[cc]), 1e-3 * scale), (cc, fd, g_theta[cc])


@pytest.mark.parametrize("shape", [(11, 13, 17), (29, 31), (1, 1), (3, 1, 2)])
def test_theta_grad_kernel_vs_oracle(dev, orc, shape):
    """The fused edge-wise dL/dtheta kernel against the oracle's face-by-face formula on the
    same random theta, lambda, x (3 systems): element-wise to 1e-13 of a bound on the sum of
    the absolute face terms of a cell."""
    from paper_1512_05820_gb300.adjoint import DiffusionProblem, theta_grad
    op = wl.DiffusionOperator(shape)
    rng = np.random.default_rng(op.n + 3)
    theta = rng.normal(0, 0.5, op.n)
    lam = rng.normal(size=(3, op.n))
    xs = rng.normal(size=(3, op.n))
    prob = DiffusionProblem.from_operator(op, device=dev)
    g = theta_grad(prob, torch.as_tensor(theta, device=dev), torch.as_tensor(lam, device=dev),
                   torch.as_tensor(xs, device=dev)).cpu().numpy()
    ref = orc.theta_grad(op.shape3, theta, lam, xs)
    # a bound free of cancellation: each of the <= 6 faces of 3 systems contributes at most
    # 2 k_max * 2|lam|_max * 2|x|_max in magnitude
    bound = 1e-13 * (6 * 3 * 8 * np.exp(np.abs(theta)).max() * np.abs(lam).max() * np.abs(xs).max())
    assert np.max(np.abs(g - ref)) <= bound, np.max(np.abs(g - ref))


def test_checkpointed_backward_matches_kept_factors(dev):
    """16^3 grid, 5 systems, window 3: the default backward recomputes each W_j, A_j W_j and
    stage-one factor from the checkpointed solutions; the gradient equals the one from the
    forward handle's kept factors (pod_cg_solve_adjoint) to the solves' accuracy (1e-13)."""
    import dataclasses
    op, theta, shifts, B, c, prob = _problem(16, 5, 4, dev)
    prob = dataclasses.replace(prob, s_max=3)
    _, g1, gB1, X1 = _gpu_loss_grad(theta, B, c, prob, dev)
    _, g2, gB2, X2 = _gpu_loss_grad(theta, B, c, dataclasses.replace(prob, checkpoint=False), dev)
    assert np.array_equal(X1, X2)
    assert np.max(np.abs(g1 - g2)) <= 1e-10 * np.max(np.abs(g2))
    assert np.max(np.abs(gB1 - gB2)) <= 1e-10 * np.max(np.abs(gB2))


def test_gradient_full_size_96_central_differences(dev):
    """The differentiation workload at full grid size: 96^3 cells (n = 884,736), theta ~
    N(0, 0.5^2), 8 systems of the sequence, loss sum_j c^T x_j, checkpointed backward.
    dL/dtheta at the three cells of largest |g| among 64 seeded random ones against the
    fourth-order central difference (h = 1e-3), solves at 1e-13: norm-wise relative error
    <= 1e-6."""
    from paper_1512_05820_gb300.adjoint import DiffusionProblem, solve_sequence
    seq = wl.diffusion3d_theta(m=96, p=8)
    r = seq.recipe
    shifts = np.stack([0.01 * (j + 1) * r["u"] for j in range(seq.p)])
    B = torch.as_tensor(np.stack([b for _, _, b in seq.systems()]), device=dev)
    c = torch.as_tensor(r["c"], device=dev)
    prob = DiffusionProblem.from_operator(seq.op, shifts=shifts, device=dev, tol=1e-13, w_max=32, s_max=40)
    th = torch.as_tensor(r["theta"], device=dev).requires_grad_(True)
    X = solve_sequence(th, B, prob)
    (X * c).sum().backward()
    g = th.grad.cpu().numpy()

    def L(theta):
        with torch.no_grad():
            return float((solve_sequence(torch.as_tensor(theta, device=dev), B, prob) * c).sum())

    rng = np.random.default_rng(5)
    cand = rng.choice(seq.n, size=64, replace=False)
    cells = cand[np.argsort(-np.abs(g[cand]))[:3]]
    h = 1e-3
    fds = []
    for cc in cells:
        e = np.zeros(seq.n)
        e[cc] = h
        th0 = r["theta"]
        fds.append((-L(th0 + 2 * e) + 8 * L(th0 + e) - 8 * L(th0 - e) + L(th0 - 2 * e)) / (12 * h))
    err = np.linalg.norm(np.array(fds) - g[cells]) / np.linalg.norm(g[cells])
    print(f"96^3, 8 systems: gradient at cells {list(cells)}, norm-wise error vs finite differences {err:.2e}")
    assert err <= 1e-6
