"""The oracle pinned against closed forms, LAPACK special cases and method invariants.

Planted-mistake builds (``-DORC_MUTANT=k``) show each pin set is sensitive: every
mutant must fail at least one pin.
"""
import numpy as np
import pytest

import pins
from oracle import Oracle


@pytest.mark.parametrize("pin", pins.ALL_PINS + [pins.pin_generator_2x2], ids=lambda f: f.__name__)
def test_pin(orc, pin):
    ok, detail = pin(orc)
    assert ok, detail


MUTANTS = {
    1: "beta dropped from the direction update",
    2: "sign of the W mu term flipped",
    3: "bhat formed with AW instead of W",
    4: "Jacobi preconditioner multiplies by diag(A) instead of its inverse",
    5: "POD lift without 1/sigma",
    6: "energy criterion on sigma instead of sigma^2",
    7: "Cholesky reads a wrong, scaled entry",
    8: "residual update with p instead of A p",
    9: "wrong sign in the eigenvector rotation",
    10: "SpMV drops the first entry of each row",
    11: "interior-face derivative uses its own cell's coefficient instead of the neighbour's",
    12: "stage two drops the stage-one deflation term from the direction update",
    13: "stage-three factor takes T2 instead of its square root",
    14: "stage-two initial residual omits the stage-one solution's product",
    15: "stage two skips the re-A-orthogonalisation of its directions",
    16: "inner reduced solves start from zero instead of the Galerkin solution over the stored basis",
    17: "one-sided Jacobi SVD rotates the second column with the wrong sign",
    18: "output-metric POD lift without 1/sigma",
    19: "A-metric POD Gram symmetrised with a sign error",
    20: "stage two's dependence test sums the Gram-Schmidt coefficients instead of the A-norm they remove",
}


@pytest.mark.parametrize("k", sorted(MUTANTS))
def test_planted_mistake_is_caught(k, tmp_path):
    mut = Oracle(mutant=k, out_dir=str(tmp_path))
    failed = []
    for pin in pins.ALL_PINS:
        try:
            ok, detail = pin(mut)
        except Exception as e:  # a crash or a numpy error also counts as caught
            ok, detail = False, repr(e)
        if not ok:
            failed.append(pin.__name__)
    assert failed, f"mutant {k} ({MUTANTS[k]}) passed every pin"


def test_cg_rounding_sensitivity_elasticity(orc):
    """The oracle's Jacobi-PCG on the 6^3-element cantilever (n = 882, system 1) against an
    independent FP64 CG written here with numpy's dot products (another summation order).
    After the same number of steps the two iterates differ by about 1e-9 in the A-norm,
    the size of the error left at tol = 1e-8: on this operator FP64 rounding alone moves
    the iterate by that much, so GPU parity on it is bounded by 5e-9, not 1e-10."""
    import scipy.sparse as sp
    from paper_1512_05820_gb300 import workloads as wl
    seq = wl.elasticity_cantilever(e=6, p=1, w_max=8, s_max=8)
    j, val, b = next(iter(seq.systems()))
    A = (seq.row_ptr, seq.col, val)
    xo, info, _, _ = orc.solve_system(A, b, None, seq.tol)
    M = sp.csr_matrix((val, seq.col, seq.row_ptr), shape=(seq.n, seq.n))
    d = M.diagonal()
    x = np.zeros(seq.n)
    r = b.copy()
    z = r / d
    p = z.copy()
    rz = float(np.dot(r, z))
    for _ in range(info["iters"]):
        q = M @ p
        a = rz / float(np.dot(p, q))
        x += a * p
        r -= a * q
        z = r / d
        rz_new = float(np.dot(r, z))
        p = z + (rz_new / rz) * p
        rz = rz_new

    def anorm(v):
        return float(np.sqrt(v @ (M @ v)))

    diff = anorm(x - xo) / anorm(xo)
    err = anorm(xo - sp.linalg.spsolve(M.tocsc(), b)) / anorm(xo)
    assert diff <= 5e-9
    assert diff >= 1e-11   # the sensitivity is real: far above a pure rounding level
    assert err <= 1e-8


GOLDEN = {"c1_sequence_oracle.json": dict(), "c1_three_stage_oracle.json": dict(three_stage=True),
          "c1_output_pod_oracle.json": dict(metric="output"), "c1_metric_a_oracle.json": dict(metric="a")}


@pytest.mark.parametrize("name", sorted(GOLDEN))
def test_golden_c1_sequence_record(name):
    """The oracle reproduces its committed records of the 64x64 sequence: two stages, three
    stages, and the POD metrics C^T C and A (written by tests/golden/make_golden.py):
    iteration counts, w, k2, y and refinements exactly, residuals and solution norms to
    1e-12 relative. Guards the oracle against unintended changes."""
    import json
    import os
    import sys
    here = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
    sys.path.insert(0, here)
    try:
        import make_golden
    finally:
        sys.path.remove(here)
    with open(os.path.join(here, name)) as f:
        ref = json.load(f)
    now = make_golden.record(**GOLDEN[name])
    assert len(now["systems"]) == len(ref["systems"])
    for a, b in zip(now["systems"], ref["systems"]):
        for k in ("system", "iters", "w", "refinements", "k2", "y"):
            assert a.get(k) == b.get(k), (k, a, b)
        for k in ("stage1_relres", "final_relres", "x_norm2", "x_sum", "stage2_relres"):
            if k in b:
                assert abs(a[k] - b[k]) <= 1e-12 * max(abs(b[k]), 1e-300), (k, a[k], b[k])


@pytest.mark.parametrize("shape", [(3, 4), (2, 3, 2), (1, 1), (4, 1, 3)])
def test_theta_grad_vs_complex_step(orc, shape):
    """The oracle's face-by-face dL/dtheta against complex-step differentiation of the
    matrix generator: -sum_j lambda_j^T (dA/dtheta_c) x_j = -Im(sum_j lambda_j^T
    A(exp(theta + i h e_c)) x_j)/h, exact to rounding for h = 1e-30 (arbitrary lambda, x)."""
    from paper_1512_05820_gb300 import workloads as wl
    op = wl.DiffusionOperator(shape)
    rng = np.random.default_rng(op.n)
    theta = rng.normal(0, 0.5, op.n)
    lam = rng.normal(size=(2, op.n))
    xs = rng.normal(size=(2, op.n))
    g = orc.theta_grad(op.shape3, theta, lam, xs)
    h = 1e-30
    ref = np.zeros(op.n)
    for c in range(op.n):
        th = theta.astype(np.complex128)
        th[c] += 1j * h
        val = op.values(np.exp(th))
        for j in range(2):
            Ax = np.zeros(op.n, dtype=np.complex128)
            for i in range(op.n):
                for k in range(op.row_ptr[i], op.row_ptr[i + 1]):
                    Ax[i] += val[k] * xs[j, op.col[k]]
            ref[c] -= np.imag(lam[j] @ Ax) / h
    assert np.max(np.abs(g - ref)) <= 1e-13 * max(1.0, np.max(np.abs(ref)))


def test_adjoint_gradient_end_to_end(orc):
    """For exact solutions x_j = A_j^{-1} b_j and adjoints lambda_j = A_j^{-1} c, the oracle's
    dL/dtheta equals the complex-step derivative of L(theta) = sum_j c^T A_j(theta)^{-1} b_j
    computed with dense complex solves (a route that shares nothing with the face formula)."""
    from paper_1512_05820_gb300 import workloads as wl
    op = wl.DiffusionOperator((3, 3, 2))
    rng = np.random.default_rng(11)
    theta = rng.normal(0, 0.5, op.n)
    u = rng.uniform(size=op.n)
    B = rng.normal(size=(2, op.n))
    c = rng.normal(size=op.n)

    def dense(vals):
        M = np.zeros((op.n, op.n), dtype=vals.dtype)
        for i in range(op.n):
            for k in range(op.row_ptr[i], op.row_ptr[i + 1]):
                M[i, op.col[k]] += vals[k]
        return M

    xs, lams = [], []
    for j in range(2):
        M = dense(op.values(np.exp(theta), 0.01 * (j + 1) * u))
        xs.append(np.linalg.solve(M, B[j]))
        lams.append(np.linalg.solve(M, c))
    g = orc.theta_grad(op.shape3, theta, np.array(lams), np.array(xs))
    h = 1e-30
    ref = np.zeros(op.n)
    for cc in range(op.n):
        th = theta.astype(np.complex128)
        th[cc] += 1j * h
        L = 0.0
        for j in range(2):
            M = dense(op.values(np.exp(th), 0.01 * (j + 1) * u))
            L = L + c @ np.linalg.solve(M, B[j])
        ref[cc] = np.imag(L) / h
    assert np.max(np.abs(g - ref)) <= 1e-11 * np.max(np.abs(ref))


def test_stage_two_past_the_rounding_floor(orc):
    """Why the dependence stop exists: on the cond-1.002 reduced system of
    pins.pin_stage_two_dependence_stop, stage two with tolerance 0 and no stop runs all y
    iterations, and once its residual is rounding noise the single re-A-orthogonalisation
    pass against noise directions amplifies them: the iterate ends far from the Galerkin
    solution. With the stop it ends at the floor, at that solution."""
    A, D, b, Y = pins._near_identity_reduced_problem()
    y = Y.shape[1]
    xg = Y @ np.linalg.solve(Y.T @ D @ Y, Y.T @ b)
    with orc.dependence_stop(False):
        off = orc.stage_two(A, b, Y, 0, None, None, 0.0, y)
    with orc.dependence_stop(True):
        on = orc.stage_two(A, b, Y, 0, None, None, 0.0, y)
    err = lambda o: pins.a_norm(D, o["V2"] @ o["alpha"] - xg) / pins.a_norm(D, xg)
    assert off["k2"] == y and err(off) > 1.0
    assert on["k2"] < y // 2 and err(on) < 1e-12


def test_exact_stage_two_in_a_sequence():
    """The same effect in a sequence: metric-A POD (Y^T A Y = I to rounding), stage-one
    energy 0.9 and stage-two tolerance 0 on the 20^3 moving-source sequence. Without the
    dependence stop, stage two runs past the rounding floor on systems 7 and 8 and their
    solves fail (the iteration cap is reached far from the tolerance); with it, every system
    converges and stage two takes at most two steps."""
    from oracle import Oracle, OracleSequence
    from paper_1512_05820_gb300 import workloads as wl
    orc = Oracle()
    seq = wl.diffusion3d_moving(m=20, p=8, s_max=12, w_max=32, period=14)
    res = {}
    for on in (False, True):
        oseq = OracleSequence(seq.n, s_max=seq.s_max, w_max=seq.w_max, energy=0.9, oracle=orc, three_stage=True,
                              metric_a=True, y_max=12, energy_y=1 - 1e-10, tol_stage2=0.0, kmax=3000)
        with orc.dependence_stop(on):
            res[on] = [oseq.solve((seq.row_ptr, seq.col, val), b, seq.tol)[1] for _, val, b in seq.systems()]
    assert any(i["status"] != "ok" for i in res[False])
    assert all(i["status"] == "ok" and i["final_relres"] <= seq.tol for i in res[True])
    assert max(i["k2"] for i in res[True]) <= 2 and max(i["k2"] for i in res[True]) >= 1


class _KeepFirst:
    """Planted mistake: the window keeps the first s_max snapshots and drops later ones."""

    def add_snapshot(self, x):
        if len(self.snaps) < self.s_max:
            self.snaps.append(np.array(x, dtype=np.float64))


class _EvictNewest:
    """Planted mistake: a full window replaces its newest snapshot instead of its oldest."""

    def add_snapshot(self, x):
        self.snaps.append(np.array(x, dtype=np.float64))
        if len(self.snaps) > self.s_max:
            self.snaps.pop(-2)


class _ShortWindow:
    """Planted mistake: off by one, the window holds s_max - 1 snapshots."""

    def add_snapshot(self, x):
        self.snaps.append(np.array(x, dtype=np.float64))
        while len(self.snaps) >= self.s_max:
            self.snaps.pop(0)


@pytest.mark.parametrize("mistake", [_KeepFirst, _EvictNewest, _ShortWindow], ids=lambda c: c.__name__)
def test_sequence_window_mistake_is_caught(orc, mistake):
    from oracle import OracleSequence
    cls = type("Mutated" + mistake.__name__, (mistake, OracleSequence), {})
    ok, detail = pins.pin_sequence_window(orc, cls)
    assert not ok, f"{mistake.__doc__} passed the window pin: {detail}"
