"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each pin returns ``(ok, detail)`` so that the same checks serve two tests: against the
normal oracle build every pin must hold, and against each build with a planted mistake
(``-DORC_MUTANT=k``) at least one must fail. None of these re-types the oracle's own
formula: they compare against dense LAPACK results (numpy), closed forms, invariants of
the method (Galerkin orthogonality, A-orthogonality, optimality) and brute force.
"""
from __future__ import annotations

import numpy as np

from paper_1512_05820_gb300.workloads import CSR, DiffusionOperator, random_spd_csr


def dense_to_csr(D) -> CSR:
    D = np.asarray(D, dtype=np.float64)
    n = D.shape[0]
    rp = [0]
    cols, vals = [], []
    for i in range(n):
        nz = np.nonzero(D[i])[0]
        cols += list(nz)
        vals += list(D[i, nz])
        rp.append(len(cols))
    return CSR(n, np.array(rp, np.int32), np.array(cols, np.int32), np.array(vals))


def small_diffusion(m=8, seed=0, dim=2):
    rng = np.random.default_rng(seed)
    op = DiffusionOperator((m,) * dim)
    k = np.exp(rng.normal(0, 0.5, op.n))
    return op.csr(k)


def orth_basis(vectors):
    Q, _ = np.linalg.qr(np.asarray(vectors).T if np.ndim(vectors) == 2 else vectors)
    return np.asfortranarray(Q)


def a_norm(D, v):
    return float(np.sqrt(max(v @ (D @ v), 0.0)))


# ---------------------------------------------------------------------------- pins


def pin_spmv_dense(orc):
    """y = A x against the dense product (ragged rows, diagonal-only rows)."""
    A = random_spd_csr(60, 0.1, seed=3, empty_rows=4)
    x = np.random.default_rng(1).normal(size=60)
    y = orc.spmv(A.arrays(), x)
    ref = A.todense() @ x
    err = np.max(np.abs(y - ref)) / np.max(np.abs(ref))
    return err < 1e-14, f"spmv rel err {err:.2e}"


def pin_gram_spmm_dense(orc):
    """G = X^T Y and AW = A W against the dense products (a tall X with a ragged row count,
    the ragged random SPD matrix with diagonal-only rows)."""
    rng = np.random.default_rng(11)
    X = np.asfortranarray(rng.normal(size=(97, 5)))
    Y = np.asfortranarray(rng.normal(size=(97, 7)))
    G = orc.gram(X, Y)
    e1 = np.max(np.abs(G - X.T @ Y)) / np.max(np.abs(X.T @ Y))
    A = random_spd_csr(60, 0.1, seed=3, empty_rows=4)
    W = np.asfortranarray(rng.normal(size=(60, 4)))
    AW = orc.spmm(A.arrays(), W)
    ref = A.todense() @ W
    e2 = np.max(np.abs(AW - ref)) / np.max(np.abs(ref))
    return e1 < 1e-14 and e2 < 1e-14, f"gram {e1:.1e}, spmm {e2:.1e}"


def pin_cholesky_numpy(orc):
    """R^T R = G and R equals the transposed LAPACK lower factor; a non-SPD matrix fails."""
    rng = np.random.default_rng(5)
    B = rng.normal(size=(9, 9))
    G = B @ B.T + 9 * np.eye(9)
    R, st = orc.cholesky(G)
    L = np.linalg.cholesky(G)
    e1 = np.max(np.abs(R.T @ R - G)) / np.max(np.abs(G))
    e2 = np.max(np.abs(R - L.T)) / np.max(np.abs(L))
    G2 = G.copy()
    G2[4, 4] = -1.0
    _, st2 = orc.cholesky(G2)
    y = orc.chol_solve(R, np.arange(9.0))
    e3 = np.max(np.abs(G @ y - np.arange(9.0))) / 9.0
    ok = st == 0 and e1 < 1e-14 and e2 < 1e-13 and st2 == 2 and e3 < 1e-12
    return ok, f"chol st={st} recon {e1:.1e} vs lapack {e2:.1e} nonspd st={st2} solve {e3:.1e}"


def pin_jacobi_closed_form(orc):
    """Eigenvalues of the 1D Dirichlet Laplacian tridiag(-1, 2, -1) of order s are
    2 - 2 cos(k pi/(s+1)); eigenvectors sin(i k pi/(s+1)) (closed form)."""
    s = 12
    T = 2 * np.eye(s) - np.eye(s, k=1) - np.eye(s, k=-1)
    ev, V, sweeps = orc.jacobi_eig(T)
    k = np.arange(1, s + 1)
    ref = np.sort(2 - 2 * np.cos(k * np.pi / (s + 1)))[::-1]
    e1 = np.max(np.abs(ev - ref))
    # eigenvector for the largest eigenvalue (k = s): sin(i s pi/(s+1)), i = 1..s
    i = np.arange(1, s + 1)
    v = np.sin(i * s * np.pi / (s + 1))
    v /= np.linalg.norm(v)
    e2 = 1 - abs(v @ V[:, 0])
    return e1 < 1e-13 and e2 < 1e-13, f"jacobi closed-form eig err {e1:.1e}, vec {e2:.1e}, sweeps {sweeps}"


def pin_jacobi_vs_eigh(orc):
    """Random symmetric matrix: eigenvalues match LAPACK eigh; G V = V diag(ev); V^T V = I;
    largest-magnitude entry of every eigenvector is positive."""
    rng = np.random.default_rng(11)
    B = rng.normal(size=(20, 20))
    G = B + B.T
    ev, V, _ = orc.jacobi_eig(G)
    ref = np.sort(np.linalg.eigvalsh(G))[::-1]
    e1 = np.max(np.abs(ev - ref)) / np.max(np.abs(ref))
    e2 = np.max(np.abs(G @ V - V * ev)) / np.max(np.abs(ref))
    e3 = np.max(np.abs(V.T @ V - np.eye(20)))
    sign_ok = all(V[np.argmax(np.abs(V[:, j])), j] > 0 for j in range(20))
    return e1 < 1e-13 and e2 < 1e-12 and e3 < 1e-13 and sign_ok, \
        f"eigh err {e1:.1e} resid {e2:.1e} orth {e3:.1e} sign {sign_ok}"


def _snapshots(n=300, s=12, seed=2):
    rng = np.random.default_rng(seed)
    # decaying singular values so that the energy criterion bites
    U, _ = np.linalg.qr(rng.normal(size=(n, s)))
    V, _ = np.linalg.qr(rng.normal(size=(s, s)))
    sig = 10.0 ** (-0.6 * np.arange(s))
    return np.asfortranarray(U @ np.diag(sig) @ V.T), sig


def pin_pod_svd(orc):
    """POD (Section 3.1 / Algorithm 4, identity metric, unit weights):
    eigenvalues of S^T S equal the squared singular values of S (LAPACK svd);
    W^T W = I (Eq. podOrth with Theta = I); w is the smallest index whose energy fraction
    reaches the criterion; Eckart-Young: sum_i ||s_i - W W^T s_i||^2 = sum_{k>w} sigma_k^2;
    range(W) equals the span of the leading left singular vectors."""
    S, _ = _snapshots()
    energy = 0.9999
    W, w, sig2 = orc.pod_evd(S, energy, 40)
    U, sv, _ = np.linalg.svd(S, full_matrices=False)
    e_sig = np.max(np.abs(sig2 - sv ** 2)) / sv[0] ** 2
    frac = np.cumsum(sv ** 2) / np.sum(sv ** 2)
    w_ref = int(np.argmax(frac >= energy)) + 1
    e_orth = np.max(np.abs(W.T @ W - np.eye(w))) if w else 0.0
    resid = S - W @ (W.T @ S)
    ey = abs(np.sum(resid ** 2) - np.sum(sv[w:] ** 2)) / np.sum(sv ** 2)
    cosines = np.linalg.svd(U[:, :w].T @ W, compute_uv=False) if w else np.ones(1)
    ok = e_sig < 1e-13 and w == w_ref and e_orth < 1e-10 and ey < 1e-12 and cosines.min() > 1 - 1e-10
    return ok, f"pod sig2 err {e_sig:.1e} w={w} ref={w_ref} orth {e_orth:.1e} EY {ey:.1e} cos {cosines.min():.12f}"


def pin_pod_nested(orc):
    """Nesting (Eq. podordering): the first w' columns do not depend on the cap w_max >= w'."""
    S, _ = _snapshots(seed=4)
    W8, w8, _ = orc.pod_evd(S, 1.0, 8)
    W3, w3, _ = orc.pod_evd(S, 1.0, 3)
    e = np.max(np.abs(W8[:, :w3] - W3))
    return w3 == 3 and w8 == 8 and e < 1e-12, f"nesting w3={w3} w8={w8} err {e:.1e}"


def pin_stage_one_exact(orc):
    """If x* lies in range(W), the stage-one Galerkin solve (Algorithm 2) returns x*
    (Section 4.1; the A-orthogonal projection of x* onto a space containing it is x*),
    and the full solve needs zero Algorithm-1 iterations."""
    A = small_diffusion(10, seed=1)
    D = A.todense()
    rng = np.random.default_rng(7)
    xs = rng.normal(size=A.n)
    b = D @ xs
    W = orth_basis(np.stack([xs, rng.normal(size=A.n), rng.normal(size=A.n)]))
    what, R, st = orc.stage_one(A.arrays(), b, W)
    x1 = W @ what
    e = np.linalg.norm(x1 - xs) / np.linalg.norm(xs)
    x, info, _, _ = orc.solve_system(A.arrays(), b, W, 1e-10)
    return st == 0 and e < 1e-12 and info["iters"] == 0, f"stage one exact err {e:.1e} iters {info['iters']}"


def pin_stage_one_galerkin(orc):
    """Galerkin orthogonality (Eq. equivalenceResidualOrth): W^T (b - A W what) = 0, and
    the stage-one iterate is the A-orthogonal projection: equals the dense least-squares
    solution of min ||A^{1/2}(x* - W y)||."""
    A = small_diffusion(9, seed=2)
    D = A.todense()
    rng = np.random.default_rng(9)
    b = rng.normal(size=A.n)
    W = orth_basis(rng.normal(size=(5, A.n)))
    what, R, st = orc.stage_one(A.arrays(), b, W)
    r = b - D @ (W @ what)
    e1 = np.max(np.abs(W.T @ r)) / np.linalg.norm(b)
    xs = np.linalg.solve(D, b)
    L = np.linalg.cholesky(D)
    y_ref = np.linalg.lstsq(L.T @ W, L.T @ xs, rcond=None)[0]
    e2 = np.max(np.abs(what - y_ref)) / np.max(np.abs(y_ref))
    return st == 0 and e1 < 1e-13 and e2 < 1e-10, f"galerkin orth {e1:.1e} projection {e2:.1e}"


def pin_empty_basis_is_pcg(orc):
    """Algorithm 1 with an empty augmenting basis is plain PCG: bitwise equal iterate and
    the same iteration count as the separately written PCG."""
    A = small_diffusion(12, seed=3)
    b = np.random.default_rng(4).normal(size=A.n)
    tol = 1e-9 * np.linalg.norm(b)
    x1, info, _, _ = orc.aug_pcg(A.arrays(), b, None, None, None, tol)
    x2, k2, st2 = orc.pcg(A.arrays(), b, None, tol)
    same = np.array_equal(x1, x2)
    return same and info["iters"] == k2 and info["status"] == "ok", \
        f"aug(W=0) vs pcg bitwise {same}, iters {info['iters']} vs {k2}"


def _aug_problem(n_side=10, w=4, seed=5):
    A = small_diffusion(n_side, seed=seed)
    D = A.todense()
    rng = np.random.default_rng(seed + 100)
    xs = rng.normal(size=A.n)
    b = D @ xs
    # basis: POD-like vectors close to (but not containing) the solution
    W = orth_basis(np.stack([xs + 0.3 * rng.normal(size=A.n) for _ in range(w)]))
    return A, D, b, W


def pin_dense_agreement(orc):
    """Full solve at tol 1e-14 agrees with the dense direct solve in the A-norm."""
    A, D, b, W = _aug_problem()
    x, info, _, _ = orc.solve_system(A.arrays(), b, W, 1e-14)
    xs = np.linalg.solve(D, b)
    e = a_norm(D, x - xs) / a_norm(D, xs)
    return info["status"] == "ok" and e < 1e-12, f"dense agreement {e:.1e} status {info['status']} iters {info['iters']}"


def pin_a_orthogonality(orc):
    """Directions stay A-orthogonal to W (Eq. Ajorthogonality: W^T A P = 0) and to each
    other (P^T A P diagonal)."""
    A, D, b, W = _aug_problem(seed=6)
    x, info, P, g = orc.solve_system(A.arrays(), b, W, 1e-10, p_cap=400)
    k = info["iters"]
    P = P[:, :k]
    AP = D @ P
    pa = np.sqrt(np.einsum("ij,ij->j", P, AP))
    wa = np.sqrt(np.einsum("ij,ij->j", W, D @ W))
    e1 = np.max(np.abs(W.T @ AP) / np.outer(wa, pa)) if k else 0.0
    C = (P.T @ AP) / np.outer(pa, pa)
    off = C - np.diag(np.diag(C))
    # loss of orthogonality in finite precision grows with k; check the first 15
    e2 = np.max(np.abs(off[:15, :15])) if k else 0.0
    e3 = np.max(np.abs(np.diag(P.T @ AP) - g[:k]) / g[:k]) if k else 0.0
    return k > 5 and e1 < 1e-10 and e2 < 1e-8 and e3 < 1e-12, \
        f"W^T A p {e1:.1e}, p_i^T A p_k {e2:.1e}, gamma {e3:.1e} (k={k})"


def pin_optimality(orc):
    """After k iterations the iterate minimises the A-norm error over
    range(W) + span(p_0..p_{k-1}) (Eq. KrylovSolveAugment / Section 4.3's projection):
    it equals the dense Galerkin solution on B = [W, P]."""
    A, D, b, W = _aug_problem(n_side=12, seed=8)
    x, info, P, g = orc.solve_system(A.arrays(), b, W, 1e-4, p_cap=400)
    k = info["iters"]
    B = np.concatenate([W, P[:, :k]], axis=1)
    y = np.linalg.solve(B.T @ D @ B, B.T @ b)
    xg = B @ y
    e = a_norm(D, x - xg) / a_norm(D, xg)
    return k >= 3 and e < 1e-9, f"optimality err {e:.1e} (k={k})"


def pin_finite_termination(orc):
    """CG terminates in at most as many steps as the preconditioned operator has distinct
    eigenvalues. A symmetric circulant tridiagonal matrix of order 32 has a constant
    diagonal (Jacobi = scaling) and 17 distinct eigenvalues a + 2 b cos(2 pi k/32)."""
    n = 32
    C = 4.0 * np.eye(n) - np.eye(n, k=1) - np.eye(n, k=-1)
    C[0, -1] = C[-1, 0] = -1.0
    A = dense_to_csr(C)
    b = np.random.default_rng(1).normal(size=n)
    x, info, _, _ = orc.aug_pcg(A.arrays(), b, None, None, None, 1e-11 * np.linalg.norm(b))
    xs = np.linalg.solve(C, b)
    e = np.linalg.norm(x - xs) / np.linalg.norm(xs)
    return info["iters"] <= 17 and e < 1e-10, f"finite termination iters {info['iters']} <= 17, err {e:.1e}"


def pin_generator_2x2(orc=None):
    """The 2x2 five-point operator with unit coefficients, assembled by hand: each cell has
    two interior faces (conductance 1) and two Dirichlet faces (conductance 2)."""
    op = DiffusionOperator((2, 2))
    A = op.csr(np.ones(4)).todense()
    ref = np.array([[6, -1, -1, 0], [-1, 6, 0, -1], [-1, 0, 6, -1], [0, -1, -1, 6]], float)
    return np.array_equal(A, ref), "generator 2x2"


def pin_theta_grad_complex_step(orc):
    """dL/dtheta = -sum_j lambda_j^T (dA_j/dtheta) x_j against complex-step differentiation of
    the generator's assembly (h = 1e-30, exact to rounding) on a 3 x 2 x 2 grid with random
    theta, lambda, x."""
    op = DiffusionOperator((2, 2, 3))
    rng = np.random.default_rng(5)
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
    e = float(np.max(np.abs(g - ref)) / max(1.0, np.max(np.abs(ref))))
    return e <= 1e-13, f"theta gradient vs complex step: {e:.1e}"


def _three_stage_problem(n_side=10, y=10, w=3, seed=3):
    """A small diffusion system and an orthonormal augmenting basis Y of y vectors near the
    solution; the stage-one basis is its first w columns."""
    A = small_diffusion(n_side, seed=seed)
    D = A.todense()
    rng = np.random.default_rng(seed + 4)
    xs = rng.normal(size=A.n)
    b = D @ xs
    Y = orth_basis(np.stack([xs + 0.5 * rng.normal(size=A.n) for _ in range(y)]))
    return A, D, b, Y, w


def pin_stage_two_optimality(orc):
    """After k stage-two iterations (Section 4.2) the iterate W what + V2 alpha minimises the
    A-norm error over range(W) + Y K_k(H, rhat0): the Krylov space of the reduced operator
    Ahat = Y^T A Y deflated by the stage-one coordinates Phi = [I_w; 0],
    H = Ahat - Ahat Phi (Phi^T Ahat Phi)^{-1} Phi^T Ahat, from rhat0 = Y^T (b - A W what).
    The reference is a dense Galerkin solve on that space, built from explicit powers of
    the dense reduced matrix."""
    A, D, b, Y, w = _three_stage_problem()
    W = np.asfortranarray(Y[:, :w])
    what, R, st = orc.stage_one(A.arrays(), b, W)
    Ah = Y.T @ D @ Y
    Phi = np.eye(Y.shape[1])[:, :w]
    H = Ah - Ah @ Phi @ np.linalg.solve(Phi.T @ Ah @ Phi, Phi.T @ Ah)
    r0 = Y.T @ (b - D @ (W @ what))
    worst = 0.0
    for k in (1, 2, 3, 4):
        out = orc.stage_two(A.arrays(), b, Y, w, R, what, 0.0, k)
        x2 = W @ what + out["V2"] @ out["alpha"]
        K = [r0]
        for _ in range(k - 1):
            K.append(H @ K[-1])
        Q, _ = np.linalg.qr(np.concatenate([W, Y @ np.stack(K, axis=1)], axis=1))
        xg = Q @ np.linalg.solve(Q.T @ D @ Q, Q.T @ b)
        worst = max(worst, a_norm(D, x2 - xg) / a_norm(D, xg))
        if out["k2"] != k:
            return False, f"stage two stopped at {out['k2']} < {k}"
    return st == 0 and worst < 1e-11, f"stage-two optimality err {worst:.1e}"


def pin_stage_two_full(orc):
    """With no tolerance and y - w iterations stage two solves the reduced system exactly
    (augmented CG on a y-dimensional SPD system with w directions deflated): the result is
    the Galerkin solution over range(Y), Y (Y^T A Y)^{-1} Y^T b (dense LAPACK solve). Its
    basis satisfies Section 4.2's properties V2^T A W = 0 and V2^T A V2 = diag(T2)."""
    A, D, b, Y, w = _three_stage_problem(seed=9)
    W = np.asfortranarray(Y[:, :w])
    what, R, st = orc.stage_one(A.arrays(), b, W)
    y = Y.shape[1]
    out = orc.stage_two(A.arrays(), b, Y, w, R, what, 0.0, y - w)
    V2 = out["V2"]
    x2 = W @ what + V2 @ out["alpha"]
    xg = Y @ np.linalg.solve(Y.T @ D @ Y, Y.T @ b)
    e = a_norm(D, x2 - xg) / a_norm(D, xg)
    AV = D @ V2
    va = np.sqrt(np.einsum("ij,ij->j", V2, AV))
    wa = np.sqrt(np.einsum("ij,ij->j", W, D @ W))
    e1 = np.max(np.abs(W.T @ AV) / np.outer(wa, va))
    C = V2.T @ AV
    e2 = np.max(np.abs(C - np.diag(out["T2"])) / np.outer(va, va))
    ok = out["k2"] == y - w and e < 1e-11 and e1 < 1e-12 and e2 < 1e-11
    return ok, f"stage two full: Galerkin err {e:.1e}, V2^T A W {e1:.1e}, V2^T A V2 - T2 {e2:.1e}, k2={out['k2']}"


def pin_three_stage_optimality(orc):
    """Stage three (Section 4.3) started from the stage-two solution with augmenting basis
    [W, V2] and the block-diagonal factor blockdiag(R, sqrt(T2)): after k iterations the
    iterate is the A-orthogonal projection onto range(W) + range(V2) + range(P) (dense
    Galerkin on the explicit basis); at tol 1e-14 it agrees with the dense direct solve."""
    A, D, b, Y, w = _three_stage_problem(n_side=12, y=8, w=3, seed=11)
    tol, tol2 = 1e-4, 1e-2
    x, info, P, g = orc.solve_system3(A.arrays(), b, Y, w, tol, tol2, 64, p_cap=400)
    W = np.asfortranarray(Y[:, :w])
    what, R, _ = orc.stage_one(A.arrays(), b, W)
    out = orc.stage_two(A.arrays(), b, Y, w, R, what, tol2 * tol * np.linalg.norm(b), Y.shape[1] - w)
    k = info["iters"]
    B = np.concatenate([W, out["V2"], P[:, :k]], axis=1)
    xg = B @ np.linalg.solve(B.T @ D @ B, B.T @ b)
    e = a_norm(D, x - xg) / a_norm(D, xg)
    x2, info2, _, _ = orc.solve_system3(A.arrays(), b, Y, w, 1e-14, tol2, 64)
    xs = np.linalg.solve(D, b)
    e2 = a_norm(D, x2 - xs) / a_norm(D, xs)
    ok = (info["k2"] == out["k2"] and info["k2"] >= 1 and k >= 3 and info["refinements"] == 0
          and e < 1e-9 and info2["status"] == "ok" and e2 < 1e-12)
    return ok, (f"three-stage optimality err {e:.1e} (k2={info['k2']}, k={k}), "
                f"dense agreement {e2:.1e} ({info2['status']})")


def pin_three_stage_collapse(orc):
    """With Y = W (no room for stage two) the three-stage solve is the two-stage solve:
    Algorithm 3 with an empty stage-two basis. Bitwise equal solutions."""
    A, D, b, W = _aug_problem(seed=7)
    x1, i1, _, _ = orc.solve_system(A.arrays(), b, W, 1e-9)
    x3, i3, _, _ = orc.solve_system3(A.arrays(), b, W, W.shape[1], 1e-9, 1e-3, 64)
    ok = np.array_equal(x1, x3) and i3["k2"] == 0 and i1["iters"] == i3["iters"]
    return ok, f"collapse: bitwise {np.array_equal(x1, x3)}, k2={i3['k2']}, iters {i1['iters']}/{i3['iters']}"


def pin_stage_two_reorthogonalised(orc):
    """An ill-conditioned reduced system (cond(Y^T A Y) ~ 1e5: Y holds the 20 lowest and 20
    highest eigenvectors of a 24x24 diffusion operator with coefficients exp(N(0, 2^2)),
    perturbed) run to y - w stage-two iterations: the stage-two basis stays A-orthogonal
    (V2^T A V2 diagonal to 1e-10 in the A-normalised columns) and the result is the
    Galerkin solution over range(Y) (dense LAPACK solve) to 1e-10. Without the stage-two
    re-A-orthogonalisation the directions lose orthogonality completely here."""
    rng = np.random.default_rng(3)
    op = DiffusionOperator((24, 24))
    A = op.csr(np.exp(rng.normal(0, 2.0, op.n)))
    D = A.todense()
    _, V = np.linalg.eigh(D)
    b = D @ rng.normal(size=A.n)
    idx = np.concatenate([np.arange(20), np.arange(A.n - 20, A.n)])
    Y = orth_basis((V[:, idx] + 1e-3 * rng.normal(size=(A.n, 40))).T)
    w = 3
    W = np.asfortranarray(Y[:, :w])
    what, R, _ = orc.stage_one(A.arrays(), b, W)
    out = orc.stage_two(A.arrays(), b, Y, w, R, what, 0.0, 40 - w)
    V2 = out["V2"]
    C = V2.T @ D @ V2
    na = np.sqrt(np.diag(C))
    Cn = C / np.outer(na, na)
    off = float(np.max(np.abs(Cn - np.diag(np.diag(Cn)))))
    x2 = W @ what + V2 @ out["alpha"]
    xg = Y @ np.linalg.solve(Y.T @ D @ Y, Y.T @ b)
    e = a_norm(D, x2 - xg) / a_norm(D, xg)
    return off < 1e-10 and e < 1e-10, f"ill-conditioned stage two: V2 A-orthogonality {off:.1e}, Galerkin err {e:.1e}"


def pin_stage3_full_matches_direct(orc):
    """The stage-three option of Section 4.3.1 with exact inner solves (tol_in = 0) and an
    exact stage two (tol2 = 0) is Algorithm 1 augmented with all of Y and exact reduced
    solves, i.e. the two-stage solve with stage-one basis W = Y (dense Cholesky of
    Y^T A Y): same iterations (within 1) and solutions within 1e-11 in the A-norm. With a
    wider Y (y = 20) stage two stops on its tolerance before exhausting the reduced space,
    the inner solves take the remaining reduced directions, and the solve agrees with a
    dense solve at tol 1e-13."""
    A, D, b, Y, w = _three_stage_problem(n_side=12, y=8, w=3, seed=13)
    x1, i1, _, _ = orc.solve_system(A.arrays(), b, Y, 1e-10)
    x2, i2 = orc.solve_system3_it(A.arrays(), b, Y, w, 1e-10, 0.0, 0.0)
    e = a_norm(D, x1 - x2) / a_norm(D, x1)
    A3, D3, b3, Y3, w3 = _three_stage_problem(n_side=14, y=20, w=3, seed=13)
    x3, i3 = orc.solve_system3_it(A3.arrays(), b3, Y3, w3, 1e-13, 1e-2, 1e-12)
    xs = np.linalg.solve(D3, b3)
    e3 = a_norm(D3, x3 - xs) / a_norm(D3, xs)
    ok = (i2["status"] == "ok" and abs(i1["iters"] - i2["iters"]) <= 1 and e < 1e-11
          and i3["status"] == "ok" and e3 < 1e-11 and i3["k2"] < 20 - 3 and i3["inner"] >= 1)
    return ok, (f"it stage three vs W = Y: err {e:.1e}, iters {i1['iters']}/{i2['iters']}; inner-driven run: "
                f"dense agreement {e3:.1e}, k2 {i3['k2']}, inner {i3['inner']}")


def pin_jacobi_svd_numpy(orc):
    """One-sided Jacobi SVD against LAPACK (numpy.linalg.svd) for a tall and a wide matrix
    (the wide one has s - q zero singular values), and V orthogonal."""
    rng = np.random.default_rng(21)
    worst = 0.0
    for q, s in ((9, 5), (3, 6)):
        B = rng.normal(size=(q, s)) * np.exp(rng.normal(size=s))
        sig, V, _ = orc.jacobi_svd(np.asfortranarray(B))
        ref = np.zeros(s)
        r = np.linalg.svd(B, compute_uv=False)
        ref[:len(r)] = r
        worst = max(worst, float(np.max(np.abs(sig - ref)) / ref[0]),
                    float(np.max(np.abs(V.T @ V - np.eye(s)))))
    return worst < 1e-13, f"Jacobi SVD vs LAPACK / orthogonality {worst:.1e}"


def pin_pod_output_metric(orc):
    """POD with the metric C^T C (Algorithm 5; q = 12 random U[0,1] functionals): sigma^2
    equal the squared singular values of C S (LAPACK); W is C^T C-orthonormal; the
    Eckart-Young identity in the C-seminorm, sum_i ||C s_i - CW (CW)^T C s_i||^2 =
    sum_{k>w} sigma_k^2; and with C = I the basis and spectrum are the identity-metric
    POD's (Algorithm 4), an independent route."""
    S, _ = _snapshots(n=300, s=8, seed=4)
    rng = np.random.default_rng(5)
    C = rng.uniform(0.0, 1.0, size=(12, 300))
    W, w, sig2 = orc.pod_svd(S, C, 0.999, 8)
    ref = np.linalg.svd(C @ S, compute_uv=False) ** 2
    e1 = float(np.max(np.abs(sig2[:len(ref)] - ref)) / ref[0])
    CW = C @ W
    e2 = float(np.max(np.abs(CW.T @ CW - np.eye(w))))
    CS = C @ S
    resid = CS - CW @ (CW.T @ CS)
    e3 = abs(float(np.sum(resid ** 2)) - float(np.sum(sig2[w:]))) / float(np.sum(sig2))
    We, we, sig2e = orc.pod_evd(S, 0.999, 8)
    Wi, wi, sig2i = orc.pod_svd(S, np.eye(300), 0.999, 8)
    e4 = float(np.max(np.abs(sig2i - sig2e)) / sig2e[0])
    cos = np.linalg.svd(Wi.T @ We, compute_uv=False) if wi == we else np.zeros(1)
    ok = 0 < w < 8 and e1 < 1e-12 and e2 < 1e-10 and e3 < 1e-12 and wi == we and e4 < 1e-12 and cos.min() > 1 - 1e-10
    return ok, (f"output POD: sigma^2 vs LAPACK {e1:.1e}, C-orthonormality {e2:.1e}, Eckart-Young {e3:.1e}, "
                f"C = I vs Algorithm 4: w {wi}/{we}, sigma^2 {e4:.1e}, cos {cos.min():.12f}")


def pin_pod_a_metric(orc):
    """POD with the metric A (Algorithm 4 with Theta = A): eigenvalues equal LAPACK's of
    S^T A S; W^T A W = I; the Eckart-Young identity in the A-norm,
    sum_i ||s_i - W W^T A s_i||_A^2 = sum_{k>w} lambda_k; and A = I reproduces the
    identity-metric POD."""
    S, _ = _snapshots(n=300, s=8, seed=6)
    A = small_diffusion(10, seed=2)
    n = A.n
    S = np.asfortranarray(S[:n])
    D = A.todense()
    W, w, lam = orc.pod_evd_metric(S, A.arrays(), 0.999, 8)
    ref = np.sort(np.linalg.eigvalsh(S.T @ D @ S))[::-1]
    e1 = float(np.max(np.abs(lam - ref)) / ref[0])
    e2 = float(np.max(np.abs(W.T @ D @ W - np.eye(w))))
    R = S - W @ (W.T @ (D @ S))
    e3 = abs(float(np.einsum("ij,ij->", R, D @ R)) - float(np.sum(lam[w:]))) / float(np.sum(lam))
    I = dense_to_csr(np.eye(n))
    Wi, wi, lami = orc.pod_evd_metric(S, I.arrays(), 0.999, 8)
    We, we, lame = orc.pod_evd(S, 0.999, 8)
    e4 = float(np.max(np.abs(lami - lame)) / lame[0])
    ok = 0 < w < 8 and e1 < 1e-12 and e2 < 1e-10 and e3 < 1e-10 and wi == we and e4 < 1e-13
    return ok, f"A-metric POD: lambda vs LAPACK {e1:.1e}, A-orthonormality {e2:.1e}, Eckart-Young {e3:.1e}, A = I {e4:.1e}"


def pin_a_metric_stage_two_one_step(orc):
    """With the POD metric A of the system being solved, the augmenting basis is
    A-orthonormal, Y^T A Y = I, so stage two (Algorithm 1 on the reduced system, M = I)
    converges in at most one iteration and reaches the Galerkin solution over range(Y)
    (the well-conditioned case the three-stage algorithm is designed for)."""
    A = small_diffusion(10, seed=8)
    D = A.todense()
    rng = np.random.default_rng(9)
    xs = rng.normal(size=A.n)
    b = D @ xs
    S = np.asfortranarray(np.stack([xs + 0.4 * rng.normal(size=A.n) for _ in range(8)], axis=1))
    Y, y, _ = orc.pod_evd_metric(S, A.arrays(), 2.0, 8)
    w = 3
    W = np.asfortranarray(Y[:, :w])
    what, R, _ = orc.stage_one(A.arrays(), b, W)
    out = orc.stage_two(A.arrays(), b, Y, w, R, what, 1e-12 * np.linalg.norm(b), y - w)
    x2 = W @ what + out["V2"] @ out["alpha"]
    xg = Y @ np.linalg.solve(Y.T @ D @ Y, Y.T @ b)
    e = a_norm(D, x2 - xg) / a_norm(D, xg)
    return y == 8 and out["k2"] <= 1 and e < 1e-10, f"A-metric stage two: k2 = {out['k2']}, Galerkin err {e:.1e}"


def _near_identity_reduced_problem(seed=5, y=40):
    """Y: y columns A_1-orthonormal (Cholesky of Z^T A_1 Z, Z random) for a 12x12 diffusion
    operator A_1; the system is A_2 = A_1 + diag(0.01 u), so cond(Y^T A_2 Y) is about 1.002:
    the well-conditioned reduced system Theorem 5 describes."""
    A1 = small_diffusion(12, seed=3)
    D1 = A1.todense()
    rng = np.random.default_rng(seed)
    Z = rng.normal(size=(A1.n, y))
    Lc = np.linalg.cholesky(Z.T @ D1 @ Z)
    Y = np.asfortranarray(Z @ np.linalg.inv(Lc).T)
    u = rng.uniform(0.0, 1.0, A1.n)
    rp, col, val = A1.arrays()
    rows = np.repeat(np.arange(A1.n), np.diff(rp))
    val2 = val + np.where(col == rows, 0.01 * u[rows], 0.0)
    b = rng.normal(size=A1.n)
    return (rp, col, val2), D1 + np.diag(0.01 * u), b, Y


def pin_stage_two_dependence_stop(orc):
    """Stage two with tolerance 0 on a reduced system with cond(Y^T A Y) = 1.002 reaches the
    rounding floor within a few iterations; with the dependence stop on (a direction whose
    A-norm squared after re-A-orthogonalisation is at most the part removed is not taken)
    it ends there, well before y - w iterations, at the Galerkin solution over range(Y)
    (dense LAPACK solve) to 1e-12, with and without deflated stage-one directions."""
    A, D, b, Y = _near_identity_reduced_problem()
    y = Y.shape[1]
    xg = Y @ np.linalg.solve(Y.T @ D @ Y, Y.T @ b)
    worst, ks = 0.0, []
    for w in (0, 3):
        W = np.asfortranarray(Y[:, :w])
        what, R, _ = orc.stage_one(A, b, W) if w else (None, None, 0)
        with orc.dependence_stop():
            out = orc.stage_two(A, b, Y, w, R, what, 0.0, y - w)
        x2 = out["V2"] @ out["alpha"] + (W @ what if w else 0.0)
        worst = max(worst, a_norm(D, x2 - xg) / a_norm(D, xg))
        ks.append(out["k2"])
    ok = worst < 1e-12 and all(0 < k < y // 2 for k in ks)
    return ok, f"dependence stop: Galerkin err {worst:.1e}, k2 {ks} of {y}"


def pin_sequence_window(orc, seq_cls=None):
    """The sequence driver's snapshot set (Section 3.1 with previous solutions as snapshots,
    the window of the last s_max): after p > s_max solves, the basis for the next system is
    the POD of exactly the last s_max recorded solutions. Checked against LAPACK's SVD of
    those solutions: the eigenvalues are their squared singular values, w is the smallest
    index whose energy fraction reaches the criterion, and range(W) is the span of the
    leading w left singular vectors. Each solution is the solution (residual <= tol), not the
    right-hand side. ``seq_cls`` lets a test substitute a driver with a planted mistake."""
    from oracle import OracleSequence
    cls = seq_cls or OracleSequence
    A = small_diffusion(8, seed=6)
    D = A.todense()
    n, s_max, p, energy = A.n, 4, 7, 0.999
    rng = np.random.default_rng(21)
    c = rng.normal(size=n)
    seq = cls(n, s_max=s_max, w_max=6, energy=energy, oracle=orc)
    xs = []
    for j in range(p):
        b = D @ (c + 0.05 * rng.normal(size=n))   # solutions share one dominant direction
        x, info = seq.solve(A.arrays(), b, 1e-12)
        if np.linalg.norm(b - D @ x) > 1e-11 * np.linalg.norm(b):
            return False, f"system {j}: the recorded iterate is not the solution"
        xs.append(x)
    W, w, sig2 = seq.basis()
    S = np.stack(xs[-s_max:], axis=1)
    U, sv, _ = np.linalg.svd(S, full_matrices=False)
    frac = np.cumsum(sv ** 2) / np.sum(sv ** 2)
    w_ref = int(np.argmax(frac >= energy)) + 1
    if len(sig2) != s_max or w != w_ref or not 1 <= w < s_max:
        return False, f"window: {len(sig2)} eigenvalues (want {s_max}), w={w} (want {w_ref})"
    e_sig = np.max(np.abs(np.asarray(sig2) - sv ** 2)) / sv[0] ** 2
    cos = np.linalg.svd(U[:, :w].T @ W, compute_uv=False)
    ok = e_sig < 1e-12 and cos.min() > 1 - 1e-10
    return ok, f"window sig2 err {e_sig:.1e} w={w} cos {cos.min():.12f}"


ALL_PINS = [pin_spmv_dense, pin_gram_spmm_dense, pin_cholesky_numpy, pin_jacobi_closed_form, pin_jacobi_vs_eigh,
            pin_pod_svd, pin_pod_nested, pin_stage_one_exact, pin_stage_one_galerkin,
            pin_empty_basis_is_pcg, pin_dense_agreement, pin_a_orthogonality, pin_optimality,
            pin_finite_termination, pin_theta_grad_complex_step, pin_stage_two_optimality,
            pin_stage_two_full, pin_three_stage_optimality, pin_three_stage_collapse,
            pin_stage_two_reorthogonalised, pin_stage3_full_matches_direct, pin_jacobi_svd_numpy,
            pin_pod_output_metric, pin_pod_a_metric, pin_a_metric_stage_two_one_step,
            pin_stage_two_dependence_stop, pin_sequence_window]
