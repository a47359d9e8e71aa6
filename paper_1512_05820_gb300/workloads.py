"""Seeded synthetic workloads: sequences of sparse SPD systems A_j x_j = b_j.

This module only generates inputs (CSR matrices and right-hand sides). It holds none of
the solver's arithmetic and is shared by the GPU path, the oracle-based tests and the
benchmark. The paper's systems (Sierra/SolidMechanics exports, Section 5.1) are not
available; these stand in for them with the shapes of the benchmark configurations:

* ``diffusion2d_drift``   64x64 5-point variable-coefficient diffusion, 10 systems,
  A_j = A_0 + diag(0.01 j u), drifting Gaussian-bump sources (w <= 8, FP64).
* ``diffusion3d_moving``  128^3 7-point diffusion, 50 systems, log-coefficients
  perturbed by 0.5% per step, a heat source moving on a circle (s <= 40, w <= 32).
* ``diffusion3d_theta``   96^3 7-point diffusion parameterised by per-cell
  log-coefficients theta (the differentiation workload), 20 systems.

Discretisation (cell-centred finite volumes, unit spacing): the conductance of the face
between cells a and b is the harmonic mean 2 k_a k_b / (k_a + k_b); every boundary face
is a homogeneous Dirichlet face at half-cell distance with conductance 2 k_a. Row a of A
holds the sum of its face conductances on the diagonal and -k_f for each neighbour.
Cells are numbered x fastest, then y, then z; CSR columns are sorted within each row.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np


@dataclass
class CSR:
    """CSR matrix with 32-bit indices (row_ptr[n+1], col[nnz]) and float64 values."""
    n: int
    row_ptr: np.ndarray
    col: np.ndarray
    val: np.ndarray

    @property
    def nnz(self) -> int:
        return int(self.row_ptr[-1])

    def arrays(self):
        return self.row_ptr, self.col, self.val

    def todense(self) -> np.ndarray:
        D = np.zeros((self.n, self.n))
        rows = np.repeat(np.arange(self.n), np.diff(self.row_ptr))
        np.add.at(D, (rows, self.col), self.val)
        return D


def _hm(a, b):
    return 2.0 * a * b / (a + b)


class DiffusionOperator:
    """Sparsity pattern and value assembly of the 2D 5-point / 3D 7-point operator.

    ``shape`` is (my, mx) or (mz, my, mx). The pattern is built once; ``values(k, d)``
    assembles the CSR values for cell coefficients ``k`` (length n) plus an optional extra
    diagonal ``d``.
    """

    def __init__(self, shape):
        shape = tuple(int(s) for s in shape)
        if len(shape) == 2:
            shape = (1,) + shape
        self.shape3 = shape
        self.dim = 2 if shape[0] == 1 else 3
        mz, my, mx = shape
        n = mx * my * mz
        self.n = n
        iz, iy, ix = np.meshgrid(np.arange(mz), np.arange(my), np.arange(mx), indexing="ij")
        ix, iy, iz = ix.ravel(), iy.ravel(), iz.ravel()
        i = np.arange(n, dtype=np.int64)
        # slots in ascending column order: z-1, y-1, x-1, self, x+1, y+1, z+1
        steps = [mx * my, mx, 1]
        valid = [iz > 0, iy > 0, ix > 0, np.ones(n, bool), ix < mx - 1, iy < my - 1, iz < mz - 1]
        cols = [i - steps[0], i - steps[1], i - steps[2], i, i + steps[2], i + steps[1], i + steps[0]]
        if self.dim == 2:
            keep = [1, 2, 3, 4, 5]
            valid = [valid[s] for s in keep]
            cols = [cols[s] for s in keep]
        self.slots = len(valid)
        self.mask = np.stack(valid, axis=1)
        colmat = np.stack(cols, axis=1)
        self.col = colmat[self.mask].astype(np.int32)
        counts = self.mask.sum(axis=1)
        self.row_ptr = np.zeros(n + 1, dtype=np.int32)
        np.cumsum(counts, out=self.row_ptr[1:])
        self.nnz = int(self.row_ptr[-1])

    def face_conductances(self, k):
        """Interior face conductances per axis: (fx, fy, fz) on the face grids."""
        K = np.asarray(k).reshape(self.shape3)
        fx = _hm(K[:, :, :-1], K[:, :, 1:])
        fy = _hm(K[:, :-1, :], K[:, 1:, :])
        fz = _hm(K[:-1, :, :], K[1:, :, :])
        return fx, fy, fz

    def values(self, k, extra_diag=None) -> np.ndarray:
        """CSR values; ``k`` may be complex (complex-step differentiation in tests)."""
        K = np.asarray(k)
        K = K.astype(np.complex128 if np.iscomplexobj(K) else np.float64).reshape(self.shape3)
        fx, fy, fz = self.face_conductances(K)
        mz, my, mx = self.shape3
        diag = np.zeros(self.shape3, dtype=K.dtype)
        diag[:, :, :-1] += fx
        diag[:, :, 1:] += fx
        diag[:, :, 0] += 2.0 * K[:, :, 0]
        diag[:, :, -1] += 2.0 * K[:, :, -1]
        diag[:, :-1, :] += fy
        diag[:, 1:, :] += fy
        diag[:, 0, :] += 2.0 * K[:, 0, :]
        diag[:, -1, :] += 2.0 * K[:, -1, :]
        if self.dim == 3:
            diag[:-1, :, :] += fz
            diag[1:, :, :] += fz
            diag[0, :, :] += 2.0 * K[0, :, :]
            diag[-1, :, :] += 2.0 * K[-1, :, :]
        d = diag.ravel()
        if extra_diag is not None:
            d = d + np.asarray(extra_diag, dtype=np.float64)
        n = self.n
        V = np.zeros((n, 7), dtype=K.dtype)

        def put(slot, arr, sl):
            tmp = np.zeros(self.shape3, dtype=K.dtype)
            tmp[sl] = -arr
            V[:, slot] = tmp.ravel()

        # each interior face couples its two cells; place -k_f in both rows
        put(0, fz, (slice(1, None), slice(None), slice(None)))   # z-1 neighbour
        put(1, fy, (slice(None), slice(1, None), slice(None)))   # y-1
        put(2, fx, (slice(None), slice(None), slice(1, None)))   # x-1
        V[:, 3] = d
        put(4, fx, (slice(None), slice(None), slice(None, -1)))  # x+1
        put(5, fy, (slice(None), slice(None, -1), slice(None)))  # y+1
        put(6, fz, (slice(None, -1), slice(None), slice(None)))  # z+1
        if self.dim == 2:
            V = V[:, 1:6]
        return V[self.mask]

    def csr(self, k, extra_diag=None) -> CSR:
        return CSR(self.n, self.row_ptr, self.col, self.values(k, extra_diag))

    def gaussian(self, center, sigma, amplitude=1.0) -> np.ndarray:
        """Gaussian bump sampled at cell indices; ``center`` is (x, y[, z]) in cell units."""
        mz, my, mx = self.shape3
        iz, iy, ix = np.meshgrid(np.arange(mz), np.arange(my), np.arange(mx), indexing="ij")
        c = list(center) + [0.0] * (3 - len(center))
        r2 = (ix - c[0]) ** 2 + (iy - c[1]) ** 2 + ((iz - c[2]) ** 2 if self.dim == 3 else 0.0)
        return (amplitude * np.exp(-r2 / (2.0 * sigma * sigma))).ravel()


@dataclass
class Sequence:
    """A sequence of systems sharing one sparsity pattern, plus its solver settings."""
    name: str
    op: DiffusionOperator
    p: int
    tol: float
    s_max: int
    w_max: int
    energy: float
    seed: int
    recipe: dict = field(default_factory=dict)
    _gen: object = None

    @property
    def n(self):
        return self.op.n

    @property
    def nnz(self):
        return self.op.nnz

    @property
    def row_ptr(self):
        return self.op.row_ptr

    @property
    def col(self):
        return self.op.col

    def systems(self):
        """Yield (j, val_j, b_j) for j = 1..p in order (values float64, length nnz / n)."""
        return self._gen(self)

    def all_systems(self):
        return list(self.systems())


def _drift2d_gen(seq: Sequence):
    rng = np.random.default_rng(seq.seed)
    n = seq.n
    theta = rng.normal(0.0, seq.recipe["coef_sigma"], n)
    u = rng.uniform(0.0, 1.0, n)
    k = np.exp(theta)
    my, mx = seq.op.shape3[1], seq.op.shape3[2]
    for j in range(1, seq.p + 1):
        val = seq.op.values(k, 0.01 * j * u)
        cx = seq.recipe["x0"] + seq.recipe["drift"] * j
        b = seq.op.gaussian((cx, my / 2.0), seq.recipe["sigma"])
        yield j, val, b


def diffusion2d_drift(m: int = 64, p: int = 10, seed: int = 1234, w_max: int = 8,
                      s_max: int = 40, energy: float = 0.9999, tol: float = 1e-8) -> Sequence:
    """2D 5-point diffusion on an m x m grid; lognormal(0, 0.5) cell coefficients,
    A_j = A_0 + diag(0.01 j u) with u ~ U(0, 1), Gaussian bump (amplitude 1, sigma 3 cells)
    centred at (m/4 + j, m/2), drifting one cell per system.

    Random draws, in order, from ``numpy.random.default_rng(seed)``: theta ~ N(0, 0.5^2)
    (n values), then u ~ U(0, 1) (n values)."""
    op = DiffusionOperator((m, m))
    recipe = {"coef_sigma": 0.5, "x0": m / 4.0, "drift": 1.0, "sigma": 3.0 * m / 64.0 if m < 64 else 3.0}
    return Sequence("diffusion2d_drift", op, p, tol, s_max, w_max, energy, seed, recipe, _drift2d_gen)


def _moving3d_gen(seq: Sequence):
    rng = np.random.default_rng(seq.seed)
    n = seq.n
    r = seq.recipe
    theta = rng.normal(0.0, r["coef_sigma"], n)
    m = seq.op.shape3[2]
    for j in range(1, seq.p + 1):
        if j > 1:
            xi = rng.normal(0.0, 1.0, n)
            theta = theta + np.log1p(r["perturb"] * xi)
        val = seq.op.values(np.exp(theta))
        ang = 2.0 * np.pi * j / r["period"]
        c = (m / 2.0 + m / 4.0 * np.cos(ang), m / 2.0 + m / 4.0 * np.sin(ang), m / 2.0)
        b = seq.op.gaussian(c, r["sigma"])
        yield j, val, b


def diffusion3d_moving(m: int = 128, p: int = 50, seed: int = 1235, w_max: int = 32,
                       s_max: int = 40, energy: float = 0.9999, tol: float = 1e-8,
                       period: float | None = None, coef_sigma: float = 1.0) -> Sequence:
    """3D 7-point diffusion on an m^3 grid; lognormal(0, 1) coefficients perturbed by
    0.5% per system (theta <- theta + log(1 + 0.005 xi), xi ~ N(0, 1) per cell); a
    Gaussian heat source (sigma 4 cells at m = 128, scaled with m) moving on the circle
    (m/2 + m/4 cos(2 pi j/P), m/2 + m/4 sin(2 pi j/P), m/2) with P = 50.

    Random draws, in order: theta_1 ~ N(0, 1) (n values); then for each j >= 2 one
    xi ~ N(0, 1) draw of n values."""
    op = DiffusionOperator((m, m, m))
    recipe = {"coef_sigma": coef_sigma, "perturb": 0.005, "period": float(period or 50),
              "sigma": max(1.5, 4.0 * m / 128.0)}
    return Sequence("diffusion3d_moving", op, p, tol, s_max, w_max, energy, seed, recipe, _moving3d_gen)


def _theta3d_gen(seq: Sequence):
    r = seq.recipe
    theta, u = r["theta"], r["u"]
    m = seq.op.shape3[2]
    k = np.exp(theta)
    for j in range(1, seq.p + 1):
        val = seq.op.values(k, 0.01 * j * u)
        ang = 2.0 * np.pi * j / r["period"]
        c = (m / 2.0 + m / 4.0 * np.cos(ang), m / 2.0 + m / 4.0 * np.sin(ang), m / 2.0)
        b = seq.op.gaussian(c, r["sigma"])
        yield j, val, b


def diffusion3d_theta(m: int = 96, p: int = 20, seed: int = 1238, w_max: int = 32,
                      s_max: int = 40, energy: float = 0.9999, tol: float = 1e-8,
                      theta=None) -> Sequence:
    """3D 7-point diffusion parameterised by per-cell log-coefficients theta
    (k = exp(theta)), A_j(theta) = A(theta) + diag(0.01 j u), sources as in
    ``diffusion3d_moving`` with period 50; loss L = sum_j c^T x_j with c ~ N(0, 1).

    Random draws, in order: theta ~ N(0, 0.5^2) (n values), u ~ U(0, 1) (n values),
    c ~ N(0, 1) (n values). ``theta`` may be given to override the drawn one."""
    op = DiffusionOperator((m, m, m))
    rng = np.random.default_rng(seed)
    th = rng.normal(0.0, 0.5, op.n)
    u = rng.uniform(0.0, 1.0, op.n)
    c = rng.normal(0.0, 1.0, op.n)
    recipe = {"theta": th if theta is None else np.asarray(theta, dtype=np.float64), "u": u, "c": c,
              "period": 50.0, "sigma": max(1.5, 4.0 * m / 128.0)}
    return Sequence("diffusion3d_theta", op, p, tol, s_max, w_max, energy, seed, recipe, _theta3d_gen)


def batch_sequences(nseq: int = 256, p: int = 8, n_min: int = 2000, n_max: int = 260000, seed: int = 1237,
                    w_range=(4, 24), s_max: int = 8, energy: float = 0.9999, tol: float = 1e-8) -> list[Sequence]:
    """Many independent sequences of uneven sizes (the batched workload): n drawn
    log-uniformly in [n_min, n_max]; with probability 1/2 a 2D five-point sequence on an
    m x m grid (m = round(sqrt n)) evolving like ``diffusion2d_drift``, else a 3D seven-point
    sequence on m^3 (m = round(cbrt n)) evolving like ``diffusion3d_moving``; coefficients
    lognormal(0, 0.5) in both; w_max drawn uniformly in w_range (inclusive).

    Random draws from ``numpy.random.default_rng(seed)``, per sequence in order: log n
    (uniform), the 2D/3D coin, w_max, and the sequence's own seed."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(nseq):
        n_t = float(np.exp(rng.uniform(np.log(n_min), np.log(n_max))))
        is3d = rng.random() >= 0.5
        w_i = int(rng.integers(w_range[0], w_range[1] + 1))
        s_i = int(rng.integers(0, 2**31 - 1))
        if is3d:
            m = max(3, int(round(n_t ** (1.0 / 3.0))))
            out.append(diffusion3d_moving(m=m, p=p, seed=s_i, w_max=w_i, s_max=s_max, energy=energy, tol=tol,
                                          period=p, coef_sigma=0.5))
        else:
            m = max(3, int(round(np.sqrt(n_t))))
            out.append(diffusion2d_drift(m=m, p=p, seed=s_i, w_max=w_i, s_max=s_max, energy=energy, tol=tol))
    return out


def hex8_stiffness(E: float = 1.0, nu: float = 0.3, h: float = 1.0) -> np.ndarray:
    """24x24 stiffness of a trilinear hexahedron of edge h (linear isotropic elasticity,
    2x2x2 Gauss quadrature). Local node a = ax + 2 ay + 4 az (ax, ay, az in {0, 1}); dof
    3a + c for displacement component c."""
    lam = E * nu / ((1 + nu) * (1 - 2 * nu))
    mu = E / (2 * (1 + nu))
    D = np.zeros((6, 6))
    D[:3, :3] = lam
    D[np.arange(3), np.arange(3)] = lam + 2 * mu
    D[3, 3] = D[4, 4] = D[5, 5] = mu
    corners = np.array([[(a >> 0) & 1, (a >> 1) & 1, (a >> 2) & 1] for a in range(8)], float) * 2 - 1
    g = 1.0 / np.sqrt(3.0)
    K = np.zeros((24, 24))
    for gz in (-g, g):
        for gy in (-g, g):
            for gx in (-g, g):
                xi = np.array([gx, gy, gz])
                dN = np.zeros((8, 3))   # dN/dxi
                for a in range(8):
                    ca = corners[a]
                    f = 1 + ca * xi
                    dN[a, 0] = ca[0] * f[1] * f[2] / 8
                    dN[a, 1] = f[0] * ca[1] * f[2] / 8
                    dN[a, 2] = f[0] * f[1] * ca[2] / 8
                dNx = dN * (2.0 / h)           # x = h (xi + 1)/2
                B = np.zeros((6, 24))
                for a in range(8):
                    bx, by, bz = dNx[a]
                    B[0, 3 * a] = bx
                    B[1, 3 * a + 1] = by
                    B[2, 3 * a + 2] = bz
                    B[3, 3 * a] = by
                    B[3, 3 * a + 1] = bx
                    B[4, 3 * a + 1] = bz
                    B[4, 3 * a + 2] = by
                    B[5, 3 * a] = bz
                    B[5, 3 * a + 2] = bx
                K += B.T @ D @ B * (h / 2) ** 3
    return K


class ElasticityOperator:
    """3D linear elasticity on a block of ex x ey x ez unit trilinear hexahedra, three
    displacement dofs per node, the nodes of the face x = 0 clamped (their dofs removed).
    Free node (ix >= 1, iy, iz) has index (ix - 1) + (nx - 1)(iy + ny iz); dof 3 node + c.
    CSR rows list the up to 27 neighbouring free nodes in increasing node order, each with
    its three components. ``values(E)`` assembles for per-element Young's moduli."""

    def __init__(self, ex: int, ey: int, ez: int, nu: float = 0.3):
        self.ex, self.ey, self.ez = ex, ey, ez
        self.nx, self.ny, self.nz = ex + 1, ey + 1, ez + 1
        nx, ny, nz = self.nx, self.ny, self.nz
        self.nfree = (nx - 1) * ny * nz
        self.n = 3 * self.nfree
        self.Ke = hex8_stiffness(1.0, nu)
        iz, iy, ix = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(1, nx), indexing="ij")
        self.fix, self.fiy, self.fiz = ix.ravel(), iy.ravel(), iz.ravel()
        offs = [(dz, dy, dx) for dz in (-1, 0, 1) for dy in (-1, 0, 1) for dx in (-1, 0, 1)]
        self.offs = offs
        valid = np.zeros((self.nfree, 27), bool)
        nbr = np.zeros((self.nfree, 27), np.int64)
        for s_, (dz, dy, dx) in enumerate(offs):
            jx, jy, jz = self.fix + dx, self.fiy + dy, self.fiz + dz
            ok = (jx >= 1) & (jx < nx) & (jy >= 0) & (jy < ny) & (jz >= 0) & (jz < nz)
            valid[:, s_] = ok
            nbr[:, s_] = np.where(ok, (jx - 1) + (nx - 1) * (jy + ny * jz), 0)
        self.slot_valid = valid
        mask = np.repeat(np.repeat(valid, 3, axis=1)[:, None, :], 3, axis=1).reshape(self.n, 81)
        self.mask = mask
        cols = (3 * np.repeat(nbr, 3, axis=1) + np.tile(np.arange(3), 27)[None, :])
        cols = np.repeat(cols[:, None, :], 3, axis=1).reshape(self.n, 81)
        self.col = cols[mask].astype(np.int32)
        counts = mask.sum(axis=1)
        self.row_ptr = np.zeros(self.n + 1, dtype=np.int32)
        np.cumsum(counts, out=self.row_ptr[1:])
        self.nnz = int(self.row_ptr[-1])
        ez_, ey_, ex_ = np.meshgrid(np.arange(ez), np.arange(ey), np.arange(ex), indexing="ij")
        self.eix, self.eiy, self.eiz = ex_.ravel(), ey_.ravel(), ez_.ravel()

    def element_centres(self):
        return np.stack([self.eix + 0.5, self.eiy + 0.5, self.eiz + 0.5], axis=1)

    def values(self, E) -> np.ndarray:
        E = np.asarray(E, dtype=np.float64)
        nx, ny = self.nx, self.ny
        V = np.zeros((self.nfree, 3, 81))
        for a in range(8):
            ax, ay, az = a & 1, (a >> 1) & 1, (a >> 2) & 1
            nxa, nya, nza = self.eix + ax, self.eiy + ay, self.eiz + az
            fa = nxa >= 1
            rows = (nxa - 1) + (nx - 1) * (nya + ny * nza)
            for b in range(8):
                bx, by, bz = b & 1, (b >> 1) & 1, (b >> 2) & 1
                fb = self.eix + bx >= 1
                ok = fa & fb
                s_ = 9 * (bz - az + 1) + 3 * (by - ay + 1) + (bx - ax + 1)
                r_ok, e_ok = rows[ok], E[ok]
                blk = self.Ke[3 * a:3 * a + 3, 3 * b:3 * b + 3]
                V[r_ok, :, 3 * s_:3 * s_ + 3] += e_ok[:, None, None] * blk[None, :, :]
        return V.reshape(self.n, 81)[self.mask]

    def csr(self, E) -> CSR:
        return CSR(self.n, self.row_ptr, self.col, self.values(E))

    def end_traction(self, phi: float) -> np.ndarray:
        """Unit traction (0, cos phi, sin phi) on the face x = L, lumped to its nodes with
        the bilinear face weights (corner 1/4, edge 1/2, interior 1)."""
        b = np.zeros((self.nfree, 3))
        on = self.fix == self.nx - 1
        wy = np.where((self.fiy == 0) | (self.fiy == self.ny - 1), 0.5, 1.0)
        wz = np.where((self.fiz == 0) | (self.fiz == self.nz - 1), 0.5, 1.0)
        wgt = np.where(on, wy * wz, 0.0)
        b[:, 1] = wgt * np.cos(phi)
        b[:, 2] = wgt * np.sin(phi)
        return b.ravel()


def _elasticity_gen(seq: Sequence):
    r = seq.recipe
    op = seq.op
    rng = np.random.default_rng(seq.seed)
    E0 = np.exp(rng.normal(0.0, r["e_sigma"], op.ex * op.ey * op.ez))
    xc = op.element_centres()
    for j in range(1, seq.p + 1):
        c = np.array([op.ex * j / (seq.p + 1), op.ey / 2.0, op.ez / 2.0])
        d = r["damage"] * np.exp(-np.sum((xc - c) ** 2, axis=1) / (2.0 * r["damage_width"] ** 2))
        val = op.values(E0 * (1.0 - d))
        b = op.end_traction(2.0 * np.pi * j / seq.p)
        yield j, val, b


def elasticity_cantilever(e: int = 64, p: int = 30, seed: int = 1236, w_max: int = 48, s_max: int = 40,
                          energy: float = 0.9999, tol: float = 1e-8) -> Sequence:
    """3D cantilever of e^3 unit trilinear hexahedra, clamped at x = 0, Poisson ratio 0.3;
    Young's modulus lognormal(0, 0.3) per element scaled by (1 - d_j), d_j = 0.3
    exp(-|x_e - c_j|^2/(2 8^2)) a damage spot moving along the beam (c_j = (e j/(p+1),
    e/2, e/2)); load: a unit end traction rotating about the beam axis,
    phi_j = 2 pi j/p. Draws: E0 ~ lognormal(0, 0.3) (e^3 values)."""
    op = ElasticityOperator(e, e, e)
    recipe = {"e_sigma": 0.3, "damage": 0.3, "damage_width": 8.0 * e / 64.0}
    return Sequence("elasticity_cantilever", op, p, tol, s_max, w_max, energy, seed, recipe, _elasticity_gen)


def random_spd_csr(n: int, density: float, seed: int, shift: float = 1.0, empty_rows: int = 0) -> CSR:
    """Random sparse SPD matrix with ragged row lengths (symmetric pattern, strictly
    diagonally dominant): used for edge-case tests (heavy-tailed rows, ``empty_rows``
    rows holding only their diagonal)."""
    rng = np.random.default_rng(seed)
    rows, cols, vals = [], [], []
    lengths = np.minimum(n - 1, rng.zipf(1.6, n) * max(1, int(density * n)) // 4)
    lengths[:empty_rows] = 0
    for i in range(n):
        if lengths[i] == 0:
            continue
        js = rng.choice(n, size=int(lengths[i]), replace=False)
        js = js[js != i]
        if empty_rows:
            js = js[js >= empty_rows]
        v = -rng.uniform(0.1, 1.0, len(js))
        rows += [i] * len(js) + list(js)
        cols += list(js) + [i] * len(js)
        vals += list(v) + list(v)
    rows = np.array(rows, dtype=np.int64)
    cols = np.array(cols, dtype=np.int64)
    vals = np.array(vals, dtype=np.float64)
    # merge duplicates
    key = rows * n + cols
    uk, inv = np.unique(key, return_inverse=True)
    acc = np.zeros(len(uk))
    np.add.at(acc, inv, vals)
    r_u, c_u = uk // n, uk % n
    diag = np.zeros(n)
    np.add.at(diag, r_u, np.abs(acc))
    diag = diag + shift + rng.uniform(0.0, 1.0, n)
    r_all = np.concatenate([r_u, np.arange(n)])
    c_all = np.concatenate([c_u, np.arange(n)])
    v_all = np.concatenate([acc, diag])
    order = np.lexsort((c_all, r_all))
    r_all, c_all, v_all = r_all[order], c_all[order], v_all[order]
    row_ptr = np.zeros(n + 1, dtype=np.int32)
    np.add.at(row_ptr, r_all + 1, 1)
    row_ptr = np.cumsum(row_ptr).astype(np.int32)
    return CSR(n, row_ptr, c_all.astype(np.int32), v_all)


def smooth_snapshots(op: DiffusionOperator, s: int, modes: int = 24, decay: float = 0.7,
                     seed: int = 1239) -> np.ndarray:
    """s smooth fields on the operator's grid, an (n, s) Fortran-ordered block: each column
    is sum_m decay^m g_mk f_m with separable sine modes
    f_m = sin(pi a_m (x+1/2)/mx) sin(pi b_m (y+1/2)/my) sin(pi c_m (z+1/2)/mz), wave numbers
    a_m, b_m, c_m ~ U{1..4} and g_mk ~ N(0, 1). The squared singular values fall roughly
    like decay^(2m), so an energy cut keeps a handful to a few tens of modes.

    Random draws, in order, from ``numpy.random.default_rng(seed)``: the wave numbers
    (modes x 3 integers), then g (modes x s values)."""
    rng = np.random.default_rng(seed)
    mz, my, mx = op.shape3
    waves = rng.integers(1, 5, size=(modes, 3))
    g = rng.normal(0.0, 1.0, size=(modes, s)) * (decay ** np.arange(modes))[:, None]
    F = np.empty((op.n, modes))
    for m, (a, b, c) in enumerate(waves):
        fx = np.sin(np.pi * a * (np.arange(mx) + 0.5) / mx)
        fy = np.sin(np.pi * b * (np.arange(my) + 0.5) / my)
        fz = np.sin(np.pi * c * (np.arange(mz) + 0.5) / mz) if op.dim == 3 else np.ones(1)
        F[:, m] = (fz[:, None, None] * fy[None, :, None] * fx[None, None, :]).ravel()
    return np.asfortranarray(F @ g)
