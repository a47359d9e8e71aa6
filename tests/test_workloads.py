"""The seeded input generators against independent constructions: the finite-volume
diffusion operator assembled cell by cell, the hexahedron stiffness against rigid-body
modes and the energy of a uniform strain, the assembled cantilever's symmetry, definiteness
and 3x3 block pattern, and the documented structure of the other generators."""
import numpy as np

from paper_1512_05820_gb300 import workloads as wl


def dense_fv(shape, k):
    """Cell-by-cell assembly: each interior face between cells a, b adds the harmonic mean
    2 k_a k_b/(k_a + k_b) to both diagonals and its negative to both off-diagonals; each
    boundary face of cell a adds 2 k_a to its diagonal."""
    mz, my, mx = shape
    n = mx * my * mz
    K = np.asarray(k).reshape(shape)
    D = np.zeros((n, n))
    idx = lambda z, y, x: x + mx * (y + my * z)
    for z in range(mz):
        for y in range(my):
            for x in range(mx):
                a = idx(z, y, x)
                for dz, dy, dx in ((1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0), (0, 0, 1), (0, 0, -1)):
                    if mz == 1 and dz != 0:
                        continue
                    zz, yy, xx = z + dz, y + dy, x + dx
                    if 0 <= zz < mz and 0 <= yy < my and 0 <= xx < mx:
                        b = idx(zz, yy, xx)
                        kf = 2 * K[z, y, x] * K[zz, yy, xx] / (K[z, y, x] + K[zz, yy, xx])
                        D[a, a] += kf
                        D[a, b] -= kf
                    else:
                        D[a, a] += 2 * K[z, y, x]
    return D


def test_diffusion_operator_matches_cell_assembly():
    rng = np.random.default_rng(0)
    for shape in ((3, 4, 5), (1, 6, 7)):
        op = wl.DiffusionOperator(shape if shape[0] > 1 else shape[1:])
        k = np.exp(rng.normal(size=op.n))
        A = op.csr(k)
        assert np.allclose(A.todense(), dense_fv(shape, k), rtol=1e-14, atol=0)
        for i in range(A.n):   # sorted columns, diagonal included
            cols = A.col[A.row_ptr[i]:A.row_ptr[i + 1]]
            assert np.all(np.diff(cols) > 0) and i in cols
        assert np.linalg.eigvalsh(A.todense()).min() > 0


def test_hex8_rigid_modes_and_uniform_strain():
    E, nu, h = 2.5, 0.3, 1.5
    K = wl.hex8_stiffness(E, nu, h)
    assert np.allclose(K, K.T, rtol=0, atol=1e-14 * np.abs(K).max())
    X = np.array([[(a >> 0) & 1, (a >> 1) & 1, (a >> 2) & 1] for a in range(8)], float) * h
    modes = []
    for c in range(3):   # translations
        u = np.zeros((8, 3))
        u[:, c] = 1.0
        modes.append(u.ravel())
    for w in np.eye(3):  # rotations u = w x X
        modes.append(np.cross(w, X).ravel())
    R = np.array(modes).T
    assert np.abs(K @ R).max() <= 1e-13 * np.abs(K).max()
    ev = np.linalg.eigvalsh(K)
    assert np.sum(ev < 1e-12 * ev.max()) == 6 and ev[6] > 1e-6 * ev.max()
    # a linear displacement with symmetric gradient G is reproduced exactly by the element
    # and integrated exactly by 2x2x2 Gauss: u^T K u = h^3 (lam tr(G)^2 + 2 mu G:G)
    rng = np.random.default_rng(1)
    G = rng.normal(size=(3, 3))
    G = 0.5 * (G + G.T)
    u = (X @ G.T).ravel()
    lam = E * nu / ((1 + nu) * (1 - 2 * nu))
    mu = E / (2 * (1 + nu))
    energy = h ** 3 * (lam * np.trace(G) ** 2 + 2 * mu * np.sum(G * G))
    assert abs(u @ K @ u - energy) <= 1e-12 * energy


def test_cantilever_assembly():
    op = wl.ElasticityOperator(3, 2, 2)
    rng = np.random.default_rng(2)
    E = np.exp(rng.normal(0, 0.3, op.ex * op.ey * op.ez))
    A = op.csr(E)
    D = A.todense()
    assert np.allclose(D, D.T, rtol=0, atol=1e-13 * np.abs(D).max())
    assert np.linalg.eigvalsh(D).min() > 0     # the clamped face removes the rigid modes
    for node in range(op.nfree):               # rows of a node share one pattern of whole 3x3 blocks
        rows = [A.col[A.row_ptr[3 * node + c]:A.row_ptr[3 * node + c + 1]] for c in range(3)]
        assert np.array_equal(rows[0], rows[1]) and np.array_equal(rows[0], rows[2])
        cols = rows[0]
        assert len(cols) % 3 == 0 and len(cols) <= 81
        assert np.array_equal(cols[0::3] + 1, cols[1::3]) and np.array_equal(cols[0::3] + 2, cols[2::3])
        assert np.all(cols[0::3] % 3 == 0) and np.all(np.diff(cols[0::3]) > 0)
    # uniform modulus, end traction along +y: the free end moves along +y
    b = op.end_traction(0.0)
    x = np.linalg.solve(op.csr(np.ones_like(E)).todense(), b).reshape(-1, 3)
    tip = op.fix == op.nx - 1
    assert np.all(x[tip, 1] > 0) and np.abs(x[tip, 1]).mean() > 10 * np.abs(x[tip, 2]).mean()


def test_random_spd_csr_structure():
    A = wl.random_spd_csr(300, 0.05, seed=3, empty_rows=7)
    D = A.todense()
    assert np.array_equal(D, D.T)
    off = np.abs(D).sum(1) - np.abs(np.diag(D))
    assert np.all(np.diag(D) > off)             # strictly diagonally dominant
    assert np.all(np.diff(A.row_ptr)[:7] == 1)  # the empty rows hold their diagonal only
    assert np.diff(A.row_ptr).max() > 5 * np.median(np.diff(A.row_ptr))   # heavy-tailed rows


def test_smooth_snapshots():
    op = wl.DiffusionOperator((6, 7, 8))
    S = wl.smooth_snapshots(op, 12, modes=5, seed=4)
    assert S.shape == (op.n, 12) and S.flags.f_contiguous
    assert np.array_equal(S, wl.smooth_snapshots(op, 12, modes=5, seed=4))
    sv = np.linalg.svd(S, compute_uv=False)
    assert np.sum(sv > 1e-10 * sv[0]) <= 5


def test_moving_source_sequence():
    seq = wl.diffusion3d_moving(m=16, p=4)
    prev = None
    for j, val, b in seq.systems():
        assert len(val) == seq.nnz and len(b) == seq.n
        # the source peak sits at the documented centre on the circle
        m = 16
        ang = 2 * np.pi * j / 50.0
        cx, cy = m / 2 + m / 4 * np.cos(ang), m / 2 + m / 4 * np.sin(ang)
        z, y, x = np.unravel_index(np.argmax(b), (m, m, m))
        assert abs(x - cx) <= 1 and abs(y - cy) <= 1 and abs(z - m / 2) <= 1
        if prev is not None:   # coefficients perturbed by about 0.5% per system
            rel = np.abs(val / prev - 1)
            assert 1e-4 < np.median(rel) < 2e-2
        prev = val
