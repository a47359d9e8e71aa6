"""The paper's own POD ingredients on the GPU (Section 3, Algorithm 3): snapshots are the
accumulated stage-three directions, A_j-normalised; previous / RBF weights; compression by
the weighted POD in the metric A_j; the stage-one set chosen by nu. Each sequence is run by
the library (pod_cg_set_krylov) and by the oracle's OracleKrylovSequence with the same
settings, system by system: same stage-three iteration counts (within one), same basis
sizes and compressions, solutions within 1e-10 in the A-norm, every true residual <= tol.
"""
import numpy as np
import pytest

from oracle import Oracle, OracleKrylovSequence
from paper_1512_05820_gb300 import workloads as wl

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-10


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1512_05820_gb300 import _lib
    _lib.load()
    return torch.device("cuda:0")


def _run(seq, systems, **kc):
    """Both sides over the sequence; returns per-system (gpu x, gpu stats, gpu state, oracle x,
    oracle info, oracle z, oracle w)."""
    from paper_1512_05820_gb300.solver import DeviceCSR, PodCG
    orc = Oracle()
    o = OracleKrylovSequence(seq.n, y_threshold=kc["y_threshold"] or 10 ** 6, y_keep=kc["y_keep"],
                             w_keep=kc["w_keep"], nu=kc["nu"], weights=kc["weights"], p_cap=kc["p_cap"], oracle=orc)
    h = PodCG(seq.n, three_stage=1, w_max=32, s_max=40, tol_stage2=1e-4)
    h.set_krylov(**kc)
    A0 = DeviceCSR.from_numpy(seq.row_ptr, seq.col, np.zeros(seq.nnz))
    out = []
    for j, val, b in systems:
        A = A0.with_values(torch.as_tensor(val, device="cuda"))
        x, st = h.solve(A, torch.as_tensor(b, device="cuda"), TOL)
        state = h.krylov_state(with_basis=True)
        xo, info = o.solve((seq.row_ptr, seq.col, val), b, TOL)
        out.append((x.cpu().numpy(), st, state, xo, info, o.Z.shape[1], len(o.w_idx), (val, b)))
    h.close()
    return out, orc


def _check(seq, out, orc):
    for j, (x, st, state, xo, info, oz, ow, (val, b)) in enumerate(out):
        A = (seq.row_ptr, seq.col, val)
        assert st["status"] == "ok", (j, st)
        rel = np.linalg.norm(b - orc.spmv(A, x)) / np.linalg.norm(b)
        assert rel <= TOL * (1 + 1e-9), (j, rel)
        assert abs(st["iters"] - info["iters"]) <= 1, (j, st["iters"], info["iters"])
        assert state["z"] == oz and state["w"] == ow, (j, state["z"], oz, state["w"], ow)
        dx = x - xo
        err = np.sqrt(max(dx @ orc.spmv(A, dx), 0.0) / (xo @ orc.spmv(A, xo)))
        assert err <= 1e-10, (j, err)


@pytest.mark.parametrize("nu,weights", [(1.0, "rbf"), (0.0, "rbf"), (0.05, "prev")],
                         ids=["all-in-W-rbf", "stage-two-only-rbf", "nu-0.05-prev"])
def test_krylov_sequence_matches_oracle(dev, nu, weights):
    """Compressions every system past the first: 24 directions per system against a storage
    threshold of 40, kept to 20 (the first 4 form W)."""
    seq = wl.diffusion2d_drift(m=20, p=6)
    out, orc = _run(seq, seq.all_systems(), y_threshold=40, y_keep=20, w_keep=4, nu=nu, weights=weights, p_cap=24)
    _check(seq, out, orc)
    assert out[-1][2]["compressions"] >= 3
    iters = [o[1]["iters"] for o in out]
    assert all(it < iters[0] for it in iters[1:]), iters


def test_krylov_accumulation_without_compression(dev):
    """Storage threshold 0 (no automatic compression): Z grows by p_cap per system up to 60
    columns; the stage-one set is every direction (nu = 1)."""
    seq = wl.diffusion2d_drift(m=24, p=5, seed=7)
    out, orc = _run(seq, seq.all_systems(), y_threshold=0, y_keep=20, w_keep=4, nu=1.0, weights="rbf", p_cap=12)
    _check(seq, out, orc)
    assert [o[2]["z"] for o in out] == [min(12 * (j + 1), 60) for j in range(5)]


def test_compressed_basis_is_a_orthonormal_and_weights_match(dev):
    """After a compression Z^T A_j Z = I (the metric-A POD, Section 3.3); the previous
    weights the library forms are the pseudo-inverse solution (Z^T A Z)^+ Z^T b recomputed
    on the host from the library's own Z; a forced compression with given weights spans the
    oracle's weighted POD subspace of the same Z."""
    from paper_1512_05820_gb300.solver import DeviceCSR, PodCG
    seq = wl.diffusion2d_drift(m=20, p=3, seed=11)
    systems = seq.all_systems()
    orc = Oracle()
    h = PodCG(seq.n, three_stage=1, tol_stage2=1e-4)
    h.set_krylov(y_threshold=0, y_keep=16, w_keep=3, nu=1.0, weights="rbf", p_cap=20)
    A0 = DeviceCSR.from_numpy(seq.row_ptr, seq.col, np.zeros(seq.nnz))
    for _, val, b in systems[:2]:
        A = A0.with_values(torch.as_tensor(val, device="cuda"))
        h.solve(A, torch.as_tensor(b, device="cuda"), TOL)
    _, val, b = systems[2]
    A = A0.with_values(torch.as_tensor(val, device="cuda"))
    D = wl.CSR(seq.n, seq.row_ptr, seq.col, val).todense()
    Z = h.krylov_state(with_basis=True)["Z"].cpu().numpy()
    c, eta = h.krylov_coords(A, torch.as_tensor(b, device="cuda"))
    G = Z.T @ D @ Z
    ref = np.linalg.lstsq(0.5 * (G + G.T), Z.T @ b, rcond=1e-13)[0]
    c = c.cpu().numpy()
    # the pseudo-inverse solutions agree in the A-norm of the vectors they expand
    assert np.sqrt((c - ref) @ G @ (c - ref)) <= 1e-9 * np.sqrt(ref @ G @ ref)
    eta_h = np.linspace(1.0, 2.0, Z.shape[1])
    h.krylov_compress(A, torch.as_tensor(eta_h, device="cuda"), 10, 3)
    st = h.krylov_state(with_basis=True)
    Zc = st["Z"].cpu().numpy()
    assert st["z"] == 10 and st["w"] == 3 and st["compressions"] == 1
    assert np.max(np.abs(Zc.T @ D @ Zc - np.eye(10))) <= 1e-10
    Wk, yk, _ = orc.pod_evd_metric(Z * eta_h[None, :], (seq.row_ptr, seq.col, val), 2.0, 10)
    # same A-orthogonal projector onto the 10-dimensional weighted POD subspace
    Pg = Zc @ (Zc.T @ D)
    Po = Wk @ (Wk.T @ D)
    assert yk == 10 and np.max(np.abs(Pg - Po)) <= 1e-8 * np.max(np.abs(Po))
    h.close()


def test_krylov_mode_rejects_bad_settings(dev):
    from paper_1512_05820_gb300.solver import PodCG, PodCGError
    h = PodCG(400, three_stage=1)
    with pytest.raises(PodCGError):
        h.set_krylov(y_threshold=50, p_cap=20)          # 50 + 20 > 64
    with pytest.raises(PodCGError):
        h.set_krylov(y_threshold=30, y_keep=40)         # y_keep above the threshold
    h.close()
    h = PodCG(400, precision=1, three_stage=1)
    with pytest.raises(PodCGError):
        h.set_krylov()                                  # MIXED handle
    h.close()
    h = PodCG(400)
    with pytest.raises(PodCGError):
        h.set_krylov()                                  # two-stage handle
    h.close()


def test_krylov_sequence_3d_matches_oracle(dev):
    """A 3D sequence (24^3 moving source) with 32 directions per system, a storage threshold
    of 32, compression to 16 after every system past the first (W = the first 6 modes) and
    ν = 0.05 (a few new directions join W between compressions): system by system against
    the oracle, as in the 2D cases."""
    seq = wl.diffusion3d_moving(m=24, p=5, period=10)
    out, orc = _run(seq, seq.all_systems(), y_threshold=32, y_keep=16, w_keep=6, nu=0.05, weights="rbf", p_cap=32)
    _check(seq, out, orc)
    assert out[-1][2]["compressions"] == 4
