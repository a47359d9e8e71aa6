"""The failure path of the bounded device waits, exercised without a GPU fault.

The tensor-core Gram and the FP32 passes staged by the TMA engine wait on mbarriers that their
own copies complete. pod_cg_debug_wait_timeout makes those kernels issue no copies and cut
every wait to 2e6 SM clocks (about a millisecond), so each wait expires with nothing in
flight: the kernel records the timeout status (7) and returns. The persistent FP32 loop waits
at grid barriers; with its bit set the last CTA to arrive does not release the barrier, so
every wait runs out (about 2e6 ns) and each CTA leaves the loop. The tests check that the
status reaches the caller (ERR_TIMEOUT from a solve, NaN from the stateless Gram), and that
with the override cleared the same handle, or the same call, gives the normal result: the
context and the handle stay usable.
"""
import numpy as np
import pytest

from paper_1512_05820_gb300 import workloads as wl

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

CYCLES = 2_000_000


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1512_05820_gb300 import _lib
    L = _lib.load()
    yield L
    assert L.pod_cg_debug_wait_timeout(0, 0) == 0


@pytest.fixture()
def override(lib):
    def set_mask(mask):
        assert lib.pod_cg_debug_wait_timeout(mask, CYCLES if mask else 0) == 0
    yield set_mask
    set_mask(0)


def test_override_rejects_bad_arguments(lib):
    assert lib.pod_cg_debug_wait_timeout(8, CYCLES) == 1
    assert lib.pod_cg_debug_wait_timeout(1, 10) == 1
    assert lib.pod_cg_debug_wait_timeout(-1, CYCLES) == 1


def test_gram_tc_wait_expires(lib, override):
    from paper_1512_05820_gb300 import solver
    rng = np.random.default_rng(3)
    n = 8192
    Xh, Yh = rng.normal(size=(n, 8)).astype(np.float32), rng.normal(size=(n, 9)).astype(np.float32)
    X, Y = torch.as_tensor(Xh, device="cuda"), torch.as_tensor(Yh, device="cuda")
    override(1)
    G = solver.gram_tc(X, Y)
    torch.cuda.synchronize()
    assert torch.isnan(G).all()
    override(0)
    G = solver.gram_tc(X, Y).cpu().numpy()
    ref = Xh.astype(np.float64).T @ Yh.astype(np.float64)
    bound = 1e-6 * n * np.outer(np.linalg.norm(Xh, axis=0), np.linalg.norm(Yh, axis=0)) / n ** 0.5
    assert np.all(np.abs(G - ref) <= bound)


def _sequence_case():
    seq = wl.diffusion3d_moving(m=24, p=3, period=6)
    return seq, seq.all_systems()


def _solve_pair(mask, override, **cfg):
    """Solve system 1, record its solution, then system 2 with `mask` set on the same
    handle; then system 2 again with the override cleared. Also system 2 on a fresh handle
    with the same snapshot. Returns the three (x, stats)."""
    from paper_1512_05820_gb300.solver import DeviceCSR, PodCG
    seq, systems = _sequence_case()
    A0 = DeviceCSR.from_numpy(seq.row_ptr, seq.col, np.zeros(seq.nnz))
    mats = [A0.with_values(torch.as_tensor(v, device="cuda")) for _, v, _ in systems]
    bs = [torch.as_tensor(b, device="cuda") for _, _, b in systems]

    def handle():
        return PodCG(seq.n, w_max=seq.w_max, s_max=seq.s_max, energy=seq.energy, precision=1, **cfg)
    h = handle()
    x1, st1 = h.solve(mats[0], bs[0], seq.tol)
    assert st1["status"] == "ok"
    h.add_snapshots(x1)
    override(mask)
    bad = h.solve(mats[1], bs[1], seq.tol, raise_on_error=False)
    override(0)
    again = h.solve(mats[1], bs[1], seq.tol, raise_on_error=False)
    h.close()
    f = handle()
    f.add_snapshots(x1)
    fresh = f.solve(mats[1], bs[1], seq.tol, raise_on_error=False)
    f.close()
    return bad, again, fresh, seq


@pytest.mark.parametrize("mask,cfg", [(2, dict(proj_form=1)), (1, dict(use_tc_gram=1)), (4, dict(loop_mode=2))],
                         ids=["staged-passes", "tensor-core-gram", "persistent-loop-barrier"])
def test_solve_wait_expires_then_recovers(lib, override, mask, cfg):
    (xb, stb), (xa, sta), (xf, stf), seq = _solve_pair(mask, override, **cfg)
    assert stb["status"] == "timeout", stb
    assert sta["status"] == "ok" and stf["status"] == "ok" and sta["w"] > 0, (sta, stf)
    assert sta["final_relres"] <= seq.tol
    # the handle that saw the timeout solves exactly as a fresh one
    assert sta["iters"] == stf["iters"]
    assert torch.equal(xa, xf)
