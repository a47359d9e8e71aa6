"""The cost-tuned cap on the basis size (w_select = 1): once 8 snapshots are held the handle
times each candidate cap on two solves, in the order c1 .. ck ck .. c1, then keeps the cap
with the least mean device time. Every solve still meets its tolerance, later bases respect
the cap, and the record reports the choice."""
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


@pytest.mark.parametrize("precision", [0, 1], ids=["fp64", "mixed"])
def test_cost_tuned_cap(dev, precision):
    from paper_1512_05820_gb300.sequence import DeviceSequence, run_sequence
    from paper_1512_05820_gb300.solver import PodCG
    seq = wl.diffusion3d_moving(m=24, p=24, period=12)
    dseq = DeviceSequence(seq)
    h = PodCG(seq.n, w_max=16, s_max=seq.s_max, energy=seq.energy, precision=precision, w_select=1)
    assert h.tuning()["w_cap"]["cap"] == 16
    stats = run_sequence(h, dseq)
    rec = h.tuning()["w_cap"]
    ms = rec["ms_per_solve"]
    assert sorted(int(k) for k in ms) == [2, 4, 8, 16]
    assert all(v > 0 for v in ms.values()), ms
    assert rec["cap"] == int(min(ms, key=ms.get))
    assert all(s["status"] == "ok" and s["final_relres"] <= seq.tol for s in stats)
    # explored from the 9th system (8 snapshots held) for 2 x 4 solves; later ones use the cap
    assert all(s["w"] <= rec["cap"] for s in stats[8 + 8:])
    # a second pass keeps the tuned cap
    stats2 = run_sequence(h, dseq)
    assert all(s["w"] <= rec["cap"] and s["final_relres"] <= seq.tol for s in stats2)
    h.close()


def test_energy_rule_is_default(dev):
    from paper_1512_05820_gb300.sequence import DeviceSequence, run_sequence
    from paper_1512_05820_gb300.solver import PodCG
    seq = wl.diffusion2d_drift(m=32, p=6)
    h = PodCG(seq.n, w_max=8, s_max=seq.s_max, energy=seq.energy)
    run_sequence(h, DeviceSequence(seq))
    rec = h.tuning()["w_cap"]
    assert rec == {"cap": 8, "ms_per_solve": {}}
    h.close()
