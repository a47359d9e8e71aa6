"""Batched persistent solver against the FP64 oracle, sequence by sequence.

The batch runs each sequence with its own (FP32-inner, FP64-refined) solutions as
snapshots, so it is compared with the oracle's run of the same sequence: every system's
FP64 true residual <= tol (re-checked on the CPU), solutions within the accuracy two
solutions of residual <= tol can differ by, and POD dimensions within one."""
import numpy as np
import pytest

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


def small_batch():
    seqs = wl.batch_sequences(nseq=7, p=4, n_min=150, n_max=5000, seed=5, w_range=(3, 10), s_max=4)
    seqs.append(wl.diffusion2d_drift(m=3, p=3, seed=1, w_max=2, s_max=3))   # n = 9
    return seqs


@pytest.mark.parametrize("cluster", [1, 2, 4, 0])
def test_batch_matches_oracle(dev, cluster):
    from paper_1512_05820_gb300.batch import BatchSolver
    seqs = small_batch()
    systems = [s.all_systems() for s in seqs]
    bs = BatchSolver(seqs, device=dev, cluster=cluster, systems=systems)
    stats, ms = bs.solve()
    orc = Oracle()
    k = 0
    for i, (seq, sy) in enumerate(zip(seqs, systems)):
        X = bs.solutions(i).cpu().numpy()
        oseq = OracleSequence(seq.n, s_max=min(seq.s_max, 16), w_max=seq.w_max, energy=seq.energy, oracle=orc)
        for j, (_, val, b) in enumerate(sy):
            A = (seq.row_ptr, seq.col, val)
            xo, info = oseq.solve(A, b, seq.tol)
            st = stats[k]
            k += 1
            x = X[j]
            true_rel = np.linalg.norm(b - orc.spmv(A, x)) / np.linalg.norm(b)
            assert st["status"] == "ok", (i, j, st)
            assert true_rel <= seq.tol and st["final_relres"] <= seq.tol * 1.0000001, (i, j, true_rel, st)
            assert abs(st["w"] - info["w"]) <= 1, (i, j, st["w"], info["w"])
            dx = x - xo
            err = np.sqrt(max(dx @ orc.spmv(A, dx), 0.0) / (xo @ orc.spmv(A, xo)))
            assert err <= 1e-5, (i, j, err)
    if cluster == 0:
        assert bs.info()["cluster"] in (2, 4, 8)
    bs.close()


def test_batch_repeatable(dev):
    """Two launches of the same batch give identical solutions (fixed reduction order)."""
    from paper_1512_05820_gb300.batch import BatchSolver
    seqs = small_batch()[:4]
    bs = BatchSolver(seqs, device=dev, cluster=2)
    bs.solve()
    first = [bs.solutions(i).clone() for i in range(len(seqs))]
    bs.solve()
    for i in range(len(seqs)):
        assert torch.equal(first[i], bs.solutions(i))
    bs.close()


def tile_batch():
    """Sequences of all three size classes of the tile autotuner (n < 16k, < 64k, larger),
    with n a multiple of 4 and not, so both row widths run."""
    return [wl.diffusion2d_drift(m=63, p=3, seed=2, w_max=6, s_max=4),          # n = 3969
            wl.diffusion3d_moving(m=22, p=3, s_max=4, w_max=8, period=6),       # n = 10648
            wl.diffusion3d_moving(m=31, p=3, s_max=4, w_max=8, period=6),       # n = 29791
            wl.diffusion3d_moving(m=42, p=3, s_max=4, w_max=8, period=6)]       # n = 74088


@pytest.mark.parametrize("lanes,rows", [(1, 1), (1, 4), (2, 4), (4, 4), (8, 1), (8, 4)])
def test_batch_tiles_match_oracle(dev, lanes, rows):
    """Every tile shape of the inner loop (lanes per CSR row, rows per thread) on sequences
    of every size class against the oracle's run of the same sequences."""
    from paper_1512_05820_gb300.batch import BatchSolver
    seqs = tile_batch()
    systems = [s.all_systems() for s in seqs]
    bs = BatchSolver(seqs, device=dev, cluster=4, systems=systems)
    bs.set_tiles(lanes, rows)
    stats, _ = bs.solve()
    orc = Oracle()
    k = 0
    for i, (seq, sy) in enumerate(zip(seqs, systems)):
        X = bs.solutions(i).cpu().numpy()
        oseq = OracleSequence(seq.n, s_max=min(seq.s_max, 16), w_max=seq.w_max, energy=seq.energy, oracle=orc)
        for j, (_, val, b) in enumerate(sy):
            A = (seq.row_ptr, seq.col, val)
            xo, info = oseq.solve(A, b, seq.tol)
            st = stats[k]
            k += 1
            x = X[j]
            assert st["status"] == "ok", (i, j, st)
            assert np.linalg.norm(b - orc.spmv(A, x)) / np.linalg.norm(b) <= seq.tol
            dx = x - xo
            assert np.sqrt(max(dx @ orc.spmv(A, dx), 0.0) / (xo @ orc.spmv(A, xo))) <= 1e-5, (i, j)
    bs.close()


def test_batch_tile_autotuner_record(dev):
    """With cluster = 0 the handle tunes the cluster size, then the tiles per size class:
    every class present has timings for all four candidates and keeps the fastest."""
    from paper_1512_05820_gb300.batch import BatchSolver
    seqs = tile_batch()
    bs = BatchSolver(seqs, device=dev, cluster=0)
    tiles = bs.info()["tiles"]
    stats, _ = bs.solve()
    bs.close()
    assert all(s["status"] == "ok" for s in stats)
    for cls in ("n<16k", "16k<=n<64k", "n>=64k"):
        rec = tiles[cls]
        ms = rec["ms"]
        assert all(v > 0 for v in ms.values()), (cls, ms)
        best = min(ms, key=ms.get)
        assert best == f"lanes{rec['spmv_lanes']}_rows{rec['rows_per_thread']}"
