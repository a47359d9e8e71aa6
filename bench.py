#!/usr/bin/env python
"""Benchmark: systems solved/s and SpMV-equivalent GB/s, POD-augmented CG vs plain CG.

Workload (default): the 128^3 seven-point variable-coefficient diffusion sequence of 50
systems (lognormal(0, 1) coefficients perturbed 0.5% per system, moving heat source),
POD of the last 40 solutions truncated at 99.99% energy to w <= 32, Jacobi
preconditioner, relative residual 1e-8. One step = solving the whole sequence on the GPU
(POD + stage one + stage three for each system, snapshots recorded as it goes), inputs
resident in HBM. A_j values (117 MB each) and the basis blocks (~1 GB) exceed the 129 MB
L2, so no L2 flush is needed between steps.

Prints one JSON line on rank 0. ``--impl reference`` times the FP64 CPU oracle (the
reference arm: the paper has no code to run) on a bounded sample of the same workload
instead.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "systems solved/s and SpMV-equiv HBM GB/s to rel. residual 1e-8: POD-aug vs plain CG"
FALLBACK_HBM_GBS = 6800.0


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--grid", type=int, default=128, help="grid edge m (m^3 cells)")
    ap.add_argument("--systems", type=int, default=50)
    ap.add_argument("--w-max", type=int, default=32, help="largest POD basis (the sequence's w_max)")
    ap.add_argument("--energy", type=float, default=0.9999, help="POD energy fraction kept")
    ap.add_argument("--w-select", choices=["cost", "energy"], default="cost",
                    help="basis size: energy criterion under a cap tuned by measured cost (the handle times "
                         "candidate caps on its first pass over the sequence), or the energy criterion alone")
    ap.add_argument("--precision", choices=["fp64", "mixed"], default="mixed")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-compare", action="store_true")
    ap.add_argument("--kernel-reps", type=int, default=20)
    ap.add_argument("--no-batch", action="store_true", help="skip the batched-sequences measurement")
    ap.add_argument("--diff-check", type=int, default=0, metavar="K",
                    help="differentiation check on the 96^3, 20-system theta workload: adjoint dL/dtheta "
                         "against fourth-order central differences at K random cells")
    ap.add_argument("--kernel-profile", type=int, default=0, metavar="W",
                    help="profiling target: one full-size system with W synthetic snapshots, a 5-iteration "
                         "solve, then each stage-three kernel launched --kernel-reps times (few launches)")
    ap.add_argument("--gram-profile", action="store_true",
                    help="profiling target: the tensor-core Gram W^T [AW, b] at n = 2,097,152, w = 22 (FP32 "
                         "inputs), launched --kernel-reps times")
    ap.add_argument("--no-gram", action="store_true", help="skip the stage-one Gram measurement")
    ap.add_argument("--elasticity", type=int, default=0, metavar="K",
                    help="the 64^3-element cantilever, first K systems: POD-aug (mixed; tensor-core and "
                         "CUDA-core stage-one Gram) against plain Jacobi CG (mixed), one JSON line")
    ap.add_argument("--proj-form", choices=["auto", "direct", "staged"], default="auto",
                    help="FP32 update/direction form: timed per width bucket (auto), row-parallel float4, "
                         "or tiles staged by bulk copies")
    ap.add_argument("--spmv-lanes", type=int, default=0, choices=[0, 1, 2, 4, 8, 16, 32],
                    help="CSR SpMV lanes per row (0: timed by the handle); profiling commands force the "
                         "timed choice so the profiled kernels are the ones the bench times")
    ap.add_argument("--three-stage", action="store_true",
                    help="the three-stage algorithm (Section 4) against the two-stage form on the same "
                         "sequence (the --grid/--systems diffusion sequence, or the cantilever with "
                         "--elasticity K), each timed over the sequence after one untimed pass; one JSON line")
    ap.add_argument("--stage2-profile", type=int, default=0, metavar="Y",
                    help="profiling target: system 1 of the workload with Y seeded random snapshots, FP64, "
                         "stage two run to its cap (y - w reduced iterations, host-driven launches), then 5 "
                         "iterations of stage three with [W, V2] and 5 with the whole Y; one JSON line")
    ap.add_argument("--output-pod", type=int, default=0, metavar="Q",
                    help="output-oriented POD (metric C^T C, Q random U[0,1] functionals) against the identity "
                         "metric on the --grid/--systems diffusion sequence; one JSON line")
    ap.add_argument("--bsr", type=int, default=-1, choices=[-1, 0, 1],
                    help="CG product in 3x3 block form: -1 when the pattern allows (default), 0 never, 1 required")
    ap.add_argument("--batch-seqs", type=int, default=256)
    ap.add_argument("--batch-profile", type=int, default=0, metavar="N",
                    help="a short launch sequence for kernel profilers of the batched solver: N sequences of "
                         "the batch workload, cluster 4, 1 lane per CSR row, 4 rows per thread, two solves")
    ap.add_argument("--krylov", action="store_true",
                    help="the paper's Krylov-vector snapshots (Algorithm 3): the 128^3 sequence against "
                         "POD of previous solutions, and the POD-weights study (ideal / previous / RBF)")
    ap.add_argument("--loop-mode", choices=["graph", "chunked", "persistent"], default="graph",
                    help="graph: conditional CUDA graph; chunked: plain graphs of 16 iterations (profilable); "
                         "persistent: as graph, the mixed inner loop at w <= 8 as one cooperative launch")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def workload(args):
    from paper_1512_05820_gb300 import workloads as wl
    return wl.diffusion3d_moving(m=args.grid, p=args.systems, w_max=args.w_max, energy=args.energy)


def config_dict(seq, args, precision):
    return {"workload": f"diffusion3d_moving {args.grid}^3 7-point, {seq.p} systems",
            "n": seq.n, "nnz": seq.nnz, "systems": seq.p, "s_max": seq.s_max, "w_max": seq.w_max,
            "energy": seq.energy, "tol": seq.tol, "precision": precision, "preconditioner": "jacobi",
            "w_select": getattr(args, "w_select", "energy"),
            "l2": l2_note(seq), "parallelism": "replicas" if args.gpus > 1 else "single"}


L2_BYTES = 129e6   # GB300 L2


def l2_note(seq):
    """How the data one iteration reads compares with L2 (no flush between iterations):
    the matrix (values, column indices, row pointers) and the W and A W blocks."""
    mat_mb = (12 * seq.nnz + 4 * (seq.n + 1)) / 1e6
    blocks_mb = 2 * seq.w_max * seq.n * 4 / 1e6   # W and A W in FP32, at w_max
    if (mat_mb + blocks_mb) * 1e6 > L2_BYTES:
        return (f"inputs larger than L2 (matrix {mat_mb:.0f} MB per system, W and AW up to "
                f"{blocks_mb:.0f} MB); no flush")
    return f"inputs fit in L2 (matrix {mat_mb:.1f} MB); no flush: a small case, not the benchmark size"


def b_spmv(n, nnz, fp32=False):
    """Bytes of one CSR SpMV that move once: values, column indices, row pointers, the
    input vector and the output vector (FP64: 12 nnz + 4(n+1) + 16 n; FP32 values and
    vectors: 8 nnz + 4(n+1) + 8 n)."""
    return (8 * nnz + 4 * (n + 1) + 8 * n) if fp32 else (12 * nnz + 4 * (n + 1) + 16 * n)


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return FALLBACK_HBM_GBS, "fallback"


def measured_bf16_tflops():
    """Dense bf16 tensor peak for a kernel timed alone (the burst figure), or the fallback."""
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            return float(json.load(f).get("bf16_tflops", 1900.0))
    return 1900.0


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        with open(self.path) as f:
            for line in f:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}

        def num(v):
            try:
                return float(v)
            except ValueError:
                return float("nan")
        sm = [num(r[1]) for r in rows]
        smax = [num(r[2]) for r in rows]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].lower() == "active"})
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "samples": len(rows),
                "reasons": reasons}


KERNEL_SOURCE = {"k_update": "k_cg.cu", "k_dir": "k_cg.cu", "k_init": "k_cg.cu", "k_update_tma": "k_cg.cu",
                 "k_dir_tma": "k_cg.cu", "k_update_v4": "k_cg.cu", "k_dir_v4": "k_cg.cu", "k_spmv_cg": "k_sparse.cu", "k_residual": "k_sparse.cu",
                 "k_gram_tc": "k_gram_tc.cu", "k_cg_loop": "k_loop.cu"}


def traffic_from_profiles(kernel: str, precision: str, w: int):
    """Per-launch DRAM bytes of `kernel` from a committed ncu summary (profiles/*.txt lines
    `traffic_bytes_per_launch <kernel> <precision> <w> <bytes> <sha1 prefix of its source>`),
    or None when there is none for this kernel, precision and w, or when the kernel's source
    file has changed since the counters were taken."""
    d = os.path.join(ROOT, "profiles")
    src = KERNEL_SOURCE.get(kernel)
    if not os.path.isdir(d) or src is None:
        return None
    with open(os.path.join(ROOT, "paper_1512_05820_gb300", "csrc", src), "rb") as f:
        digest = hashlib.sha1(f.read()).hexdigest()
    for fn in sorted(os.listdir(d)):
        if not fn.endswith(".txt"):
            continue
        with open(os.path.join(d, fn)) as f:
            for line in f:
                parts = line.split()
                if (len(parts) >= 6 and parts[0] == "traffic_bytes_per_launch" and parts[1] == kernel
                        and parts[2] == precision and int(parts[3]) == w and digest.startswith(parts[5])):
                    return float(parts[4])
    return None


# ----------------------------------------------------------------------- reference arm


CPU_PREFIX = 2   # the oracle's sample: systems 1..CPU_PREFIX of the sequence


def oracle_prefix_sample(grid: int, systems_total: int, k: int = CPU_PREFIX) -> dict:
    """One bounded sample of the workload on the FP64 oracle, single-threaded: the first k
    systems of the sequence solved in order by the POD-augmented method (OracleSequence:
    POD of the solutions so far, stage one, Algorithm 1, each solution recorded as a
    snapshot), then plain Jacobi PCG on the same systems. System 1 has no snapshots, so its
    POD-augmented solve is plain PCG (pinned bit for bit), and its time counts for both."""
    from oracle import Oracle, OracleSequence
    from paper_1512_05820_gb300 import workloads as wl
    seq = wl.diffusion3d_moving(m=grid, p=systems_total)
    it = seq.systems()
    sy = [next(it) for _ in range(k)]
    orc = Oracle()
    oseq = OracleSequence(seq.n, s_max=seq.s_max, w_max=seq.w_max, energy=seq.energy, oracle=orc)
    xs, t_sys, its, ws = [], [], [], []
    for j, val, b in sy:
        t0 = time.perf_counter()
        x, info = oseq.solve((seq.row_ptr, seq.col, val), b, seq.tol)
        t_sys.append(time.perf_counter() - t0)
        xs.append(x)
        its.append(info["iters"])
        ws.append(info["w"])
    t_plain, its_plain = [t_sys[0]], [its[0]]
    for j, val, b in sy[1:]:
        t0 = time.perf_counter()
        _, info, _, _ = orc.solve_system((seq.row_ptr, seq.col, val), b, None, seq.tol)
        t_plain.append(time.perf_counter() - t0)
        its_plain.append(info["iters"])
    return {"xs": xs, "t_pod_aug": sum(t_sys), "t_plain": sum(t_plain), "iters": its, "w": ws,
            "iters_plain": its_plain, "k": k}


def _reference_worker(task):
    grid, systems_total, k = task
    r = oracle_prefix_sample(grid, systems_total, k)
    del r["xs"]
    return r


def run_reference(args, rank, world):
    """The FP64 CPU oracle on the host cores. One step = one bounded sample of the workload
    (oracle_prefix_sample: systems 1-2 by the POD-augmented method, then plain PCG on the
    same systems, one thread). The W warm-up steps, then the K timed steps, run as
    independent single-threaded processes, min(cores, K) at a time; value = K x 2 systems
    over the wall time of the timed steps (the host's aggregate rate), ms_per_step = that
    wall time / K."""
    if rank != 0:
        return 0
    import multiprocessing as mp
    from paper_1512_05820_gb300 import workloads as wl
    seq = wl.diffusion3d_moving(m=args.grid, p=args.systems)
    ncpu = os.cpu_count() or 1
    procs = max(1, min(ncpu, args.steps))
    task = (args.grid, args.systems, CPU_PREFIX)
    ctx = mp.get_context("spawn")
    with ctx.Pool(procs) as pool:
        if args.warmup:
            pool.map(_reference_worker, [task] * args.warmup, chunksize=1)
        t0 = time.perf_counter()
        res = pool.map(_reference_worker, [task] * args.steps, chunksize=1)
        wall = time.perf_counter() - t0
    systems = args.steps * CPU_PREFIX
    value = systems / wall
    one = statistics.mean(r["t_pod_aug"] for r in res)
    plain = statistics.mean(r["t_plain"] for r in res)
    r0 = res[0]
    sample = (f"systems 1-{CPU_PREFIX} of {seq.p} at full size by the oracle's POD-augmented method "
              f"(w {r0['w']}, iterations {r0['iters']}), then plain PCG on the same systems (iterations "
              f"{r0['iters_plain']}); {args.steps} independent single-threaded copies, {procs} at a time on "
              f"{ncpu} host cores; per copy (one thread): POD-aug {CPU_PREFIX / one:.4f} systems/s, plain PCG "
              f"{CPU_PREFIX / plain:.4f} systems/s")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "systems/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": wall / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": config_dict(seq, args, args.precision),   # the timed arm's config; dtype says f64
            "cpu_baseline": {"value": value, "unit": "systems/s", "cores": procs, "kind": "oracle",
                             "nproc": ncpu, "sample": sample},
            "e2e": {"value": value, "unit": "systems/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def a_norm_rel(orc, A, x, xo) -> float:
    """||x - xo||_A / ||xo||_A with the oracle's FP64 SpMV."""
    d = np.asarray(x, dtype=np.float64) - xo
    return float(np.sqrt(max(d @ orc.spmv(A, d), 0.0) / max(xo @ orc.spmv(A, xo), 1e-300)))


# ----------------------------------------------------------------------------- ours


def batch_section(args, rank=0, world=1):
    """Many independent sequences (256 x 8 systems, n log-uniform in [2k, 260k], 2D/3D mixed,
    w_max in [4, 24]) in one persistent launch under a CUDA graph, cluster size autotuned,
    FP32 inner + FP64 refinement; compared with the single-sequence engine in FP64 on the
    first 32 sequences at the same tolerance."""
    import torch
    from paper_1512_05820_gb300 import workloads as wl
    from paper_1512_05820_gb300.batch import BatchSolver
    from paper_1512_05820_gb300.sequence import DeviceSequence, run_sequence
    from paper_1512_05820_gb300.solver import PodCG
    from paper_1512_05820_gb300.dist import combine, shard_by_work
    all_seqs = wl.batch_sequences(nseq=args.batch_seqs)
    mine = shard_by_work([float(s.nnz) * s.p * s.n ** (1 / 3) for s in all_seqs], rank, world)
    seqs = [all_seqs[i] for i in mine]   # independent sequences: each rank solves its share
    systems = [s.all_systems() for s in seqs]
    t0 = time.perf_counter()
    bs = BatchSolver(seqs, systems=systems, cluster=0)
    tune_s = time.perf_counter() - t0
    bs.solve()
    times, stats = [], None
    for _ in range(max(1, args.steps)):
        stats, ms = bs.solve()
        times.append(ms)
    ms_local = statistics.median(times)
    ms, total = combine(ms_local, float(len(stats)))
    total = int(total)
    ok = int(combine(0.0, float(sum(1 for s in stats if s["status"] == "ok")))[1])
    info = bs.info()
    # algorithmic bytes of every FP32 inner iteration (SpMV 8 nnz + 4(n+1) + 8n; update: d, r
    # read and written, p, q, M^{-1}, A W read: 28n + 4wn; direction: M^{-1}, r, W read, p
    # read and written: 16n + 4wn); setup, POD and FP64 residuals are not counted
    it_bytes, k = 0.0, 0
    for sq in seqs:
        for _ in range(sq.p):
            st_ = stats[k]
            it_bytes += st_["iters"] * (8 * sq.nnz + 4 * (sq.n + 1) + 52 * sq.n + 8 * st_["w"] * sq.n)
            k += 1
    peak, _ = peaks()
    out = {"workload": f"{len(all_seqs)} sequences x {all_seqs[0].p} systems, n in [2k, 260k] log-uniform, 2D/3D",
           "rows_per_layer": int(sum(s.n for s in all_seqs)), "systems": total, "converged": ok,
           "sharding": "independent sequences, no collective" if world > 1 else "single GPU",
           "systems_per_s": total / (ms / 1e3), "ms_per_batch": ms,
           "max_final_relres": max(s["final_relres"] for s in stats),
           "mean_iters": float(np.mean([s["iters"] for s in stats])),
           "cluster": info["cluster"], "workers": info["workers"],
           "autotune_ms": {str(k): v for k, v in info["tune_ms"].items()}, "tiles": info["tiles"], "setup_s": tune_s,
           "roofline": {"bound": "hbm", "kernel": "k_batch", "achieved": it_bytes / (ms_local / 1e3) / 1e9, "peak": peak,
                        "unit": "GB/s", "frac": it_bytes / (ms_local / 1e3) / 1e9 / peak,
                        "bytes": "inner FP32 iterations only (lower bound on the bytes moved)"}}
    out["err_vs_fp64_oracle"] = batch_oracle_error(seqs, systems, bs)
    bs.close()
    if world > 1:
        return out
    # single-sequence engine, FP64, same tolerance, first 32 sequences
    sub = seqs[:32]
    t_single, n_single = 0.0, 0
    for seq, sy in zip(sub, systems[:32]):
        dseq = DeviceSequence(seq, systems=sy)
        solver = PodCG(seq.n, w_max=seq.w_max, s_max=seq.s_max, energy=seq.energy, precision=0)
        run_sequence(solver, dseq)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(solver.stream)
        run_sequence(solver, dseq)
        e1.record(solver.stream)
        torch.cuda.synchronize()
        t_single += e0.elapsed_time(e1)
        n_single += dseq.p
        solver.close()
    out["single_sequence_fp64"] = {"systems_per_s": n_single / (t_single / 1e3), "sample": "first 32 sequences",
                                   "ms": t_single}
    out["speedup_vs_single_fp64"] = out["systems_per_s"] / out["single_sequence_fp64"]["systems_per_s"]
    return out


def batch_profile(args):
    """Two launches of the batched persistent kernel with fixed settings (no autotuning, so a
    profiled run launches the same kernel as a plain one): the first N sequences of the
    batch workload, cluster 4, tiles lanes 1 / rows 4. Prints the second launch's device time
    and the algorithmic bytes of its inner FP32 iterations."""
    from paper_1512_05820_gb300 import workloads as wl
    from paper_1512_05820_gb300.batch import BatchSolver
    seqs = wl.batch_sequences(nseq=args.batch_profile)
    bs = BatchSolver(seqs, cluster=4)
    bs.set_tiles(1, 4)
    bs.solve()
    stats, ms = bs.solve()
    it_bytes, k = 0.0, 0
    for sq in seqs:
        for _ in range(sq.p):
            it_bytes += stats[k]["iters"] * (8 * sq.nnz + 4 * (sq.n + 1) + 52 * sq.n + 8 * stats[k]["w"] * sq.n)
            k += 1
    peak, _ = peaks()
    bs.close()
    print(json.dumps({"batch_profile": True, "sequences": len(seqs), "systems": len(stats), "ms": ms,
                      "inner_bytes": it_bytes, "GB/s": it_bytes / (ms / 1e3) / 1e9,
                      "frac_hbm": it_bytes / (ms / 1e3) / 1e9 / peak,
                      "n_total": int(sum(sq.n for sq in seqs)),
                      "converged": sum(1 for st in stats if st["status"] == "ok")}), flush=True)
    return 0


def cpu_baseline(args, seq, gpu_xs):
    """The oracle sample of the reference arm (systems 1-2, POD-augmented then plain PCG),
    once, single-threaded. Returns the cpu_baseline record and the error of the GPU's
    solutions of the same systems (gpu_xs: host arrays per precision) against the FP64
    oracle's, in the A-norm."""
    from oracle import Oracle
    r = oracle_prefix_sample(args.grid, args.systems)
    k = r["k"]
    rec = {"value": k / r["t_pod_aug"], "unit": "systems/s", "cores": 1, "kind": "oracle",
           "nproc": os.cpu_count() or 1,
           "sample": f"systems 1-{k} of {seq.p} at full size by the oracle's POD-augmented method (w {r['w']}, "
                     f"iterations {r['iters']}, {r['t_pod_aug']:.1f} s); plain PCG on the same systems: "
                     f"{k / r['t_plain']:.4f} systems/s (iterations {r['iters_plain']}); one thread"}
    orc = Oracle()
    it = seq.systems()
    mats = [(seq.row_ptr, seq.col, next(it)[1]) for _ in range(k)]
    err = {}
    for name, xs in gpu_xs.items():
        e = [a_norm_rel(orc, mats[j], xs[j], r["xs"][j]) for j in range(min(k, len(xs)))]
        err[name] = {"max_a_norm_rel": max(e), "systems": f"1-{k}", "per_system": e}
    return rec, err


def batch_oracle_error(seqs, systems, bs, count=4):
    """A-norm error of the batch's solutions against the FP64 oracle's solve of the same
    sequences (each side recycling its own solutions), on the `count` smallest sequences."""
    from oracle import Oracle, OracleSequence
    orc = Oracle()
    order = sorted(range(len(seqs)), key=lambda i: seqs[i].n)[:count]
    worst = 0.0
    for i in order:
        seq, sy = seqs[i], systems[i]
        X = bs.solutions(i).cpu().numpy()
        oseq = OracleSequence(seq.n, s_max=min(seq.s_max, 16), w_max=seq.w_max, energy=seq.energy, oracle=orc)
        for j, (_, val, b) in enumerate(sy):
            A = (seq.row_ptr, seq.col, val)
            xo, _ = oseq.solve(A, b, seq.tol)
            worst = max(worst, a_norm_rel(orc, A, X[j], xo))
    return {"max_a_norm_rel": worst, "sample": f"the {len(order)} smallest sequences, all systems"}


def kernel_profile(args):
    """A short, fixed launch sequence for kernel profilers: system 1 of the workload (the
    64^3 cantilever with --elasticity) with W seeded random snapshots (so the POD basis
    has about W columns), a solve capped at 5 iterations, then pod_cg_time_kernels.
    Prints the per-kernel times as one JSON line."""
    import torch
    from paper_1512_05820_gb300 import workloads as wl
    from paper_1512_05820_gb300.solver import DeviceCSR, PodCG
    seq = wl.elasticity_cantilever(e=64, p=1) if args.elasticity else wl.diffusion3d_moving(m=args.grid, p=1)
    j, val, b = next(iter(seq.systems()))
    prec = 1 if args.precision == "mixed" else 0
    solver = PodCG(seq.n, w_max=48, s_max=64, energy=0.9999, precision=prec, k_max=5, max_refine=0,
                   loop_mode=1, proj_form={"auto": -1, "direct": 0, "staged": 1}[args.proj_form],
                   spmv_lanes=args.spmv_lanes, bsr=args.bsr)
    snaps = torch.as_tensor(np.random.default_rng(7).normal(size=(seq.n, args.kernel_profile)), device="cuda")
    solver.add_snapshots(snaps)
    A = DeviceCSR.from_numpy(seq.row_ptr, seq.col, val)
    bt = torch.as_tensor(b, device="cuda")
    _, st = solver.solve(A, bt, seq.tol, raise_on_error=False)
    ms = solver.time_kernels(A, bt, reps=args.kernel_reps)
    print(json.dumps({"kernel_profile": True, "workload": "elasticity 64^3" if args.elasticity else f"diffusion {args.grid}^3",
                      "n": seq.n, "nnz": seq.nnz, "bsr": args.bsr, "w": st["w"], "precision": args.precision,
                      "ms": dict(zip(["spmv_cg", "update", "direction", "residual"], ms)),
                      "tuning": solver.tuning()}), flush=True)
    return 0


def stage2_profile(args):
    """A short launch sequence for kernel profilers of stage two (Section 4.2) and of the
    whole-Y stage three (Section 4.3.1): system 1 of the workload, Y seeded random
    snapshots (flat POD spectrum: y = Y, w from energy 0.5), FP64, stage-two tolerance 0 so
    it takes all y - w reduced iterations, stage three capped at 5 iterations, plain
    launches (loop_mode 1). Prints the solve statistics as one JSON line."""
    import torch
    from paper_1512_05820_gb300 import workloads as wl
    from paper_1512_05820_gb300.solver import DeviceCSR, PodCG
    seq = wl.diffusion3d_moving(m=args.grid, p=1)
    j, val, b = next(iter(seq.systems()))
    A = DeviceCSR.from_numpy(seq.row_ptr, seq.col, val)
    bt = torch.as_tensor(b, device="cuda")
    snaps = torch.as_tensor(np.random.default_rng(7).normal(size=(seq.n, args.stage2_profile)), device="cuda")
    out = {"stage2_profile": True, "n": seq.n, "nnz": seq.nnz, "snapshots": args.stage2_profile}
    for mode in (1, 2):
        solver = PodCG(seq.n, w_max=32, s_max=40, energy=0.5, precision=0, k_max=5, max_refine=0, loop_mode=1,
                       three_stage=mode, y_max=min(40, args.stage2_profile), energy_y=1.0 - 1e-12, tol_stage2=0.0,
                       spmv_lanes=args.spmv_lanes)
        solver.add_snapshots(snaps)
        _, st = solver.solve(A, bt, seq.tol, raise_on_error=False)
        torch.cuda.synchronize()
        out[f"three_stage_{mode}"] = {k: st[k] for k in ("status", "y", "w", "stage2_iters", "iters", "inner_iters",
                                                         "ms_stage1", "ms_stage2", "ms_stage3")}
        solver.close()
    print(json.dumps(out), flush=True)
    return 0


GRAM_CASES = [("diffusion3d 128^3 stage one", 2_097_152, 22), ("elasticity 64^3 stage one", 811_200, 48)]


def _gram_inputs(n, w, dtype, seed):
    import torch
    g = torch.Generator(device="cuda").manual_seed(seed)
    X = torch.randn((w, n), generator=g, device="cuda", dtype=torch.float64).to(dtype)
    Y = torch.randn((w, n), generator=g, device="cuda", dtype=torch.float64).to(dtype)
    e = torch.randn(n, generator=g, device="cuda", dtype=torch.float64)
    return X, Y, e


def gram_section(args):
    """Stage-one reduced matrix W^T [AW, b] (n x w panels): the FP64 CUDA-core Gram
    (pod_cg_gram) against the tensor-core split-bf16 Gram (pod_cg_gram_tc) on FP32 and FP64
    panels. Device time per call (CUDA events, median of --kernel-reps after 3 warm-ups),
    algorithmic bytes (each panel element and b read once), HBM and tensor fractions, and
    the TC result's largest error relative to sum_i |w_ia| |y_ic| against the FP64 Gram."""
    import ctypes
    import torch
    from paper_1512_05820_gb300 import _lib
    from paper_1512_05820_gb300.solver import _check as lib_check
    L = _lib.load()
    peak_hbm, _ = peaks()
    peak_tc = measured_bf16_tflops()
    reps = max(3, min(args.kernel_reps, 20))
    out = []
    for name, n, w in GRAM_CASES:
        q = w + 1
        X64, Y64, e = _gram_inputs(n, w, torch.float64, n + w)
        Yb = torch.cat([Y64, e[None, :]], 0).contiguous()
        G64 = torch.empty((w, q), dtype=torch.float64, device="cuda")
        ws = max(int(L.pod_cg_gram_workspace(n, w, q)), int(L.pod_cg_gram_tc_workspace(n, w, q)))
        work = torch.empty(ws, dtype=torch.uint8, device="cuda")
        strm = torch.cuda.current_stream()
        sp = ctypes.c_void_p(strm.cuda_stream)

        def run64():
            lib_check(L.pod_cg_gram(n, X64.data_ptr(), w, Yb.data_ptr(), q, G64.data_ptr(), work.data_ptr(), ws, sp))

        def timed(fn):
            for _ in range(3):
                fn()
            ts = []
            for _ in range(reps):
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record(strm)
                fn()
                b.record(strm)
                b.synchronize()
                ts.append(a.elapsed_time(b))
            return statistics.median(ts)

        ms64 = timed(run64)
        absum = X64.abs() @ Yb.abs().t()
        row = {"case": name, "n": n, "p": w, "q": q,
               "fp64_cuda_cores": {"ms": ms64, "GB/s": (2 * w * n * 8 + 8 * n) / (ms64 / 1e3) / 1e9}}
        for tag, dt, el in (("tc_fp32_panels", torch.float32, 4), ("tc_fp64_panels", torch.float64, 8)):
            X = X64.to(dt).contiguous()
            Y = Y64.to(dt).contiguous()
            Gt = torch.empty((w, q), dtype=torch.float64, device="cuda")

            def runtc():
                lib_check(L.pod_cg_gram_tc(n, el, X.data_ptr(), w, Y.data_ptr(), w, e.data_ptr(), Gt.data_ptr(),
                                           work.data_ptr(), ws, sp))

            ms = timed(runtc)
            run64()
            # the FP64 reference of the FP32-rounded panels, so only the TC arithmetic is measured
            Xr, Yr = X.to(torch.float64), torch.cat([Y.to(torch.float64), e.to(torch.float32).to(torch.float64)[None]])
            lib_check(L.pod_cg_gram(n, Xr.contiguous().data_ptr(), w, Yr.contiguous().data_ptr(), q, G64.data_ptr(),
                                    work.data_ptr(), ws, sp))
            torch.cuda.synchronize()
            err = float(((Gt - G64).abs() / absum).max())
            nbytes = 2 * w * n * el + 8 * n
            pairs = 3 if 3 * w <= 128 else 4
            N = (q + 15) // 16 * 16
            mma_flops = ((n + 31) // 32) * 2 * pairs * 2 * 128 * N * 16
            row[tag] = {"ms": ms, "GB/s": nbytes / (ms / 1e3) / 1e9, "frac_hbm": nbytes / (ms / 1e3) / 1e9 / peak_hbm,
                        "mma_tflops": mma_flops / (ms / 1e3) / 1e12,
                        "frac_tensor": mma_flops / (ms / 1e3) / 1e12 / peak_tc if peak_tc else None,
                        "max_err_rel_abs": err, "speedup_vs_fp64": ms64 / ms}
        out.append(row)
        del X64, Y64, e, Yb, work
    return out


def elasticity_bench(args):
    """The 64^3-element cantilever of trilinear hexahedra (n = 811,200, ~78.5 nonzeros per
    row, w <= 48), its first K systems (seeded, generated on the host): POD-augmented CG in
    mixed precision with the tensor-core split-bf16 stage-one Gram and with the CUDA-core
    FP32 Gram, against plain Jacobi CG in mixed precision, each timed over the K systems
    (CUDA events) after one untimed pass; the CG product in 3x3 block form (the default
    for this pattern) and, for comparison, in CSR. Prints one JSON line."""
    import torch
    from paper_1512_05820_gb300 import workloads as wl
    from paper_1512_05820_gb300.sequence import DeviceSequence, run_sequence
    from paper_1512_05820_gb300.solver import PodCG
    K = args.elasticity
    seq = wl.elasticity_cantilever(e=64, p=K)
    t0 = time.perf_counter()
    systems = seq.all_systems()
    gen_s = time.perf_counter() - t0
    dseq = DeviceSequence(seq, systems=systems)
    xs = [torch.empty(seq.n, dtype=torch.float64, device="cuda") for _ in range(K)]

    def one(recycle, tc, bsr=-1):
        solver = PodCG(seq.n, w_max=seq.w_max, s_max=seq.s_max, energy=seq.energy, precision=1, use_tc_gram=tc,
                       spmv_lanes=args.spmv_lanes, bsr=bsr)
        run_sequence(solver, dseq, xs, recycle=recycle)
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(solver.stream)
        st = run_sequence(solver, dseq, xs, recycle=recycle)
        b.record(solver.stream)
        torch.cuda.synchronize()
        ms = a.elapsed_time(b)
        tun = solver.tuning()
        solver.close()
        return {"systems_per_s": K / (ms / 1e3), "ms": ms, "iters": [s["iters"] for s in st],
                "w": [s["w"] for s in st], "stage1_relres": [s["stage1_relres"] for s in st],
                "ms_stage1_mean": float(np.mean([s["ms_stage1"] for s in st])),
                "max_final_relres": max(s["final_relres"] for s in st), "spmv_lanes": tun["spmv_lanes"]}

    out = {"elasticity": True, "workload": f"elasticity_cantilever 64^3 elements, first {K} systems",
           "n": seq.n, "nnz": seq.nnz, "w_max": seq.w_max, "tol": seq.tol, "generation_s": gen_s,
           "pod_aug_tc_gram": one(True, 1), "pod_aug_cuda_core_gram": one(True, 0), "plain_cg": one(False, 0),
           "pod_aug_tc_gram_csr": one(True, 1, 0), "plain_cg_csr": one(False, 0, 0)}
    out["speedup_pod_aug_vs_plain"] = out["pod_aug_tc_gram"]["systems_per_s"] / out["plain_cg"]["systems_per_s"]
    out["speedup_bsr_vs_csr_pod_aug"] = (out["pod_aug_tc_gram"]["systems_per_s"] /
                                         out["pod_aug_tc_gram_csr"]["systems_per_s"])
    out["speedup_bsr_vs_csr_plain"] = out["plain_cg"]["systems_per_s"] / out["plain_cg_csr"]["systems_per_s"]
    print(json.dumps(out), flush=True)
    return 0


def output_pod_bench(args):
    """The POD metrics of Section 3.3 on one sequence: the identity metric, the output-
    oriented metric C^T C (Q functionals of U[0,1] entries, as in the paper's output
    experiment) and the metric A of each system (also with the three-stage algorithm, whose
    stage two then sees Y^T A Y = I); same precision and tolerance, each timed over the
    sequence (CUDA events) after one untimed pass. Also reports the relative output error ||C (x0 - x)|| / ||C x|| of the
    stage-one iterate x0 (the part the POD metric shapes) for the last system. Prints one
    JSON line."""
    import torch
    from paper_1512_05820_gb300.sequence import DeviceSequence, run_sequence
    from paper_1512_05820_gb300.solver import PodCG, PodCGError
    seq = workload(args)
    prec = 1 if args.precision == "mixed" else 0
    dseq = DeviceSequence(seq, systems=seq.all_systems())
    xs = [torch.empty(seq.n, dtype=torch.float64, device="cuda") for _ in range(dseq.p)]
    gen = torch.Generator(device="cuda").manual_seed(17)
    C = torch.rand((args.output_pod, seq.n), generator=gen, device="cuda", dtype=torch.float64)

    def one(output, **cfg):
        try:
            return one_(output, **cfg)
        except PodCGError as e:   # reported in the line, not fatal to the other variants
            return {"config": dict(cfg), "error": str(e)[:200]}

    def one_(output, **cfg):
        cfg.setdefault("energy", seq.energy)
        solver = PodCG(seq.n, w_max=seq.w_max, s_max=seq.s_max, precision=prec, spmv_lanes=args.spmv_lanes, **cfg)
        if output:
            solver.set_output_functionals(C)
        run_sequence(solver, dseq, xs)
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(solver.stream)
        st = run_sequence(solver, dseq, xs)
        b.record(solver.stream)
        torch.cuda.synchronize()
        ms = a.elapsed_time(b)
        # stage-one iterate of the last system: a solve capped at 0 iterations
        j = dseq.p - 1
        probe = PodCG(seq.n, w_max=seq.w_max, s_max=seq.s_max, energy=cfg["energy"], precision=0, k_max=0,
                      max_refine=0, pod_metric=cfg.get("pod_metric", 0))
        if output:
            probe.set_output_functionals(C)
        for k in range(max(0, j - seq.s_max), j):
            probe.add_snapshots(xs[k])
        x0, _ = probe.solve(dseq.matrix(j), dseq.bs[j], seq.tol, raise_on_error=False)
        out_err = float(torch.linalg.norm(C @ (x0 - xs[j])) / torch.linalg.norm(C @ xs[j]))
        probe.close()
        solver.close()
        return {"systems_per_s": dseq.p / (ms / 1e3), "ms": ms,
                "mean_iters": float(np.mean([s["iters"] for s in st])),
                "mean_w": float(np.mean([s["w"] for s in st])),
                "mean_stage2_iters": float(np.mean([s["stage2_iters"] for s in st])),
                "ms_pod_mean": float(np.mean([s["ms_pod"] for s in st])),
                "last_stage1_relres": st[-1]["stage1_relres"],
                "last_stage1_output_relerr": out_err,
                "max_final_relres": max(s["final_relres"] for s in st)}

    out = {"output_pod": True, "workload": f"diffusion3d_moving {args.grid}^3 7-point, {seq.p} systems",
           "q": args.output_pod, "precision": args.precision, "tol": seq.tol,
           "identity_metric": one(False), "output_metric": one(True), "a_metric": one(False, pod_metric=1),
           "a_metric_three_stage_e099": one(False, pod_metric=1, energy=0.99, three_stage=1, y_max=seq.s_max,
                                            energy_y=0.99999999, tol_stage2=1e-4)}
    base = out["identity_metric"].get("systems_per_s")
    out["speedup_vs_identity"] = {k: out[k]["systems_per_s"] / base
                                  for k in ("output_metric", "a_metric", "a_metric_three_stage_e099")
                                  if base and "systems_per_s" in out[k]}
    print(json.dumps(out), flush=True)
    return 0


def weights_study(seq, systems, tol, p_cap, ks):
    """Section 5's POD-weights experiment on a synthetic sequence: systems 1-10 recycle every
    Krylov vector (the first p_cap directions per system, no compression), Z is compressed
    after system 10 by the A_10-metric POD with the ideal weights (the coordinates of system
    11's solution in Z), the previous weights (those of system 10's) or the RBF weights, to k
    vectors; system 11 is solved with that k-dimensional basis. Reported per k: the relative
    residual before stage three and the stage-three iterations to tol."""
    import torch
    from paper_1512_05820_gb300.solver import DeviceCSR, PodCG
    A0 = DeviceCSR.from_numpy(seq.row_ptr, seq.col, np.zeros(seq.nnz))
    mats = [A0.with_values(torch.as_tensor(v, device="cuda")) for _, v, _ in systems[:11]]
    bs = [torch.as_tensor(b, device="cuda") for _, _, b in systems[:11]]
    out = {"relres_before_stage3": {}, "stage3_iters": {}}
    for kind in ("ideal", "prev", "rbf"):
        rel, its = [], []
        for k in ks:
            h = PodCG(seq.n, three_stage=1, tol_stage2=1e-4)
            h.set_krylov(y_threshold=0, y_keep=min(k, 64), w_keep=min(k, 64), nu=1.0, weights="rbf", p_cap=p_cap)
            for j in range(10):
                h.solve(mats[j], bs[j], tol)
            if kind == "ideal":
                eta, _ = h.krylov_coords(mats[10], bs[10])
            elif kind == "prev":
                eta, _ = h.krylov_coords(mats[9], bs[9])
            else:
                _, eta = h.krylov_coords(mats[9], bs[9])
            z = h.krylov_state()["z"]
            kk = min(k, z)
            h.krylov_compress(mats[9], eta, kk, kk)
            h.set_krylov(y_threshold=0, y_keep=min(k, 64), w_keep=min(k, 64), nu=1.0, weights="rbf", p_cap=p_cap,
                         frozen=True)
            _, st = h.solve(mats[10], bs[10], tol)
            rel.append(st["stage1_relres"])
            its.append(st["iters"])
            h.close()
        out["relres_before_stage3"][kind] = rel
        out["stage3_iters"][kind] = its
    h = PodCG(seq.n, three_stage=1, tol_stage2=1e-4)
    _, st = h.solve(mats[10], bs[10], tol)
    h.close()
    out["k"] = list(ks)
    out["stage3_iters_without_recycling"] = st["iters"]
    out["z_before_compression"] = z
    return out


def krylov_bench(args):
    """The overall algorithm with the paper's own snapshots (Algorithm 3, FP64): systems/s on
    the 128^3 sequence with Krylov-vector snapshots (storage threshold 40, compression to 20,
    W = the first 5 after a compression and every new direction between (nu = 1), RBF
    weights, 24 directions kept per system) against the three-stage method on the POD of
    previous solutions, both end to end on the device; then the POD-weights study."""
    import torch
    from paper_1512_05820_gb300.solver import DeviceCSR, PodCG
    seq = workload(args)
    systems = seq.all_systems()
    A0 = DeviceCSR.from_numpy(seq.row_ptr, seq.col, np.zeros(seq.nnz))
    mats = [A0.with_values(torch.as_tensor(v, device="cuda")) for _, v, _ in systems]
    bs = [torch.as_tensor(b, device="cuda") for _, _, b in systems]
    xs = [torch.empty(seq.n, dtype=torch.float64, device="cuda") for _ in systems]

    def run(kind):
        h = PodCG(seq.n, three_stage=1, w_max=seq.w_max, s_max=seq.s_max, energy=seq.energy, tol_stage2=1e-4)
        if kind == "krylov":
            h.set_krylov(y_threshold=40, y_keep=20, w_keep=5, nu=1.0, weights="rbf", p_cap=24)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        iters, comp = [], 0
        for j in range(len(systems)):
            _, st = h.solve(mats[j], bs[j], seq.tol, x_out=xs[j])
            if kind != "krylov":
                h.add_snapshots(xs[j])
            iters.append(st["iters"])
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        if kind == "krylov":
            comp = h.krylov_state()["compressions"]
        h.close()
        rel = max(float(torch.linalg.norm(bs[j] - spmv_dev(mats[j], xs[j])) / torch.linalg.norm(bs[j]))
                  for j in range(len(systems)))
        return {"systems_per_s": len(systems) / (ms / 1e3), "mean_iters": float(np.mean(iters)),
                "iters_first": iters[0], "iters_last": iters[-1], "max_final_relres": rel,
                **({"compressions": comp} if kind == "krylov" else {})}

    res = {"krylov_vectors": run("krylov"), "pod_of_solutions": run("solutions")}
    wseq = wl_weights_workload()
    wsys = wseq.all_systems()
    study = weights_study(wseq, wsys, 1e-6, 6, [1, 2, 4, 8, 12, 16, 24, 32, 40, 48, 60])
    study["workload"] = f"{wseq.name} n = {wseq.n}, first 11 systems, 6 directions kept per system, tol 1e-6"
    line = {"metric": "systems/s, Krylov-vector snapshots (Algorithm 3) vs POD of previous solutions, FP64",
            "unit": "systems/s", "value": res["krylov_vectors"]["systems_per_s"], "higher_is_better": True,
            "config": {"workload": f"diffusion3d_moving {args.grid}^3 7-point, {seq.p} systems", "n": seq.n,
                       "tol": seq.tol, "precision": "fp64", "three_stage": 1},
            "data": "synthetic", **res, "weights_study": study}
    print(json.dumps(line))


def spmv_dev(A, x):
    from paper_1512_05820_gb300.solver import spmv
    return spmv(A, x)


def wl_weights_workload():
    from paper_1512_05820_gb300 import workloads as wl
    return wl.elasticity_cantilever(e=16, p=11)


def three_stage_bench(args):
    """Three-stage solves (stage one on the dominant POD modes, stage two over all retained
    modes, stage three augmented with [W, V2]) against the two-stage form (stage one on the
    POD basis at energy 0.9999, then stage three), same sequence, same precision and
    tolerance. Each variant is timed over the whole sequence (CUDA events) after one
    untimed pass. Prints one JSON line."""
    import torch
    from paper_1512_05820_gb300 import workloads as wl
    from paper_1512_05820_gb300.sequence import DeviceSequence, run_sequence
    from paper_1512_05820_gb300.solver import PodCG
    if args.elasticity:
        seq = wl.elasticity_cantilever(e=64, p=args.elasticity)
        name = f"elasticity_cantilever 64^3 elements, first {args.elasticity} systems"
    else:
        seq = workload(args)
        name = f"diffusion3d_moving {args.grid}^3 7-point, {seq.p} systems"
    prec = 1 if args.precision == "mixed" else 0
    dseq = DeviceSequence(seq, systems=seq.all_systems())
    xs = [torch.empty(seq.n, dtype=torch.float64, device="cuda") for _ in range(dseq.p)]

    def one(**cfg):
        solver = PodCG(seq.n, w_max=seq.w_max, s_max=seq.s_max, precision=prec, spmv_lanes=args.spmv_lanes,
                       use_tc_gram=1 if prec == 1 else 0, **cfg)
        run_sequence(solver, dseq, xs)
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(solver.stream)
        st = run_sequence(solver, dseq, xs)
        b.record(solver.stream)
        torch.cuda.synchronize()
        ms = a.elapsed_time(b)
        solver.close()
        return {"config": {k: v for k, v in cfg.items()}, "systems_per_s": dseq.p / (ms / 1e3), "ms": ms,
                "mean_iters_stage3": float(np.mean([s["iters"] for s in st])),
                "mean_stage2_iters": float(np.mean([s["stage2_iters"] for s in st])),
                "mean_w_stage3": float(np.mean([s["w"] for s in st])),
                "mean_y": float(np.mean([s["y"] for s in st])),
                "ms_stage1_mean": float(np.mean([s["ms_stage1"] for s in st])),
                "ms_stage2_mean": float(np.mean([s["ms_stage2"] for s in st])),
                "ms_stage3_mean": float(np.mean([s["ms_stage3"] for s in st])),
                "spmv_total": int(sum(s["spmv_count"] for s in st)),
                "_inner": float(np.mean([s["inner_iters"] for s in st])),
                "max_final_relres": max(s["final_relres"] for s in st)}

    out = {"three_stage": True, "workload": name, "n": seq.n, "nnz": seq.nnz, "tol": seq.tol,
           "precision": args.precision, "s_max": seq.s_max,
           "two_stage": one(energy=seq.energy),
           "three_stage_e099_all_modes": one(energy=0.99, three_stage=1, y_max=seq.s_max, energy_y=0.99999999,
                                             tol_stage2=1e-4),
           "three_stage_e0999_all_modes": one(energy=0.999, three_stage=1, y_max=seq.s_max, energy_y=0.99999999,
                                              tol_stage2=1e-4),
           "three_stage_e09999_all_modes": one(energy=seq.energy, three_stage=1, y_max=seq.s_max,
                                               energy_y=0.99999999, tol_stage2=1e-4)}
    if prec == 0:   # stage three over the whole Y (Section 4.3.1) runs in FP64 only
        out["three_stage_full_y_e099"] = one(energy=0.99, three_stage=2, y_max=seq.s_max, energy_y=0.99999999,
                                             tol_stage2=1e-4)
        out["three_stage_full_y_e099"]["mean_inner_iters"] = out["three_stage_full_y_e099"].pop("_inner", 0.0)
    base = out["two_stage"]["systems_per_s"]
    for v in out.values():
        if isinstance(v, dict):
            v.pop("_inner", None)
    out["speedup_vs_two_stage"] = {k: v["systems_per_s"] / base for k, v in out.items()
                                   if isinstance(v, dict) and k.startswith("three_stage_")}
    print(json.dumps(out), flush=True)
    return 0


def gram_profile(args):
    """A short launch sequence for kernel profilers: the tensor-core Gram of the 128^3
    stage-one shape (FP32 W and AW panels, w = 22, plus b), --kernel-reps launches."""
    import ctypes
    import torch
    from paper_1512_05820_gb300 import _lib
    from paper_1512_05820_gb300.solver import _check as lib_check
    L = _lib.load()
    n, w = GRAM_CASES[0][1], GRAM_CASES[0][2]
    X, Y, e = _gram_inputs(n, w, torch.float32, 11)
    G = torch.empty((w, w + 1), dtype=torch.float64, device="cuda")
    ws = int(L.pod_cg_gram_tc_workspace(n, w, w + 1))
    work = torch.empty(ws, dtype=torch.uint8, device="cuda")
    sp = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    for _ in range(args.kernel_reps):
        lib_check(L.pod_cg_gram_tc(n, 4, X.data_ptr(), w, Y.data_ptr(), w, e.data_ptr(), G.data_ptr(),
                                   work.data_ptr(), ws, sp))
    torch.cuda.synchronize()
    print(json.dumps({"gram_profile": True, "n": n, "w": w, "finite": bool(torch.isfinite(G).all())}), flush=True)
    return 0


def diff_check(args):
    """Loss L = sum_j c^T x_j over the 96^3 sequence A_j(theta) x_j = b_j (20 systems,
    theta ~ N(0, 0.5^2) per cell): gradient by the adjoint path (forward solves with
    recycling, adjoint solves reusing each W_j, fused edge-wise kernel) against the
    fourth-order central difference (h = 1e-3) at K seeded random cells; solves at 1e-13.
    Reports the error norm-wise over the sampled cells (||g_fd - g||/||g||), as the largest
    error relative to the largest sampled |g|, and per cell (max and median of
    |g_fd - g|/|g|; cells with small |g| carry the finite-difference noise)."""
    import torch
    from paper_1512_05820_gb300 import workloads as wl
    from paper_1512_05820_gb300.adjoint import DiffusionProblem, solve_sequence
    seq = wl.diffusion3d_theta(m=96, p=20)
    r = seq.recipe
    shifts = np.stack([0.01 * (j + 1) * r["u"] for j in range(seq.p)])
    B = torch.as_tensor(np.stack([b for _, _, b in seq.systems()]), device="cuda")
    c = torch.as_tensor(r["c"], device="cuda")
    prob = DiffusionProblem.from_operator(seq.op, shifts=shifts, tol=1e-13, w_max=32, s_max=40)
    th = torch.as_tensor(r["theta"], device="cuda").requires_grad_(True)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    X = solve_sequence(th, B, prob)
    loss = (X * c).sum()
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    loss.backward()
    torch.cuda.synchronize()
    t2 = time.perf_counter()
    g = th.grad.cpu().numpy()

    def L(theta):
        with torch.no_grad():
            Xp = solve_sequence(torch.as_tensor(theta, device="cuda"), B, prob)
            return float((Xp * c).sum())

    rng = np.random.default_rng(5)
    cells = rng.choice(seq.n, size=args.diff_check, replace=False)
    th0 = r["theta"]
    h = 1e-3
    fds = []
    for cc in cells:
        e = np.zeros(seq.n)
        e[cc] = h
        fds.append((-L(th0 + 2 * e) + 8 * L(th0 + e) - 8 * L(th0 - e) + L(th0 - 2 * e)) / (12 * h))
    fds = np.array(fds)
    gs = g[cells]
    errs = np.abs(fds - gs) / np.maximum(np.abs(gs), 1e-300)
    print(json.dumps({"diff_check": True, "workload": "diffusion3d_theta 96^3, 20 systems", "cells": len(cells),
                      "solve_tol": 1e-13, "h": h,
                      "normwise_rel_err": float(np.linalg.norm(fds - gs) / np.linalg.norm(gs)),
                      "max_err_over_max_abs_g": float(np.max(np.abs(fds - gs)) / np.max(np.abs(gs))),
                      "max_rel_err": float(errs.max()), "median_rel_err": float(np.median(errs)),
                      "abs_g_range": [float(np.abs(gs).min()), float(np.abs(gs).max())],
                      "forward_s": t1 - t0, "backward_s": t2 - t1, "loss": float(loss)}), flush=True)
    return 0


def main():
    args = parse_args()
    rank, world, local = dist_env()
    if args.impl == "reference":
        return run_reference(args, rank, world)
    if args.kernel_profile:
        return kernel_profile(args)
    if args.diff_check:
        return diff_check(args)
    if args.gram_profile:
        return gram_profile(args)
    if args.stage2_profile:
        return stage2_profile(args)
    if args.three_stage:
        return three_stage_bench(args)
    if args.output_pod:
        return output_pod_bench(args)
    if args.elasticity:
        return elasticity_bench(args)
    if args.krylov:
        return krylov_bench(args)
    if args.batch_profile:
        return batch_profile(args)

    import torch
    from paper_1512_05820_gb300.sequence import DeviceSequence, run_sequence
    from paper_1512_05820_gb300.solver import PodCG

    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")

    prec = 1 if args.precision == "mixed" else 0
    seq = workload(args)
    systems = seq.all_systems()
    dseq = DeviceSequence(seq, systems=systems)
    xs = [torch.empty(seq.n, dtype=torch.float64, device="cuda") for _ in range(dseq.p)]
    loop_mode = {"graph": 0, "chunked": 1, "persistent": 2}[args.loop_mode]
    wsel = 1 if args.w_select == "cost" else 0
    solver = PodCG(seq.n, w_max=seq.w_max, s_max=seq.s_max, energy=seq.energy, precision=prec, loop_mode=loop_mode,
                   proj_form={"auto": -1, "direct": 0, "staged": 1}[args.proj_form], spmv_lanes=args.spmv_lanes,
                   w_select=wsel)
    stream = solver.stream

    def barrier():
        if dist is not None:
            dist.barrier()

    # the first pass carries every one-time tuning of the handle (SpMV lanes, projection forms,
    # the cost-tuned basis cap); it is timed on its own and reported beside the steps
    first_ms = None
    for k in range(args.warmup):
        if k == 0:
            torch.cuda.synchronize()
            f0 = time.perf_counter()
        run_sequence(solver, dseq, xs)
        if k == 0:
            torch.cuda.synchronize()
            first_ms = (time.perf_counter() - f0) * 1e3
    torch.cuda.synchronize()
    barrier()
    torch.cuda.synchronize()
    sampler = ClockSampler(local)
    sampler.start()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    all_stats = []
    for _ in range(args.steps):
        all_stats.append(run_sequence(solver, dseq, xs))
    e1.record(stream)
    torch.cuda.synchronize()
    barrier()
    torch.cuda.synchronize()
    clocks = sampler.stop()
    from paper_1512_05820_gb300.dist import combine
    # the GPU's solutions of the first systems, for the error against the FP64 oracle
    gpu_xs = {("mixed" if prec == 1 else "fp64"): [xs[j].cpu().numpy() for j in range(CPU_PREFIX)]}
    ms_total, systems_done = combine(e0.elapsed_time(e1), float(seq.p * args.steps))
    ms_step = ms_total / args.steps
    value = systems_done / (ms_total / 1e3)
    last = all_stats[-1]
    spmv_per_step = sum(s["spmv_count"] for s in last)
    bsp = b_spmv(seq.n, seq.nnz)
    spmv_gbs = world * spmv_per_step * bsp / (ms_step / 1e3) / 1e9
    launches = sum(s["launches"] + 3 for st in all_stats for s in st)   # + add_snapshots (3 kernels)
    iters = [s["iters"] for s in last]
    ws = [s["w"] for s in last]

    batch_out = None
    if not args.no_batch:   # every rank takes part (sequences shard across ranks)
        try:
            batch_out = batch_section(args, rank, world)
        except Exception as e:  # reported, not fatal to the headline measurement
            batch_out = {"error": repr(e)[:300]}

    if rank != 0:
        if dist is not None:
            dist.destroy_process_group()
        return 0

    out = {"metric": METRIC, "value": value, "unit": "systems/s", "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f64" if prec == 0 else "f32+f64", "data": "synthetic",
           "config": config_dict(seq, args, args.precision),
           "spmv_equiv_gbs": spmv_gbs,
           "pod_aug": {"systems_per_s": value, "mean_iters": float(np.mean(iters)), "iters_first": iters[0],
                       "iters_last": iters[-1], "mean_w": float(np.mean(ws)),
                       "max_final_relres": max(s["final_relres"] for s in last),
                       "ms_pod_mean": float(np.mean([s["ms_pod"] for s in last])),
                       "ms_stage1_mean": float(np.mean([s["ms_stage1"] for s in last])),
                       "ms_stage2_mean": float(np.mean([s["ms_stage2"] for s in last])),
                       "ms_stage3_mean": float(np.mean([s["ms_stage3"] for s in last])),
                       "spmv_per_step": spmv_per_step,
                       "stage_one_gram_tensor_core_solves": sum(1 for s in last if s.get("gram_tc")),
                       "first_pass_systems_per_s": (seq.p / (first_ms / 1e3)) if first_ms else None}}

    # one timed pass each: POD-aug in the other precision, plain Jacobi CG (no recycling)
    # in both precisions, same GPU, same tolerance
    def one_pass(precision, recycle, w_select=0):
        sv = PodCG(seq.n, w_max=seq.w_max, s_max=seq.s_max, energy=seq.energy, precision=precision,
                   loop_mode=loop_mode, w_select=w_select)
        run_sequence(sv, dseq, xs, recycle=recycle)
        torch.cuda.synchronize()
        a0 = torch.cuda.Event(enable_timing=True)
        a1 = torch.cuda.Event(enable_timing=True)
        a0.record(sv.stream)
        pst = run_sequence(sv, dseq, xs, recycle=recycle)
        a1.record(sv.stream)
        torch.cuda.synchronize()
        pms = a0.elapsed_time(a1)
        sv.close()
        if recycle and w_select == wsel:
            gpu_xs["mixed" if precision == 1 else "fp64"] = [xs[j].cpu().numpy() for j in range(CPU_PREFIX)]
        return {"systems_per_s": seq.p / (pms / 1e3), "ms_per_step": pms,
                "mean_iters": float(np.mean([s["iters"] for s in pst])),
                "mean_w": float(np.mean([s["w"] for s in pst])),
                "spmv_equiv_gbs": sum(s["spmv_count"] for s in pst) * bsp / (pms / 1e3) / 1e9,
                "max_final_relres": max(s["final_relres"] for s in pst)}

    if not args.no_compare:
        other = 0 if prec == 1 else 1
        out["pod_aug_" + ("fp64" if other == 0 else "mixed")] = one_pass(other, True, wsel)
        if wsel:   # the paper's rule alone (Algorithm 4 step 3), same precision
            out["pod_aug_energy_rule"] = one_pass(prec, True, 0)
        out["plain_cg_fp64"] = one_pass(0, False)
        out["plain_cg_mixed"] = one_pass(1, False)
        same = out["plain_cg_mixed" if prec == 1 else "plain_cg_fp64"]
        out["speedup_vs_plain_cg_same_precision"] = value / world / same["systems_per_s"]
        out["speedup_vs_fp64_pod_aug"] = (value / world / out["pod_aug_fp64"]["systems_per_s"]) if prec == 1 else 1.0

    # per-kernel device times of one stage-three iteration (CUDA events, launching stream)
    j_last = dseq.p - 1
    run_sequence(solver, dseq, xs)
    ms_k = solver.time_kernels(dseq.matrix(j_last), dseq.bs[j_last], reps=args.kernel_reps)
    w_meas = solver.last_w
    out["autotune"] = solver.tuning()
    n, nnz = seq.n, seq.nnz
    # algorithmic bytes per launch (each datum once): FP64 or FP32 vectors/panels
    e = 4 if prec == 1 else 8
    # the direction pass of a two-stage mixed solve (either form) reads the 16-bit copy of W
    e_w = 2 if prec == 1 else e
    kbytes = {"spmv_cg": b_spmv(n, nnz, fp32=(prec == 1)),
              "update": 4 * e * n + e * w_meas * n,          # read r, q, dinv, AW; write r
              "direction": 6 * e * n + e_w * w_meas * n,     # read x, p, r, dinv, W; write x, p
              "residual": b_spmv(n, nnz) + 16 * n}           # FP64 always; + read b, write r
    kms = dict(zip(["spmv_cg", "update", "direction", "residual"], ms_k))
    it_total = sum(iters)
    share = {k: kms[k] * it_total for k in ("spmv_cg", "update", "direction")}
    dominant = max(share, key=share.get)
    peak, peak_kind = peaks()
    achieved = kbytes[dominant] / (kms[dominant] / 1e3) / 1e9
    # FP32 with a basis runs the projection form the handle timed for the bucket
    wb = next(b for b in (0, 8, 16, 32, 48, 64) if w_meas <= b)
    rec = out["autotune"].get("projection", {}).get(f"w<={wb}", {})

    def suffix(p):
        if prec != 1:
            return ""
        return "_tma" if (w_meas > 0 and rec.get(p) == "staged") else "_v4"
    names = {"spmv_cg": "k_spmv_cg", "update": "k_update" + suffix("update"), "direction": "k_dir" + suffix("direction"),
             "residual": "k_residual"}
    out["roofline"] = {"bound": "hbm", "kernel": names[dominant], "achieved": achieved, "peak": peak, "unit": "GB/s",
                       "frac": achieved / peak, "peak_source": peak_kind,
                       "traffic": traffic_from_profiles(names[dominant], "mixed" if prec == 1 else "fp64", w_meas),
                       "algorithmic_bytes_per_launch": kbytes[dominant], "w": w_meas,
                       "ms_per_launch": kms[dominant]}
    # the FP32 inner loop as one persistent launch per refinement step (bases up to 8 wide):
    # it is then the dominant kernel; its device time comes from the kernel's own timer and
    # its algorithmic bytes are those of every inner iteration it ran (CG product 8 nnz +
    # 4(n+1) + 8n, update 16n + 4wn, direction 24n + 4wn: x, p, r, M^{-1} read, x, p written,
    # W in FP32)
    loop_ms = sum(s["ms_loop"] for s in last)
    if loop_ms > 0:
        it_loop = sum(s["iters"] for s in last if s["ms_loop"] > 0)
        loop_bytes = sum(s["iters"] * (8 * nnz + 4 * (n + 1) + 48 * n + 8 * s["w"] * n) for s in last
                         if s["ms_loop"] > 0)
        ach = loop_bytes / (loop_ms / 1e3) / 1e9
        out["roofline_three_kernel_form"] = out["roofline"]
        out["roofline"] = {"bound": "hbm", "kernel": "k_cg_loop", "achieved": ach, "peak": peak, "unit": "GB/s",
                           "frac": ach / peak, "peak_source": peak_kind,
                           "traffic": traffic_from_profiles("k_cg_loop", "mixed", 4),
                           "algorithmic_bytes_per_iteration_mean": loop_bytes / it_loop,
                           "us_per_iteration": loop_ms * 1e3 / it_loop, "iterations": it_loop,
                           "ms_in_loop_launches": loop_ms}
    out["kernels"] = {k: {"ms": kms[k], "GB/s": kbytes[k] / (kms[k] / 1e3) / 1e9,
                          "frac_hbm": kbytes[k] / (kms[k] / 1e3) / 1e9 / peak} for k in kms}

    # end to end through the public API from pinned host buffers
    if not args.no_e2e:
        import torch as T
        h_vals = [T.as_tensor(v).pin_memory() for _, v, _ in systems]
        h_bs = [T.as_tensor(b).pin_memory() for _, _, b in systems]
        h_rp = T.as_tensor(seq.row_ptr).pin_memory()
        h_col = T.as_tensor(seq.col).pin_memory()
        h_xs = [T.empty(seq.n, dtype=T.float64).pin_memory() for _ in range(dseq.p)]
        d_val = T.empty(seq.nnz, dtype=T.float64, device="cuda")
        d_b = T.empty(seq.n, dtype=T.float64, device="cuda")
        d_rp = T.empty_like(h_rp, device="cuda")
        d_col = T.empty_like(h_col, device="cuda")
        from paper_1512_05820_gb300.solver import DeviceCSR

        def e2e_step():
            solver.clear_snapshots()
            with T.cuda.stream(stream):
                d_rp.copy_(h_rp, non_blocking=True)
                d_col.copy_(h_col, non_blocking=True)
                A = DeviceCSR(d_rp, d_col, d_val)
                for j in range(dseq.p):
                    d_val.copy_(h_vals[j], non_blocking=True)
                    d_b.copy_(h_bs[j], non_blocking=True)
                    x, _ = solver.solve(A, d_b, seq.tol, x_out=xs[j])
                    solver.add_snapshots(x)
                    h_xs[j].copy_(x, non_blocking=True)
            T.cuda.synchronize()

        e2e_step()
        t0 = time.perf_counter()
        e2e_step()
        dt = time.perf_counter() - t0
        h2d = 4 * (seq.n + 1) + 4 * seq.nnz + dseq.p * (8 * seq.nnz + 8 * seq.n)
        d2h = dseq.p * 8 * seq.n
        out["e2e"] = {"value": world * seq.p / dt, "unit": "systems/s", "h2d_bytes_per_step": h2d,
                      "d2h_bytes_per_step": d2h}

    if not args.no_gram:
        out["stage_one_gram"] = gram_section(args)
    if batch_out is not None:
        out["batch"] = batch_out
    out["gpu_launches"] = launches
    out["clocks"] = clocks
    if world == 1 and not args.no_cpu_baseline:
        out["cpu_baseline"], out["err_vs_fp64_oracle"] = cpu_baseline(args, seq, gpu_xs)
    # the comparison the metric names, last on the line (a reader of the line's tail sees it)
    for key in ("pod_aug_fp64", "pod_aug_mixed", "pod_aug_energy_rule", "plain_cg_mixed", "plain_cg_fp64",
                "speedup_vs_plain_cg_same_precision", "speedup_vs_fp64_pod_aug", "err_vs_fp64_oracle"):
        if key in out:
            out[key] = out.pop(key)
    if batch_out is not None and "err_vs_fp64_oracle" in batch_out:
        out["batch_err_vs_fp64_oracle"] = batch_out["err_vs_fp64_oracle"]
    n_tc = out["pod_aug"]["stage_one_gram_tensor_core_solves"]
    out["headline"] = {"pod_aug_" + ("mixed" if prec == 1 else "fp64"): value, "roofline_frac": out["roofline"]["frac"],
                       "roofline_kernel": out["roofline"]["kernel"],
                       "stage_one_gram": f"tensor cores (split bf16) in {n_tc} of {seq.p} solves, CUDA cores in the rest",
                       "w_cap": out["autotune"].get("w_cap", {}).get("cap")}
    if "plain_cg_mixed" in out and prec == 1:
        out["headline"]["vs_plain_cg_mixed"] = value / world / out["plain_cg_mixed"]["systems_per_s"]
    print(json.dumps(out), flush=True)
    if dist is not None:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
