"""Writes the FP64 oracle's records of the 64x64 five-point sequence (10 systems, w <= 8,
tol 1e-8; the synthetic stand-in described in the workloads module):
c1_sequence_oracle.json (two stages), c1_three_stage_oracle.json (three stages),
c1_output_pod_oracle.json (POD in the metric C^T C of 12 seeded U[0, 1] functionals) and
c1_metric_a_oracle.json (POD in the metric A of the system being solved). Calls only the
oracle and the seeded input generators.

The paper prints no numeric worked example (its results are figures), so no fixture here
holds a value printed in the paper; this one is a regression record of the oracle itself,
pinned independently by the closed forms and invariants in tests/pins.py.

Run from the repository root:  python tests/golden/make_golden.py
"""
import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import Oracle, OracleSequence  # noqa: E402
from paper_1512_05820_gb300 import workloads as wl  # noqa: E402


def output_functionals(n: int, q: int = 12, seed: int = 1240) -> np.ndarray:
    """q functionals with U[0, 1] entries (the paper's output experiment), (q, n)."""
    return np.random.default_rng(seed).uniform(0.0, 1.0, size=(q, n))


def record(three_stage: bool = False, metric: str = "identity"):
    """The two-stage record, or (three_stage) the three-stage one: stage-one energy 0.99,
    the augmenting basis all modes to energy 1 - 1e-10 (y <= 8), stage-two tolerance 1e-4.
    metric: "identity", "output" (C^T C) or "a" (the system's A), two stages."""
    seq = wl.diffusion2d_drift()
    orc = Oracle()
    extra = {}
    energy = seq.energy
    if three_stage:
        energy = 0.99
        extra = dict(three_stage=True, y_max=seq.s_max, energy_y=1 - 1e-10, tol_stage2=1e-4)
    if metric == "output":
        extra["C"] = output_functionals(seq.n)
    elif metric == "a":
        extra["metric_a"] = True
    oseq = OracleSequence(seq.n, s_max=seq.s_max, w_max=seq.w_max, energy=energy, oracle=orc, **extra)
    out = []
    for j, val, b in seq.systems():
        x, info = oseq.solve((seq.row_ptr, seq.col, val), b, seq.tol)
        rec = {"system": j, "iters": info["iters"], "w": info["w"], "refinements": info["refinements"],
               "stage1_relres": info["stage1_relres"], "final_relres": info["final_relres"],
               "x_norm2": float(np.linalg.norm(x)), "x_sum": float(np.sum(x))}
        if three_stage:
            rec.update({"k2": info["k2"], "y": info["y"], "stage2_relres": info["stage2_relres"]})
        out.append(rec)
    wl_name = (f"diffusion2d_drift 64x64, {seq.p} systems, w_max {seq.w_max}, s_max {seq.s_max}, "
               f"energy {energy}, tol {seq.tol}")
    if three_stage:
        wl_name += ", three stages (energy_y 1 - 1e-10, tol_stage2 1e-4)"
    if metric == "output":
        wl_name += ", POD metric C^T C (12 U[0, 1] functionals, seed 1240)"
    elif metric == "a":
        wl_name += ", POD metric A"
    return {"workload": wl_name, "source": "oracle/ (FP64 C), written by tests/golden/make_golden.py",
            "systems": out}


if __name__ == "__main__":
    here = os.path.dirname(os.path.abspath(__file__))
    with open(os.path.join(here, "c1_sequence_oracle.json"), "w") as f:
        json.dump(record(), f, indent=1)
    with open(os.path.join(here, "c1_three_stage_oracle.json"), "w") as f:
        json.dump(record(three_stage=True), f, indent=1)
    with open(os.path.join(here, "c1_output_pod_oracle.json"), "w") as f:
        json.dump(record(metric="output"), f, indent=1)
    with open(os.path.join(here, "c1_metric_a_oracle.json"), "w") as f:
        json.dump(record(metric="a"), f, indent=1)
