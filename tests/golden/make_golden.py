"""Writes tests/golden/c1_sequence_oracle.json: the FP64 oracle's record of the 64x64
five-point sequence (10 systems, w <= 8, tol 1e-8; the synthetic stand-in described in
the workloads module). Calls only the oracle and the seeded input generator.

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


def record():
    seq = wl.diffusion2d_drift()
    orc = Oracle()
    oseq = OracleSequence(seq.n, s_max=seq.s_max, w_max=seq.w_max, energy=seq.energy, oracle=orc)
    out = []
    for j, val, b in seq.systems():
        x, info = oseq.solve((seq.row_ptr, seq.col, val), b, seq.tol)
        out.append({"system": j, "iters": info["iters"], "w": info["w"], "refinements": info["refinements"],
                    "stage1_relres": info["stage1_relres"], "final_relres": info["final_relres"],
                    "x_norm2": float(np.linalg.norm(x)), "x_sum": float(np.sum(x))})
    return {"workload": f"diffusion2d_drift 64x64, {seq.p} systems, w_max {seq.w_max}, s_max {seq.s_max}, "
                        f"energy {seq.energy}, tol {seq.tol}",
            "source": "oracle/ (FP64 C), written by tests/golden/make_golden.py", "systems": out}


if __name__ == "__main__":
    with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "c1_sequence_oracle.json"), "w") as f:
        json.dump(record(), f, indent=1)
