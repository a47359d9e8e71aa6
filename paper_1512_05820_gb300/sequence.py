"""Sequence driver on the GPU: the recycled-solution form of the paper's overall
algorithm (Section 4.4, Algorithm 3) — solve system j with the POD basis of the last
s_max solutions, then add its solution to the snapshots."""
from __future__ import annotations

import numpy as np
import torch

from .solver import DeviceCSR, PodCG


class DeviceSequence:
    """All systems of a workload resident on the GPU: one sparsity pattern, p value
    arrays and p right-hand sides."""

    def __init__(self, seq, device="cuda", systems=None):
        self.seq = seq
        self.n, self.nnz, self.p, self.tol = seq.n, seq.nnz, seq.p, seq.tol
        systems = systems if systems is not None else seq.all_systems()
        self.pattern = DeviceCSR.from_numpy(seq.row_ptr, seq.col, np.zeros(0), device=device)
        self.vals = [torch.as_tensor(v, device=device) for _, v, _ in systems]
        self.bs = [torch.as_tensor(b, device=device) for _, _, b in systems]
        self.p = len(self.vals)

    def matrix(self, j: int) -> DeviceCSR:
        return self.pattern.with_values(self.vals[j])


def run_sequence(solver: PodCG, dseq: DeviceSequence, xs: list[torch.Tensor] | None = None,
                 recycle: bool = True, tol: float | None = None):
    """Solve every system in order. With recycle=False no snapshot is recorded (plain
    Jacobi PCG for every system). Returns the list of per-system stats."""
    solver.clear_snapshots()
    tol = dseq.tol if tol is None else tol
    out = []
    for j in range(dseq.p):
        x = xs[j] if xs is not None else None
        x, st = solver.solve(dseq.matrix(j), dseq.bs[j], tol, x_out=x)
        if recycle:
            solver.add_snapshots(x)
        out.append(st)
    return out
