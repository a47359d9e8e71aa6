"""Differentiation through a sequence of POD-augmented solves (torch.autograd).

``SequenceSolve.apply(theta, B, problem)`` returns X with X[j] = A_j(theta)^{-1} B[j] for
the diffusion operator A_j(theta) = A(exp(theta)) + diag(shift_j). Forward: the matrices
are assembled on the GPU, the systems solved in order with POD recycling, and the solutions
X are checkpointed (the only per-system state kept). Backward, for an incoming gradient
G = dL/dX: adjoint solves A_j lambda_j = G[j] with the recycled basis of system j (A_j is
symmetric), then one fused edge-wise pass dL/dtheta = -sum_j lambda_j^T (dA_j/dtheta) x_j;
dL/dB[j] = lambda_j. With ``problem.checkpoint`` (the default) the backward recomputes
W_j, A_j W_j and the stage-one factor from the checkpointed solutions: W_j is the POD of
the same snapshot set the forward solve of system j used (the solutions before it, at most
s_max), so memory stays at X. Without it the forward handle keeps every system's W_j,
A_j W_j and stage-one Gram (pod_cg_solve_adjoint). All arithmetic runs in the library's
kernels; torch holds the tensors.
"""
from __future__ import annotations

import ctypes
from dataclasses import dataclass

import torch

from . import _lib
from .solver import DeviceCSR, PodCG, _check, _stream_ptr


@dataclass
class DiffusionProblem:
    """Grid (mx, my, mz) with the CSR pattern of the finite-volume operator, per-system
    diagonal shifts (p, n) or None, and the solve tolerance."""
    shape: tuple
    row_ptr: torch.Tensor
    col: torch.Tensor
    shifts: torch.Tensor | None
    tol: float = 1e-10
    w_max: int = 32
    s_max: int = 40
    energy: float = 0.9999
    checkpoint: bool = True

    @property
    def n(self) -> int:
        return self.row_ptr.numel() - 1

    @classmethod
    def from_operator(cls, op, shifts=None, device="cuda", **kw):
        mz, my, mx = op.shape3
        sh = torch.as_tensor(shifts, dtype=torch.float64, device=device) if shifts is not None else None
        return cls((mx, my, mz), torch.as_tensor(op.row_ptr, device=device), torch.as_tensor(op.col, device=device),
                   sh, **kw)


def assemble(problem: DiffusionProblem, theta: torch.Tensor, j: int, out: torch.Tensor | None = None):
    """CSR values of A_j(theta) on the GPU (pod_cg_diffusion_assemble)."""
    L = _lib.load()
    mx, my, mz = problem.shape
    if out is None:
        out = torch.empty(problem.col.numel(), dtype=torch.float64, device=theta.device)
    extra = problem.shifts[j] if problem.shifts is not None else None
    _check(L.pod_cg_diffusion_assemble(mx, my, mz, theta.data_ptr(), extra.data_ptr() if extra is not None else None,
                                       problem.row_ptr.data_ptr(), out.data_ptr(),
                                       ctypes.c_void_p(_stream_ptr(None))))
    return out


def theta_grad(problem: DiffusionProblem, theta: torch.Tensor, lambdas: torch.Tensor, xs: torch.Tensor,
               grad: torch.Tensor | None = None):
    """grad -= sum_j lambda_j^T (dA/dtheta) x_j (pod_cg_diffusion_theta_grad)."""
    L = _lib.load()
    mx, my, mz = problem.shape
    if grad is None:
        grad = torch.zeros_like(theta)
    lambdas, xs = lambdas.contiguous(), xs.contiguous()
    _check(L.pod_cg_diffusion_theta_grad(mx, my, mz, theta.data_ptr(), lambdas.shape[0], lambdas.data_ptr(),
                                         xs.data_ptr(), grad.data_ptr(), ctypes.c_void_p(_stream_ptr(None))))
    return grad


class SequenceSolve(torch.autograd.Function):
    @staticmethod
    def forward(ctx, theta, B, problem: DiffusionProblem):
        theta = theta.detach().contiguous()
        p, n = B.shape
        keep = 0 if problem.checkpoint else p
        solver = PodCG(n, w_max=problem.w_max, s_max=problem.s_max, energy=problem.energy, keep_factors=keep)
        val = torch.empty(problem.col.numel(), dtype=torch.float64, device=B.device)
        X = torch.empty_like(B)
        sysids = []
        for j in range(p):
            assemble(problem, theta, j, out=val)
            A = DeviceCSR(problem.row_ptr, problem.col, val)
            x, st = solver.solve(A, B[j].contiguous(), problem.tol, x_out=X[j])
            solver.add_snapshots(x)
            sysids.append(st["system_id"])
        ctx.save_for_backward(theta, X)
        ctx.problem, ctx.sysids = problem, sysids
        if problem.checkpoint:
            solver.close()
            ctx.solver = None
        else:
            ctx.solver = solver
        ctx.stats = None
        return X

    @staticmethod
    def backward(ctx, gX):
        theta, X = ctx.saved_tensors
        problem, solver = ctx.problem, ctx.solver
        p, n = X.shape
        Lam = torch.empty_like(X)
        val = torch.empty(problem.col.numel(), dtype=torch.float64, device=X.device)
        gX = gX.contiguous()
        if problem.checkpoint:
            # W_j recomputed: the POD of the snapshots the forward solve of system j held
            solver = PodCG(n, w_max=problem.w_max, s_max=problem.s_max, energy=problem.energy)
            for j in reversed(range(p)):
                assemble(problem, theta, j, out=val)
                A = DeviceCSR(problem.row_ptr, problem.col, val)
                solver.clear_snapshots()
                if j > 0:
                    solver.add_snapshots(X[max(0, j - problem.s_max):j].t())
                solver.solve(A, gX[j], problem.tol, x_out=Lam[j])
        else:
            for j in reversed(range(p)):
                assemble(problem, theta, j, out=val)
                A = DeviceCSR(problem.row_ptr, problem.col, val)
                solver.solve_adjoint(ctx.sysids[j], A, gX[j], problem.tol, lam_out=Lam[j])
        grad_theta = theta_grad(problem, theta, Lam, X)
        solver.close()
        return grad_theta, Lam, None


def solve_sequence(theta: torch.Tensor, B: torch.Tensor, problem: DiffusionProblem) -> torch.Tensor:
    """X[j] = A_j(theta)^{-1} B[j], differentiable in theta and B."""
    return SequenceSolve.apply(theta, B, problem)
