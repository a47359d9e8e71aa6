"""Python front end of the C ABI: torch tensors in, torch tensors out.

PyTorch provides device memory and streams only; every step of the path runs in the
library's CUDA kernels. n-by-k blocks are passed to the library column-major; in Python
they are (n, k) tensors (any layout; they are made column-major before the call).
"""
from __future__ import annotations

import ctypes

import torch

from . import _lib


class PodCGError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{_lib.STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


def _check(st: int, handle=None):
    if st != 0:
        L = _lib.load()
        msg = L.pod_cg_last_error(handle).decode(errors="replace")
        raise PodCGError(st, msg)


def _stream_ptr(stream) -> int:
    if stream is None:
        stream = torch.cuda.current_stream()
    return stream.cuda_stream


def _colmajor(X: torch.Tensor) -> torch.Tensor:
    """(n, k) tensor → contiguous (k, n) buffer = column-major n-by-k."""
    return X.t().contiguous()


class DeviceCSR:
    """A CSR matrix resident on the GPU (int32 indices, float64 values)."""

    def __init__(self, row_ptr: torch.Tensor, col: torch.Tensor, val: torch.Tensor):
        assert row_ptr.dtype == torch.int32 and col.dtype == torch.int32 and val.dtype == torch.float64
        self.row_ptr, self.col, self.val = row_ptr, col, val
        self.n = row_ptr.numel() - 1
        self.nnz = col.numel()

    @classmethod
    def from_numpy(cls, row_ptr, col, val, device="cuda"):
        return cls(torch.as_tensor(row_ptr, dtype=torch.int32, device=device),
                   torch.as_tensor(col, dtype=torch.int32, device=device),
                   torch.as_tensor(val, dtype=torch.float64, device=device))

    def with_values(self, val: torch.Tensor) -> "DeviceCSR":
        return DeviceCSR(self.row_ptr, self.col, val)

    def struct(self) -> _lib.CSRStruct:
        return _lib.CSRStruct(self.n, self.nnz, self.row_ptr.data_ptr(), self.col.data_ptr(), self.val.data_ptr())


DEFAULTS = dict(w_max=32, s_max=40, energy=0.9999, rank_tol=1e-13, k_max=100000, max_refine=5,
                precision=0, inner_tol=1e-5, use_tc_gram=-1, cond_diag=0, keep_factors=0)


def make_config(**kw) -> _lib.Config:
    L = _lib.load()
    c = _lib.Config()
    L.pod_cg_config_default(ctypes.byref(c))
    for k, v in kw.items():
        if k == "precision" and isinstance(v, str):
            v = {"fp64": 0, "mixed": 1}[v]
        setattr(c, k, v)
    return c


class PodCG:
    """POD-augmented CG solver for a sequence of systems of order n (one handle)."""

    def __init__(self, n: int, stream: torch.cuda.Stream | None = None, **config):
        self.L = _lib.load()
        self.n = n
        self.stream = stream or torch.cuda.current_stream()
        self.cfg = make_config(**config)
        h = ctypes.c_void_p()
        _check(self.L.pod_cg_create(n, ctypes.byref(self.cfg), ctypes.c_void_p(_stream_ptr(self.stream)),
                                    ctypes.byref(h)))
        self.h = h

    def close(self):
        if self.h:
            self.L.pod_cg_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def add_snapshots(self, X: torch.Tensor):
        """Append snapshots: X is a length-n vector or an (n, m) block."""
        if X.dim() == 1:
            X = X.view(-1, 1)
        assert X.shape[0] == self.n and X.dtype == torch.float64 and X.is_cuda
        Xc = _colmajor(X)
        if Xc.data_ptr() != X.data_ptr():
            Xc.record_stream(self.stream)   # the copy into the ring is stream-ordered
        _check(self.L.pod_cg_add_snapshots(self.h, Xc.data_ptr(), X.shape[1]), self.h)

    def clear_snapshots(self):
        _check(self.L.pod_cg_clear_snapshots(self.h), self.h)

    def set_output_functionals(self, C: torch.Tensor | None):
        """Output-oriented POD metric C^T C: C is (q, n) float64 on the device (None: back to
        the identity metric)."""
        if C is None:
            _check(self.L.pod_cg_set_output_functionals(self.h, None, 0), self.h)
            return
        assert C.dtype == torch.float64 and C.is_cuda and C.shape[1] == self.n
        C = C.contiguous()
        self._C = C   # the copy into the handle is stream-ordered
        _check(self.L.pod_cg_set_output_functionals(self.h, C.data_ptr(), C.shape[0]), self.h)

    def solve(self, A: DeviceCSR, b: torch.Tensor, tol: float, x_out: torch.Tensor | None = None,
              raise_on_error: bool = True):
        """Solve A x = b to ||b - A x|| <= tol ||b||. Returns (x, stats dict)."""
        assert b.dtype == torch.float64 and b.is_cuda and b.numel() == self.n
        b = b.contiguous()
        if x_out is None:
            x_out = torch.empty_like(b)
        st = _lib.Stats()
        A_s = A.struct()
        rc = self.L.pod_cg_solve(self.h, ctypes.byref(A_s), b.data_ptr(), float(tol), x_out.data_ptr(),
                                 ctypes.byref(st))
        # statuses that end a solve with x_out holding the last iterate
        if rc != 0 and (raise_on_error or rc not in (2, 3, 4, 5, 7)):
            _check(rc, self.h)
        return x_out, st.as_dict()

    def solve_adjoint(self, system_id: int, A: DeviceCSR, g: torch.Tensor, tol: float,
                      lam_out: torch.Tensor | None = None):
        g = g.contiguous()
        if lam_out is None:
            lam_out = torch.empty_like(g)
        st = _lib.Stats()
        A_s = A.struct()
        _check(self.L.pod_cg_solve_adjoint(self.h, system_id, ctypes.byref(A_s), g.data_ptr(), float(tol),
                                           lam_out.data_ptr(), ctypes.byref(st)), self.h)
        return lam_out, st.as_dict()

    def time_kernels(self, A: DeviceCSR, b: torch.Tensor, reps: int = 20) -> list[float]:
        """Mean ms per launch of the stage-three kernels [spmv_cg, update, direction, residual]
        (CUDA events on the handle's stream), on the basis of the last solve."""
        ms = (ctypes.c_float * 4)()
        A_s = A.struct()
        _check(self.L.pod_cg_time_kernels(self.h, ctypes.byref(A_s), b.contiguous().data_ptr(), int(reps), ms),
               self.h)
        return [float(v) for v in ms]

    def tuning(self) -> dict:
        """SpMV lanes per row chosen for the last solve and the autotuner's timings."""
        L = ctypes.c_int(0)
        ms = (ctypes.c_float * 6)()
        _check(self.L.pod_cg_tuning(self.h, ctypes.byref(L), ms), self.h)
        forms = (ctypes.c_int * 6)()
        pms = (ctypes.c_float * 24)()
        _check(self.L.pod_cg_proj_tuning(self.h, forms, pms), self.h)

        def name(f, bit):
            return "staged" if f & bit else "direct"
        proj = {f"w<={wb}": {"update": name(forms[b], 1), "direction": name(forms[b], 2),
                             "ms_update_direct": pms[4 * b], "ms_direction_direct": pms[4 * b + 1],
                             "ms_update_staged": pms[4 * b + 2], "ms_direction_staged": pms[4 * b + 3]}
                for b, wb in enumerate((0, 8, 16, 32, 48, 64)) if forms[b] >= 0}
        cap = ctypes.c_int(0)
        caps = (ctypes.c_int * 8)()
        cms = (ctypes.c_float * 8)()
        _check(self.L.pod_cg_w_tuning(self.h, ctypes.byref(cap), caps, cms), self.h)
        wsel = {"cap": cap.value, "ms_per_solve": {str(caps[i]): cms[i] for i in range(8) if caps[i] > 0}}
        return {"spmv_lanes": L.value, "lane_ms": {str(1 << k): ms[k] for k in range(6)}, "projection": proj,
                "w_cap": wsel}

    @property
    def last_w(self) -> int:
        w = ctypes.c_int(0)
        _check(self.L.pod_cg_get_basis(self.h, None, ctypes.byref(w)), self.h)
        return w.value

    def basis(self) -> torch.Tensor:
        """The basis W of the last solve as an (n, w) tensor."""
        w = ctypes.c_int(0)
        buf = torch.empty((self.cfg.w_max, self.n), dtype=torch.float64, device="cuda")
        _check(self.L.pod_cg_get_basis(self.h, buf.data_ptr(), ctypes.byref(w)), self.h)
        return buf[: w.value].t()

    # -- the paper's snapshots: accumulated Krylov vectors (Section 3, Algorithm 3) ----------
    def set_krylov(self, y_threshold: int = 40, y_keep: int = 20, w_keep: int = 5, nu: float = 1.0,
                   weights: str = "rbf", p_cap: int = 24, frozen: bool = False):
        """Switch to Krylov-vector snapshots (pod_cg_set_krylov); the handle must be FP64 with
        three_stage = 1. weights: "rbf" or "prev"; y_threshold = 0: compress only on request."""
        if weights not in ("rbf", "prev"):
            raise ValueError("weights must be 'rbf' or 'prev'")
        kc = _lib.KrylovConfig(int(y_threshold), int(y_keep), int(w_keep), float(nu), 0 if weights == "rbf" else 1,
                               int(p_cap), 1 if frozen else 0)
        _check(self.L.pod_cg_set_krylov(self.h, ctypes.byref(kc)), self.h)

    def krylov_state(self, with_basis: bool = False) -> dict:
        """z (columns of Z), the stage-one columns, compressions, and optionally Z (n, z)."""
        z, w, c = ctypes.c_int(0), ctypes.c_int(0), ctypes.c_int(0)
        cols = (ctypes.c_int * 64)()
        _check(self.L.pod_cg_krylov_state(self.h, ctypes.byref(z), ctypes.byref(w), ctypes.byref(c), None, cols),
               self.h)
        out = {"z": z.value, "w": w.value, "compressions": c.value, "w_cols": list(cols[: w.value])}
        if with_basis:
            Z = torch.empty((max(z.value, 1), self.n), dtype=torch.float64, device="cuda")
            _check(self.L.pod_cg_krylov_state(self.h, None, None, None, Z.data_ptr(), None), self.h)
            out["Z"] = Z[: z.value].t()
        return out

    def krylov_coords(self, A: DeviceCSR, b: torch.Tensor) -> tuple[torch.Tensor, torch.Tensor]:
        """(Z^T A Z)^+ Z^T b in the current Z and the weights the next compression would use."""
        z = self.krylov_state()["z"]
        c = torch.zeros(max(z, 1), dtype=torch.float64, device="cuda")
        eta = torch.zeros(max(z, 1), dtype=torch.float64, device="cuda")
        A_s = A.struct()
        _check(self.L.pod_cg_krylov_coords(self.h, ctypes.byref(A_s), b.contiguous().data_ptr(), c.data_ptr(),
                                           eta.data_ptr()), self.h)
        return c[:z], eta[:z]

    def krylov_compress(self, A: DeviceCSR, eta: torch.Tensor | None, y_keep: int, w_keep: int):
        """Compress Z now with weights eta (None: the accumulated ones) to y_keep columns."""
        A_s = A.struct()
        e = eta.contiguous() if eta is not None else None
        _check(self.L.pod_cg_krylov_compress(self.h, ctypes.byref(A_s), e.data_ptr() if e is not None else None,
                                             int(y_keep), int(w_keep)), self.h)

    def stage3_basis(self) -> tuple[torch.Tensor, torch.Tensor]:
        """Stage three's augmenting basis [W, V2] of the last solve and A [W, V2], as (n, w3)
        tensors (FP64 handles)."""
        w3 = ctypes.c_int(0)
        B = torch.empty((64, self.n), dtype=torch.float64, device="cuda")
        AB = torch.empty((64, self.n), dtype=torch.float64, device="cuda")
        _check(self.L.pod_cg_get_stage3_basis(self.h, B.data_ptr(), AB.data_ptr(), ctypes.byref(w3)), self.h)
        return B[: w3.value].t(), AB[: w3.value].t()


# ------------------------------------------------------------------ stateless steps


def spmv(A: DeviceCSR, x: torch.Tensor, stream=None) -> torch.Tensor:
    L = _lib.load()
    y = torch.empty_like(x)
    A_s = A.struct()
    _check(L.pod_cg_spmv(ctypes.byref(A_s), x.contiguous().data_ptr(), y.data_ptr(),
                         ctypes.c_void_p(_stream_ptr(stream))))
    return y


def spmm(A: DeviceCSR, W: torch.Tensor, stream=None) -> torch.Tensor:
    L = _lib.load()
    Wc = _colmajor(W)
    AWc = torch.empty_like(Wc)
    A_s = A.struct()
    _check(L.pod_cg_spmm(ctypes.byref(A_s), Wc.data_ptr(), W.shape[1], AWc.data_ptr(),
                         ctypes.c_void_p(_stream_ptr(stream))))
    return AWc.t()


def gram_workspace(n: int, p: int, q: int) -> int:
    return int(_lib.load().pod_cg_gram_workspace(n, p, q))


def gram(X: torch.Tensor, Y: torch.Tensor, stream=None) -> torch.Tensor:
    """G = X^T Y for (n, p) and (n, q) float64 tensors."""
    L = _lib.load()
    n, p = X.shape
    q = Y.shape[1]
    Xc, Yc = _colmajor(X), _colmajor(Y)
    G = torch.empty((p, q), dtype=torch.float64, device=X.device)
    ws = gram_workspace(n, p, q)
    work = torch.empty(max(ws, 8), dtype=torch.uint8, device=X.device)
    _check(L.pod_cg_gram(n, Xc.data_ptr(), p, Yc.data_ptr(), q, G.data_ptr(), work.data_ptr(), ws,
                         ctypes.c_void_p(_stream_ptr(stream))))
    return G


def gram_tc(X: torch.Tensor, Y: torch.Tensor | None, e: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    """G = X^T [Y, e] on the tensor cores (split-bf16 products) for (n, p) and (n, qy) tensors
    of one dtype (float32 or float64) and an optional float64 column e (n,); G is float64."""
    L = _lib.load()
    n, p = X.shape
    if X.dtype not in (torch.float32, torch.float64):
        raise TypeError("gram_tc: X must be float32 or float64")
    qy = 0 if Y is None else Y.shape[1]
    if Y is not None and Y.dtype != X.dtype:
        raise TypeError("gram_tc: X and Y must share a dtype")
    Xc = _colmajor(X)
    Yc = _colmajor(Y) if Y is not None else None
    ec = e.to(torch.float64).contiguous() if e is not None else None
    q = qy + (1 if e is not None else 0)
    G = torch.empty((p, q), dtype=torch.float64, device=X.device)
    ws = int(L.pod_cg_gram_tc_workspace(n, p, q))
    work = torch.empty(max(ws, 8), dtype=torch.uint8, device=X.device)
    _check(L.pod_cg_gram_tc(n, X.element_size(), Xc.data_ptr(), p, Yc.data_ptr() if Yc is not None else None, qy,
                            ec.data_ptr() if ec is not None else None, G.data_ptr(), work.data_ptr(), ws,
                            ctypes.c_void_p(_stream_ptr(stream))))
    return G


def pod(S: torch.Tensor, energy: float, w_max: int, rank_tol: float = 1e-13, stream=None):
    """POD basis of the (n, s) snapshot block: returns (W (n, w), w, sigma^2 (s,))."""
    L = _lib.load()
    n, s = S.shape
    Sc = _colmajor(S)
    Wc = torch.zeros((w_max, n), dtype=torch.float64, device=S.device)
    sig2 = torch.empty(s, dtype=torch.float64, device=S.device)
    w = ctypes.c_int(0)
    ws = gram_workspace(n, s, s)
    work = torch.empty(max(ws, 8), dtype=torch.uint8, device=S.device)
    _check(L.pod_cg_pod(n, s, Sc.data_ptr(), float(energy), float(rank_tol), int(w_max), Wc.data_ptr(),
                        sig2.data_ptr(), ctypes.byref(w), work.data_ptr(), ws, ctypes.c_void_p(_stream_ptr(stream))))
    torch.cuda.current_stream().synchronize()
    return Wc[: w.value].t(), w.value, sig2
