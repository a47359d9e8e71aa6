"""FP64 CPU oracle for POD-augmented CG — TEST INFRASTRUCTURE ONLY.

Plain, slow, obviously correct reference implementation (see ``pod_cg_oracle.c``) of
what the GPU library computes, used only by the test suite, the package smoke check and
the benchmark's CPU-baseline leg. It shares no code with the CUDA library and imports
nothing from it. Inputs are plain numpy arrays (CSR as ``row_ptr``/``col``/``val``,
n-by-k blocks as Fortran-ordered float64 arrays).

The sequence driver (:class:`OracleSequence`) is the paper's overall algorithm
(Section 4.4, Algorithm 3) reduced to the recycled-solution form: the POD basis for
system j is computed (Algorithm 4, identity metric, unit weights) from the last
``s_max`` solutions, stage one (Algorithm 2) solves on it directly, then augmented PCG
(Algorithm 1) iterates to the tolerance.
"""
from __future__ import annotations

import contextlib
import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "pod_cg_oracle.c")
_LOCK = threading.Lock()
_LIBS: dict[int, ctypes.CDLL] = {}

STATUS = {0: "ok", 1: "arg", 2: "not_spd", 3: "breakdown", 4: "maxit", 5: "nonfinite"}


def lib_path(mutant: int = 0, out_dir: str | None = None) -> str:
    d = out_dir or os.path.join(_HERE, "_build")
    name = "liborc.so" if mutant == 0 else f"liborc_mut{mutant}.so"
    return os.path.join(d, name)


def build(mutant: int = 0, out_dir: str | None = None, force: bool = False) -> str:
    """Compile the oracle with gcc (plain -O2, portable flags, no fused multiply-add
    contraction, so x86 and Arm builds round identically) and return the .so path.

    ``mutant`` > 0 plants the numbered mistake (``-DORC_MUTANT=k``) for the pin-sensitivity
    tests; the normal build uses 0.
    """
    out = lib_path(mutant, out_dir)
    os.makedirs(os.path.dirname(out), exist_ok=True)
    if (not force and os.path.exists(out)
            and os.path.getmtime(out) >= os.path.getmtime(_SRC)):
        return out
    tmp = out + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared", f"-DORC_MUTANT={int(mutant)}",
           _SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, out)
    return out


class _Info(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int), ("iters", ctypes.c_int),
                ("refinements", ctypes.c_int), ("w", ctypes.c_int),
                ("chol_failed", ctypes.c_int), ("pad_", ctypes.c_int),
                ("stage1_relres", ctypes.c_double), ("final_relres", ctypes.c_double),
                ("cond_gram", ctypes.c_double)]


def _p(a):
    return a.ctypes.data_as(ctypes.c_void_p) if a is not None else None


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64) if np.ndim(a) <= 1 else np.asfortranarray(a, dtype=np.float64)


def _i32(a):
    return np.ascontiguousarray(a, dtype=np.int32)


class Oracle:
    """ctypes front end of one oracle build (``mutant`` selects a planted-mistake build)."""

    def __init__(self, mutant: int = 0, out_dir: str | None = None):
        with _LOCK:
            path = build(mutant, out_dir)
            lib = ctypes.CDLL(path)
        self.lib = lib
        vp, ci, cd = ctypes.c_void_p, ctypes.c_int, ctypes.c_double
        lib.orc_spmv.argtypes = [ci, vp, vp, vp, vp, vp]
        lib.orc_theta_grad.argtypes = [ci, ci, ci, vp, ci, vp, vp, vp]
        lib.orc_dot.argtypes = [ci, vp, vp]
        lib.orc_dot.restype = cd
        lib.orc_gram.argtypes = [ci, ci, vp, ci, vp, vp]
        lib.orc_spmm.argtypes = [ci, vp, vp, vp, ci, vp, vp]
        lib.orc_cholesky.argtypes = [ci, vp, vp]
        lib.orc_chol_solve.argtypes = [ci, vp, vp, vp]
        lib.orc_jacobi_eig.argtypes = [ci, vp, vp, vp, ci]
        lib.orc_pod_evd.argtypes = [ci, ci, vp, cd, ci, cd, vp, vp]
        lib.orc_jacobi_svd.argtypes = [ci, ci, vp, vp, vp, ci]
        lib.orc_pod_evd_metric.argtypes = [ci, ci, vp, vp, vp, vp, cd, ci, cd, vp, vp]
        lib.orc_pod_svd.argtypes = [ci, ci, vp, ci, vp, cd, ci, cd, vp, vp]
        lib.orc_stage_one.argtypes = [ci, vp, vp, vp, vp, ci, vp, vp, vp]
        lib.orc_aug_pcg.argtypes = [ci, vp, vp, vp, vp, ci, vp, vp, vp, cd, ci, ci, vp,
                                    ctypes.POINTER(_Info), vp, vp, ci]
        lib.orc_pcg.argtypes = [ci, vp, vp, vp, vp, vp, cd, ci, vp, ctypes.POINTER(ci)]
        lib.orc_solve_system.argtypes = [ci, vp, vp, vp, vp, ci, vp, cd, ci, ci, vp,
                                         ctypes.POINTER(_Info), vp, vp, ci]
        lib.orc_stage_two.argtypes = [ci, vp, vp, vp, vp, ci, vp, ci, vp, vp, cd, ci,
                                      ctypes.POINTER(ci), vp, vp, vp, ctypes.POINTER(cd)]
        lib.orc_solve_system3.argtypes = [ci, vp, vp, vp, vp, ci, vp, ci, cd, cd, ci, ci, ci, vp,
                                          ctypes.POINTER(_Info), ctypes.POINTER(ci), ctypes.POINTER(cd),
                                          vp, vp, ci, cd]
        lib.orc_solve_system3_it.argtypes = [ci, vp, vp, vp, vp, ci, vp, ci, cd, cd, cd, ci, ci, vp,
                                             ctypes.POINTER(_Info), ctypes.POINTER(ci), ctypes.POINTER(ci),
                                             vp, vp, ci]
        lib.orc_set_dependence_stop.argtypes = [ci]
        lib.orc_set_dependence_stop.restype = ci

    @contextlib.contextmanager
    def dependence_stop(self, on: bool = True):
        """Within the block, stage two and the inner reduced solves stop before a direction
        that the re-A-orthogonalisation pass found numerically dependent on the stored ones
        (its A-norm squared at most the part the pass removed); off by default. The setting
        belongs to the loaded library, so it is restored on exit."""
        old = self.lib.orc_set_dependence_stop(int(on))
        try:
            yield
        finally:
            self.lib.orc_set_dependence_stop(old)

    # -- Section 2 / basic kernels -------------------------------------------------
    def spmv(self, A, x):
        rp, col, val = _i32(A[0]), _i32(A[1]), _f64(A[2])
        n = len(rp) - 1
        x = _f64(x)
        y = np.empty(n)
        self.lib.orc_spmv(n, _p(rp), _p(col), _p(val), _p(x), _p(y))
        return y

    def dot(self, a, b):
        a, b = _f64(a), _f64(b)
        return self.lib.orc_dot(len(a), _p(a), _p(b))

    def gram(self, X, Y):
        X, Y = _f64(X), _f64(Y)
        n, p = X.shape
        q = Y.shape[1]
        G = np.empty((p, q))
        self.lib.orc_gram(n, p, _p(X), q, _p(Y), _p(G))
        return G

    def spmm(self, A, W):
        rp, col, val = _i32(A[0]), _i32(A[1]), _f64(A[2])
        W = _f64(W)
        n, w = W.shape
        AW = np.empty((n, w), order="F")
        self.lib.orc_spmm(n, _p(rp), _p(col), _p(val), w, _p(W), _p(AW))
        return AW

    # -- small dense -------------------------------------------------------------------
    def cholesky(self, G):
        G = np.ascontiguousarray(G, dtype=np.float64)
        w = G.shape[0]
        R = np.empty((w, w))
        st = self.lib.orc_cholesky(w, _p(G), _p(R))
        return R, st

    def chol_solve(self, R, c):
        R = np.ascontiguousarray(R, dtype=np.float64)
        c = _f64(c)
        y = np.empty(len(c))
        self.lib.orc_chol_solve(len(c), _p(R), _p(c), _p(y))
        return y

    def jacobi_eig(self, G, max_sweeps: int = 60):
        G = np.ascontiguousarray(G, dtype=np.float64)
        s = G.shape[0]
        ev = np.empty(s)
        V = np.empty((s, s))
        sweeps = self.lib.orc_jacobi_eig(s, _p(G), _p(ev), _p(V), max_sweeps)
        return ev, V, sweeps

    # -- Algorithm 4 ----------------------------------------------------------------------
    def pod_evd(self, S, energy: float, w_max: int, rank_tol: float = 1e-13):
        S = _f64(S)
        n, s = S.shape
        W = np.zeros((n, max(w_max, 1)), order="F")
        sig2 = np.empty(max(s, 1))
        w = self.lib.orc_pod_evd(n, s, _p(S), energy, w_max, rank_tol, _p(W), _p(sig2))
        return np.asfortranarray(W[:, :w]), w, sig2[:s]

    def pod_evd_metric(self, S, A, energy: float, w_max: int, rank_tol: float = 1e-13):
        """POD with the metric A (Algorithm 4 with Theta = A): W^T A W = I."""
        S = _f64(S)
        n, s = S.shape
        rp, col, val = _i32(A[0]), _i32(A[1]), _f64(A[2])
        W = np.zeros((n, max(w_max, 1)), order="F")
        sig2 = np.empty(max(s, 1))
        w = self.lib.orc_pod_evd_metric(n, s, _p(S), _p(rp), _p(col), _p(val), energy, w_max, rank_tol, _p(W),
                                        _p(sig2))
        return np.asfortranarray(W[:, :w]), w, sig2[:s]

    # -- Algorithm 5 ----------------------------------------------------------------------
    def jacobi_svd(self, B, max_sweeps: int = 60):
        B = _f64(B)
        q, s = B.shape
        sig = np.empty(s)
        V = np.empty((s, s))
        sweeps = self.lib.orc_jacobi_svd(q, s, _p(B), _p(sig), _p(V), max_sweeps)
        return sig, V, sweeps

    def pod_svd(self, S, C, energy: float, w_max: int, rank_tol: float = 1e-13):
        """POD with the output pseudometric C^T C (Algorithm 5); C is (q, n)."""
        S = _f64(S)
        n, s = S.shape
        C = np.ascontiguousarray(C, dtype=np.float64)
        q = C.shape[0]
        W = np.zeros((n, max(w_max, 1)), order="F")
        sig2 = np.empty(max(s, 1))
        w = self.lib.orc_pod_svd(n, s, _p(S), q, _p(C), energy, w_max, rank_tol, _p(W), _p(sig2))
        return np.asfortranarray(W[:, :w]), w, sig2[:s]

    # -- Algorithm 2 ----------------------------------------------------------------------
    def stage_one(self, A, b, W):
        rp, col, val = _i32(A[0]), _i32(A[1]), _f64(A[2])
        W = _f64(W)
        n, w = W.shape
        b = _f64(b)
        R = np.zeros((w, w))
        what = np.zeros(w)
        st = self.lib.orc_stage_one(n, _p(rp), _p(col), _p(val), _p(b), w, _p(W), _p(R), _p(what))
        return what, R, st

    # -- Algorithm 1 ----------------------------------------------------------------------
    def aug_pcg(self, A, b, W, R, xhat0, tol_abs, kmax=100000, max_refine=5, p_cap=0):
        rp, col, val = _i32(A[0]), _i32(A[1]), _f64(A[2])
        n = len(rp) - 1
        b = _f64(b)
        if W is None:
            W = np.zeros((n, 0), order="F")
        W = _f64(W)
        w = W.shape[1]
        R = np.ascontiguousarray(R if R is not None else np.zeros((max(w, 1), max(w, 1))), dtype=np.float64)
        xhat0 = _f64(xhat0 if xhat0 is not None else np.zeros(max(w, 1)))
        x = np.empty(n)
        info = _Info()
        P = np.zeros((n, p_cap), order="F") if p_cap else None
        g = np.zeros(p_cap) if p_cap else None
        self.lib.orc_aug_pcg(n, _p(rp), _p(col), _p(val), _p(b), w, _p(W), _p(R), _p(xhat0),
                             tol_abs, kmax, max_refine, _p(x), ctypes.byref(info), _p(P), _p(g), p_cap)
        return x, _info_dict(info), P, g

    def pcg(self, A, b, x0, tol_abs, kmax=100000):
        rp, col, val = _i32(A[0]), _i32(A[1]), _f64(A[2])
        n = len(rp) - 1
        b = _f64(b)
        x0 = _f64(x0) if x0 is not None else None
        x = np.empty(n)
        k = ctypes.c_int(0)
        st = self.lib.orc_pcg(n, _p(rp), _p(col), _p(val), _p(b), _p(x0), tol_abs, kmax, _p(x), ctypes.byref(k))
        return x, k.value, st

    def theta_grad(self, shape, theta, lam, xs):
        """dL/dtheta = -sum_j lambda_j^T (dA_j/dtheta) x_j for the diffusion operator on a grid
        of shape (my, mx) or (mz, my, mx); lam and xs are (nsys, n)."""
        sh = tuple(shape) if len(shape) == 3 else (1,) + tuple(shape)
        mz, my, mx = sh
        lam = np.ascontiguousarray(np.atleast_2d(lam), dtype=np.float64)
        xs = np.ascontiguousarray(np.atleast_2d(xs), dtype=np.float64)
        theta = _f64(theta)
        g = np.empty(mx * my * mz)
        self.lib.orc_theta_grad(mx, my, mz, _p(theta), lam.shape[0], _p(lam), _p(xs), _p(g))
        return g

    def solve_system(self, A, b, W, tol_rel, kmax=100000, max_refine=5, p_cap=0):
        rp, col, val = _i32(A[0]), _i32(A[1]), _f64(A[2])
        n = len(rp) - 1
        b = _f64(b)
        if W is None:
            W = np.zeros((n, 0), order="F")
        W = _f64(W)
        x = np.empty(n)
        info = _Info()
        P = np.zeros((n, p_cap), order="F") if p_cap else None
        g = np.zeros(p_cap) if p_cap else None
        self.lib.orc_solve_system(n, _p(rp), _p(col), _p(val), _p(b), W.shape[1], _p(W), tol_rel,
                                  kmax, max_refine, _p(x), ctypes.byref(info), _p(P), _p(g), p_cap)
        return x, _info_dict(info), P, g

    # -- Section 4.2 / 4.3 ------------------------------------------------------------------
    def stage_two(self, A, b, Y, w, R, what, tol_abs, kcap):
        """Stage two (Section 4.2) on the reduced system Y^T A Y yhat = Y^T b from
        yhat0 = [what; 0], augmenting with the first w columns of Y (factor R of W^T A W).
        Returns dict(k2, alpha, V2 (n x k2), T2, rhat_norm, status)."""
        rp, col, val = _i32(A[0]), _i32(A[1]), _f64(A[2])
        n = len(rp) - 1
        b, Y = _f64(b), _f64(Y)
        y = Y.shape[1]
        R = np.ascontiguousarray(R if w > 0 else np.zeros((1, 1)), dtype=np.float64)
        what = _f64(what if w > 0 else np.zeros(1))
        m = max(kcap, 1)
        alpha, T2 = np.zeros(m), np.zeros(m)
        V2 = np.zeros((n, m), order="F")
        k2, rn = ctypes.c_int(0), ctypes.c_double(0.0)
        st = self.lib.orc_stage_two(n, _p(rp), _p(col), _p(val), _p(b), y, _p(Y), w, _p(R), _p(what),
                                    tol_abs, kcap, ctypes.byref(k2), _p(alpha), _p(V2), _p(T2),
                                    ctypes.byref(rn))
        k = k2.value
        return {"k2": k, "alpha": alpha[:k], "V2": np.asfortranarray(V2[:, :k]), "T2": T2[:k],
                "rhat_norm": rn.value, "status": STATUS.get(st, str(st))}

    def solve_system3(self, A, b, Y, w, tol_rel, tol2_rel, w3_cap=64, kmax=100000, max_refine=5, p_cap=0,
                      tol3_rel=-1.0):
        """Three-stage solve (Section 4): stage one on the first w columns of Y, stage two
        over range(Y) to tol2_rel * tol_rel * ||b||, stage three (Algorithm 1) augmented with
        [W, V2] to tol_rel (or tol3_rel when >= 0). info gains k2 and stage2_relres;
        info["w"] is the stage-three basis size."""
        rp, col, val = _i32(A[0]), _i32(A[1]), _f64(A[2])
        n = len(rp) - 1
        b = _f64(b)
        Y = _f64(Y if Y is not None else np.zeros((n, 0)))
        x = np.empty(n)
        info = _Info()
        k2, s2 = ctypes.c_int(0), ctypes.c_double(0.0)
        P = np.zeros((n, p_cap), order="F") if p_cap else None
        g = np.zeros(p_cap) if p_cap else None
        self.lib.orc_solve_system3(n, _p(rp), _p(col), _p(val), _p(b), Y.shape[1], _p(Y), w, tol_rel, tol2_rel,
                                   w3_cap, kmax, max_refine, _p(x), ctypes.byref(info), ctypes.byref(k2),
                                   ctypes.byref(s2), _p(P), _p(g), p_cap, float(tol3_rel))
        d = _info_dict(info)
        d["k2"] = k2.value
        d["stage2_relres"] = s2.value
        return x, d, P, g

    def solve_system3_it(self, A, b, Y, w, tol_rel, tol2_rel, tol_in, kmax=100000, max_refine=5, p_cap=0,
                         return_directions=False):
        """Three-stage solve with the stage-three option of Section 4.3.1: stage three
        augments with the entire Y, each augmentation solve an inner reduced solve to
        tol_in * ||Y^T A z||. info gains k2 (stage-two iterations) and inner (inner reduced
        iterations, summed)."""
        rp, col, val = _i32(A[0]), _i32(A[1]), _f64(A[2])
        n = len(rp) - 1
        b = _f64(b)
        Y = _f64(Y if Y is not None else np.zeros((n, 0)))
        x = np.empty(n)
        info = _Info()
        k2, inner = ctypes.c_int(0), ctypes.c_int(0)
        P = np.zeros((n, p_cap), order="F") if p_cap else None
        g = np.zeros(p_cap) if p_cap else None
        self.lib.orc_solve_system3_it(n, _p(rp), _p(col), _p(val), _p(b), Y.shape[1], _p(Y), w, tol_rel, tol2_rel,
                                      tol_in, kmax, max_refine, _p(x), ctypes.byref(info), ctypes.byref(k2),
                                      ctypes.byref(inner), _p(P), _p(g), p_cap)
        d = _info_dict(info)
        d["k2"] = k2.value
        d["inner"] = inner.value
        if return_directions:
            return x, d, P, g
        return x, d


def _info_dict(info: _Info) -> dict:
    return {"status": STATUS.get(info.status, str(info.status)), "iters": info.iters,
            "refinements": info.refinements, "w": info.w, "chol_failed": bool(info.chol_failed),
            "stage1_relres": info.stage1_relres, "final_relres": info.final_relres,
            "cond_gram": info.cond_gram}


class OracleSequence:
    """Sequence driver: POD of the last ``s_max`` solutions → stage one → Algorithm 1.

    ``solve(A, b, tol)`` solves the next system and records its solution as a snapshot;
    ``add_snapshot(x)`` records an externally supplied solution instead.

    With ``three_stage`` the POD also gives the augmenting basis Y (energy ``energy_y``,
    at most ``y_max`` modes, never fewer than the stage-one dimension w, so that W is the
    first w columns of Y: POD bases are nested) and each system runs the three-stage
    algorithm (Section 4) with stage-two tolerance ``tol_stage2`` times the system's;
    ``stage3_full`` selects the stage-three option of Section 4.3.1 (augmenting with all of
    Y, inner reduced solves to ``tol_inner``). With ``C`` (q output functionals, (q, n))
    the POD uses the output-oriented metric C^T C (Algorithm 5); with ``metric_a`` it uses
    the metric A of the system being solved (Algorithm 4 with Theta = A).
    """

    def __init__(self, n: int, s_max: int = 40, w_max: int = 32, energy: float = 0.9999,
                 kmax: int = 100000, max_refine: int = 5, oracle: Oracle | None = None,
                 three_stage: bool = False, y_max: int = 40, energy_y: float = 1.0,
                 tol_stage2: float = 1e-4, w3_cap: int = 64, stage3_full: bool = False,
                 tol_inner: float = 1e-12, C=None, metric_a: bool = False):
        self.n, self.s_max, self.w_max, self.energy = n, s_max, w_max, energy
        self.kmax, self.max_refine = kmax, max_refine
        self.three_stage, self.y_max, self.energy_y = three_stage, y_max, energy_y
        self.tol_stage2, self.w3_cap = tol_stage2, w3_cap
        self.stage3_full, self.tol_inner = stage3_full, tol_inner
        self.C = None if C is None else np.ascontiguousarray(C, dtype=np.float64)
        self.metric_a = metric_a
        self._A = None   # the current system's matrix (metric A)
        self.orc = oracle or Oracle()
        self.snaps: list[np.ndarray] = []

    def add_snapshot(self, x):
        self.snaps.append(np.array(x, dtype=np.float64))
        if len(self.snaps) > self.s_max:
            self.snaps.pop(0)

    def basis(self):
        if not self.snaps:
            return np.zeros((self.n, 0), order="F"), 0, np.zeros(0)
        S = np.asfortranarray(np.stack(self.snaps, axis=1))
        return self._pod(S, self.energy, self.w_max)

    def _pod(self, S, energy, w_max):
        if self.C is not None:   # output-oriented metric C^T C (Algorithm 5)
            return self.orc.pod_svd(S, self.C, energy, w_max)
        if self.metric_a:        # metric A of the system being solved
            return self.orc.pod_evd_metric(S, self._A, energy, w_max)
        return self.orc.pod_evd(S, energy, w_max)

    def basis_y(self):
        """(Y, w): the augmenting basis and the stage-one dimension (W = Y[:, :w])."""
        if not self.snaps:
            return np.zeros((self.n, 0), order="F"), 0
        S = np.asfortranarray(np.stack(self.snaps, axis=1))
        _, w, _ = self._pod(S, self.energy, self.w_max)
        _, y, _ = self._pod(S, self.energy_y, self.y_max)
        y = max(y, w)
        # energy 2 is never reached: all modes up to the numerical rank, capped at y
        Y, y2, _ = self._pod(S, 2.0, y)
        return Y, min(w, y2)

    def solve(self, A, b, tol_rel, record: bool = True):
        self._A = A
        if self.three_stage:
            Y, w = self.basis_y()
            if self.stage3_full:
                x, info = self.orc.solve_system3_it(A, b, Y, w, tol_rel, self.tol_stage2, self.tol_inner,
                                                    self.kmax, self.max_refine)
            else:
                x, info, _, _ = self.orc.solve_system3(A, b, Y, w, tol_rel, self.tol_stage2, self.w3_cap,
                                                       self.kmax, self.max_refine)
            info["s"] = len(self.snaps)
            info["y"] = Y.shape[1]
            if record:
                self.add_snapshot(x)
            return x, info
        W, w, sig2 = self.basis()
        x, info, _, _ = self.orc.solve_system(A, b, W, tol_rel, self.kmax, self.max_refine)
        info["s"] = len(self.snaps)
        if record:
            self.add_snapshot(x)
        return x, info


class OracleKrylovSequence:
    """The overall algorithm (Section 4.4, Algorithm 3) with the paper's own POD ingredients
    (Section 3): the augmenting basis accumulates every system's stage-three directions
    A_j-normalised, Z <- [Z, P_j T_j^{-1/2}] (reading of the printed P_j sqrt(T_j): the
    normalisation the orthogonality proof uses); new directions join the stage-one basis W
    by the rule ``nu`` (1: all, 0: none, in between: those with T_kk / sum T > nu); once the
    basis holds more than ``y_threshold`` vectors it is compressed by POD (Algorithm 4 with
    metric A_j and weights ``weights``: "prev" = the coordinates of the last solution in Z,
    "rbf" = those of the solutions since the last compression combined with weights
    2^-(i-1), Eq. (weightsRBF)) to ``y_keep`` vectors, the first ``w_keep`` of which form
    W. Each system runs stage one on W, stage two over the augmenting basis and stage three
    with [W, V2] (Section 4.3), or with ``stage3_full`` over the whole basis (Section
    4.3.1, inner reduced solves to ``tol_inner``), x_bar = 0.

    Between compressions Z only grows by appending, so the coordinates of earlier solutions
    are prefixes of the current coordinate vector (zero-padded). The coordinates are the
    previous weights of Eq. (weightsPrevious), (Z^T A_j Z)^+ Z^T b_j with x_bar = 0, with a
    pseudo-inverse where Z is rank deficient (a reading: the paper writes the inverse).

    ``normalise`` = "sqrt" appends P_j T_j^{1/2} as printed instead; it exists so that a
    test can show which of the two readings Theorem 5 holds for.
    """

    def __init__(self, n: int, y_threshold: int = 200, y_keep: int = 100, w_keep: int = 5, nu: float = 1.0,
                 weights: str = "rbf", tol_stage2: float = 1e-4, kmax: int = 100000, max_refine: int = 5,
                 p_cap: int = 5000, oracle: Oracle | None = None, stage3_full: bool = False,
                 tol_inner: float = 1e-12, normalise: str = "inv_sqrt"):
        if normalise not in ("inv_sqrt", "sqrt"):
            raise ValueError("normalise must be 'inv_sqrt' or 'sqrt'")
        self.normalise = normalise
        self.n = n
        self.y_threshold, self.y_keep, self.w_keep, self.nu = y_threshold, y_keep, w_keep, nu
        self.weights, self.tol_stage2 = weights, tol_stage2
        self.kmax, self.max_refine, self.p_cap = kmax, max_refine, p_cap
        self.stage3_full, self.tol_inner = stage3_full, tol_inner
        self.orc = oracle or Oracle()
        self.Z = np.zeros((n, 0), order="F")   # augmenting basis, append-only between compressions
        self.w_idx: list[int] = []             # columns of Z that form the stage-one basis W
        self.coords: list[np.ndarray] = []     # Galerkin coordinates of the solutions since the last compression
        self.compressions = 0

    def _prev_weights(self, A, b):
        """The previous weights of Eq. (weightsPrevious) with x_bar = 0: (Z^T A Z)^+ Z^T b,
        the Galerkin coordinates of the system's exact solution in range(Z)."""
        AZ = self.orc.spmm(A, self.Z)
        G = self.Z.T @ AZ
        return np.linalg.lstsq(0.5 * (G + G.T), self.Z.T @ b, rcond=1e-13)[0]

    def solve(self, A, b, tol_rel):
        n = self.n
        w = len(self.w_idx)
        rest = [k for k in range(self.Z.shape[1]) if k not in set(self.w_idx)]
        Y = np.asfortranarray(self.Z[:, self.w_idx + rest]) if self.Z.shape[1] else np.zeros((n, 0), order="F")
        if self.stage3_full and Y.shape[1] > 0:   # stage three over the whole basis (Section 4.3.1)
            x, info, P, g = self.orc.solve_system3_it(A, b, Y, w, tol_rel, self.tol_stage2, self.tol_inner,
                                                      kmax=self.kmax, max_refine=self.max_refine, p_cap=self.p_cap,
                                                      return_directions=True)
        else:
            x, info, P, g = self.orc.solve_system3(A, b, Y, w, tol_rel, self.tol_stage2, w3_cap=max(Y.shape[1], 1),
                                                   kmax=self.kmax, max_refine=self.max_refine, p_cap=self.p_cap)
        k = min(info["iters"], self.p_cap)
        P, g = P[:, :k], g[:k]
        scale = 1.0 / np.sqrt(g) if self.normalise == "inv_sqrt" else np.sqrt(g)
        Pn = P * scale[None, :] if k else np.zeros((n, 0))
        # new directions for the stage-one basis (Algorithm 3, rule nu)
        if self.nu >= 1.0:
            new_w = list(range(k))
        elif self.nu <= 0.0:
            new_w = []
        else:
            new_w = [i for i in range(k) if g[i] / g.sum() > self.nu]
        base = self.Z.shape[1]
        self.Z = np.asfortranarray(np.concatenate([self.Z, Pn], axis=1))
        self.w_idx = self.w_idx + [base + i for i in new_w]
        info["y"] = Y.shape[1]
        info["k"] = k
        # coordinates of this solution in the (grown) basis
        self.coords.append(self._prev_weights(A, b))
        if self.Z.shape[1] > self.y_threshold:       # compression (Algorithm 3, truncation steps)
            m = self.Z.shape[1]
            if self.weights == "prev":
                gam = self.coords[-1]
            else:
                gam = np.zeros(m)
                for i, c in enumerate(reversed(self.coords)):
                    gam[:len(c)] += c * 0.5 ** i
            Zg = np.asfortranarray(self.Z * gam[None, :])
            Wk, yk, _ = self.orc.pod_evd_metric(Zg, A, 2.0, self.y_keep)
            self.Z = np.asfortranarray(Wk)
            self.w_idx = list(range(min(self.w_keep, yk)))
            self.coords = []
            self.compressions += 1
            info["compressed_to"] = yk
        return x, info
