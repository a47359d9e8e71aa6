"""Many independent sequences in one persistent launch (pod_cg_batch_*), torch front end."""
from __future__ import annotations

import ctypes

import numpy as np
import torch

from . import _lib
from .solver import make_config


class BatchSolver:
    """Holds every system of every sequence on the GPU and solves them all with one graph
    launch of the persistent kernel. ``cluster`` = CTAs per worker (0: autotune)."""

    def __init__(self, sequences, device="cuda", cluster: int = 0, systems=None, stream=None, **config):
        self.L = _lib.load()
        self.sequences = sequences
        self.stream = stream or torch.cuda.current_stream()
        self._keep = []
        descs = (_lib.BatchSeq * len(sequences))()
        for i, seq in enumerate(sequences):
            sy = systems[i] if systems is not None else seq.all_systems()
            p = len(sy)
            rp = torch.as_tensor(seq.row_ptr, device=device)
            col = torch.as_tensor(seq.col, device=device)
            val = torch.as_tensor(np.stack([v for _, v, _ in sy]), device=device).contiguous()
            b = torch.as_tensor(np.stack([bb for _, _, bb in sy]), device=device).contiguous()
            x = torch.zeros_like(b)
            self._keep.append((rp, col, val, b, x))
            d = descs[i]
            d.n, d.nnz, d.p = seq.n, seq.nnz, p
            d.w_max, d.s_max, d.tol, d.energy = seq.w_max, min(seq.s_max, 16), seq.tol, seq.energy
            d.row_ptr, d.col, d.val = rp.data_ptr(), col.data_ptr(), val.data_ptr()
            d.b, d.x = b.data_ptr(), x.data_ptr()
        self.total = sum(k[3].shape[0] for k in self._keep)
        self.cfg = make_config(**config)
        h = ctypes.c_void_p()
        torch.cuda.synchronize()
        rc = self.L.pod_cg_batch_create(descs, len(sequences), ctypes.byref(self.cfg), cluster,
                                        ctypes.c_void_p(self.stream.cuda_stream), ctypes.byref(h))
        if rc != 0:
            raise RuntimeError(f"pod_cg_batch_create failed ({rc}): {self.L.pod_cg_last_error(None).decode()}")
        self.h = h

    def solve(self):
        """Solve everything; returns (list of per-system stat dicts, device ms)."""
        st = (_lib.BatchSysStat * self.total)()
        ms = ctypes.c_float(0.0)
        rc = self.L.pod_cg_batch_solve(self.h, st, ctypes.byref(ms))
        out = [{"status": _lib.STATUS_NAMES.get(s.status, s.status), "iters": s.iters, "refinements": s.refinements,
                "w": s.w, "final_relres": s.final_relres, "stage1_relres": s.stage1_relres} for s in st]
        if rc != 0 and rc not in (2, 3, 4, 5):
            raise RuntimeError(self.L.pod_cg_batch_last_error(self.h).decode())
        return out, ms.value

    def set_tiles(self, lanes: int, rows: int):
        """The same inner-loop tiles for every size class (instead of the autotuner's)."""
        a, b = (ctypes.c_int * 3)(lanes, lanes, lanes), (ctypes.c_int * 3)(rows, rows, rows)
        rc = self.L.pod_cg_batch_set_tiles(self.h, a, b)
        if rc != 0:
            raise RuntimeError(self.L.pod_cg_batch_last_error(self.h).decode())

    def solutions(self, i: int) -> torch.Tensor:
        return self._keep[i][4]

    def info(self) -> dict:
        cl, wk = ctypes.c_int(0), ctypes.c_int(0)
        tm = (ctypes.c_float * 3)()
        self.L.pod_cg_batch_info(self.h, ctypes.byref(cl), ctypes.byref(wk), tm)
        lanes, rows, ms = (ctypes.c_int * 3)(), (ctypes.c_int * 3)(), (ctypes.c_float * 12)()
        self.L.pod_cg_batch_tiles(self.h, lanes, rows, ms)
        cands = [(1, 1), (1, 4), (2, 4), (4, 4)]
        classes = ["n<16k", "16k<=n<64k", "n>=64k"]
        tiles = {classes[c]: {"spmv_lanes": lanes[c], "rows_per_thread": rows[c],
                              "ms": {f"lanes{a}_rows{b}": ms[4 * c + k] for k, (a, b) in enumerate(cands)}}
                 for c in range(3)}
        return {"cluster": cl.value, "workers": wk.value, "tune_ms": {2: tm[0], 4: tm[1], 8: tm[2]}, "tiles": tiles}

    def close(self):
        if getattr(self, "h", None):
            self.L.pod_cg_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
