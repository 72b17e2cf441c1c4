"""Python front end of libpdhcg (argument marshalling only).

PyTorch provides device memory and the current CUDA stream; numpy arrays are
passed as host pointers, which the library copies in and out itself.  Every
computation runs in the library's CUDA kernels; if the library is missing the
import of :mod:`capi` raises.
"""
from __future__ import annotations

import ctypes
from dataclasses import dataclass
from typing import Optional

import numpy as np

from . import capi

try:
    import torch
except Exception:  # pragma: no cover - torch is part of the environment
    torch = None


def _is_torch(a) -> bool:
    return torch is not None and isinstance(a, torch.Tensor)


def _ptr(a) -> Optional[int]:
    if a is None:
        return None
    if _is_torch(a):
        return a.data_ptr()
    if isinstance(a, np.ndarray):
        assert a.flags["C_CONTIGUOUS"]
        return a.ctypes.data
    raise TypeError(type(a))


def _contig(a, dtype):
    if a is None:
        return None
    if _is_torch(a):
        return a.to(dtype=getattr(torch, np.dtype(dtype).name)).contiguous()
    return np.ascontiguousarray(a, dtype=dtype)


def _empty_like_loc(ref, n, dtype):
    if _is_torch(ref):
        return torch.empty(n, dtype=getattr(torch, np.dtype(dtype).name), device=ref.device)
    return np.empty(n, dtype=dtype)


def _stream() -> int:
    if torch is not None and torch.cuda.is_available():
        return torch.cuda.current_stream().cuda_stream
    return 0


@dataclass
class SolveOutput:
    p: object
    util: object
    x: object
    info: dict
    status: int


class Solver:
    """Owns one library handle (device workspace) bound to the current stream."""

    def __init__(self, stream: Optional[int] = None):
        capi.load()
        self.h = capi.pdhcg_create(_stream() if stream is None else stream)

    def close(self):
        if getattr(self, "h", None):
            capi.pdhcg_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ------------------------------------------------------------------
    @staticmethod
    def market(row_ptr, col, val, w, m, val_f32=None):
        """Build a pdhcg_market (keeps references to the arrays it points at)."""
        row_ptr = _contig(row_ptr, np.int64)
        col = _contig(col, np.int32)
        if val_f32 is None:
            val_f32 = (_is_torch(val) and val.dtype == torch.float32) or (
                isinstance(val, np.ndarray) and val.dtype == np.float32)
        val = _contig(val, np.float32 if val_f32 else np.float64)
        w = _contig(w, np.float64)
        n = (row_ptr.shape[0] if _is_torch(row_ptr) else len(row_ptr)) - 1
        nnz = int(row_ptr[-1])
        mk = capi.pdhcg_market(n, m, nnz, _ptr(row_ptr), _ptr(col), _ptr(val),
                               capi.PDHCG_VAL_F32 if val_f32 else capi.PDHCG_VAL_F64, _ptr(w))
        mk._keep = (row_ptr, col, val, w)
        return mk

    def fisher_solve(self, row_ptr, col, val, w, m, tol=1e-6, precision="mixed", x0=None, p0=None,
                     return_x=False, check=True, **prm) -> SolveOutput:
        mk = self.market(row_ptr, col, val, w, m)
        mixed = precision == "mixed"
        params = capi.default_params(tol=tol, prec=capi.PDHCG_MIXED if mixed else capi.PDHCG_FP64, **prm)
        ref = mk._keep[0]
        p = _empty_like_loc(ref, m, np.float64)
        util = _empty_like_loc(ref, mk.n, np.float64)
        x = _empty_like_loc(ref, mk.nnz, np.float32 if mixed else np.float64) if return_x else None
        x0c = _contig(x0, np.float32 if mixed else np.float64)
        p0c = _contig(p0, np.float64)
        info = capi.pdhcg_info()
        st = capi.pdhcg_fisher_solve(self.h, mk, params, _ptr(p0c), _ptr(x0c), _ptr(p), _ptr(util), _ptr(x), info)
        if check and st not in (capi.PDHCG_OK, capi.PDHCG_ERR_NOT_CONVERGED):
            raise capi.PdhcgError(st, "pdhcg_fisher_solve")
        return SolveOutput(p, util, x, info.as_dict(), st)

    def fisher_solve_pdhg(self, row_ptr, col, val, w, m, tol=1e-6, restart_every=1000, return_x=False, check=True,
                          **prm) -> SolveOutput:
        """Restarted PDHG (Alg. 1) in FP64 on the GPU: pdhcg_fisher_solve_pdhg."""
        mk = self.market(row_ptr, col, val, w, m)
        params = capi.default_params(tol=tol, prec=capi.PDHCG_FP64, **prm)
        ref = mk._keep[0]
        p = _empty_like_loc(ref, m, np.float64)
        util = _empty_like_loc(ref, mk.n, np.float64)
        x = _empty_like_loc(ref, mk.nnz, np.float64) if return_x else None
        info = capi.pdhcg_info()
        st = capi.pdhcg_fisher_solve_pdhg(self.h, mk, params, restart_every, _ptr(p), _ptr(util), _ptr(x), info)
        if check and st not in (capi.PDHCG_OK, capi.PDHCG_ERR_NOT_CONVERGED):
            raise capi.PdhcgError(st, "pdhcg_fisher_solve_pdhg")
        return SolveOutput(p, util, x, info.as_dict(), st)

    def ad_solve(self, row_ptr, col, val, w0, m, E=None, outer_tol=1e-6, max_outer=100, tol=1e-8,
                 precision="mixed", check=True, **prm):
        mk = self.market(row_ptr, col, val, w0, m)
        mixed = precision == "mixed"
        params = capi.default_params(tol=tol, prec=capi.PDHCG_MIXED if mixed else capi.PDHCG_FP64, **prm)
        ref = mk._keep[0]
        p = _empty_like_loc(ref, m, np.float64)
        wout = _empty_like_loc(ref, mk.n, np.float64)
        e_rp = e_col = e_val = None
        if E is not None:
            e_rp, e_col, e_val = _contig(E[0], np.int64), _contig(E[1], np.int32), _contig(E[2], np.float64)
        outer = ctypes.c_int32(0)
        info = capi.pdhcg_info()
        st = capi.pdhcg_ad_solve(self.h, mk, _ptr(e_rp), _ptr(e_col), _ptr(e_val), outer_tol, max_outer, params,
                                 _ptr(p), _ptr(wout), outer, info)
        if check and st not in (capi.PDHCG_OK, capi.PDHCG_ERR_NOT_CONVERGED):
            raise capi.PdhcgError(st, "pdhcg_ad_solve")
        d = info.as_dict()
        d["outer"] = outer.value
        return SolveOutput(p, wout, None, d, st)

    def solve_batched(self, batch, tol=1e-6, precision="mixed", device=True, check=True, **prm):
        """batch: synth.MarketBatch-like object (row_off, good_off, nnz_off, row_ptr, col, val, w)."""
        B = batch.B
        arrs = dict(row_off=batch.row_off, good_off=batch.good_off, nnz_off=batch.nnz_off, row_ptr=batch.row_ptr)
        conv = {k: _contig(v, np.int64) for k, v in arrs.items()}
        col = _contig(batch.col, np.int32)
        val_f32 = (np.asarray(batch.val).dtype == np.float32) if not _is_torch(batch.val) else batch.val.dtype == torch.float32
        val = _contig(batch.val, np.float32 if val_f32 else np.float64)
        w = _contig(batch.w, np.float64)
        if device and torch is not None and not _is_torch(col):
            dev = torch.device("cuda")
            conv = {k: torch.from_numpy(np.asarray(v)).to(dev) for k, v in conv.items()}
            col, val, w = (torch.from_numpy(np.asarray(a)).to(dev) for a in (col, val, w))
        mixed = precision == "mixed"
        params = capi.default_params(tol=tol, prec=capi.PDHCG_MIXED if mixed else capi.PDHCG_FP64, **prm)
        M = int(batch.good_off[-1])
        N = int(batch.row_off[-1])
        p = _empty_like_loc(col, M, np.float64)
        util = _empty_like_loc(col, N, np.float64)
        infos = (capi.pdhcg_info * B)()
        st = capi.pdhcg_fisher_solve_batched(self.h, B, _ptr(conv["row_off"]), _ptr(conv["good_off"]),
                                             _ptr(conv["nnz_off"]), _ptr(conv["row_ptr"]), _ptr(col), _ptr(val),
                                             capi.PDHCG_VAL_F32 if val_f32 else capi.PDHCG_VAL_F64, _ptr(w),
                                             params, _ptr(p), _ptr(util), ctypes.addressof(infos))
        if check and st not in (capi.PDHCG_OK, capi.PDHCG_ERR_NOT_CONVERGED):
            raise capi.PdhcgError(st, "pdhcg_fisher_solve_batched")
        return SolveOutput(p, util, None, [infos[b].as_dict() for b in range(B)], st)

    def backward(self, grad_p, grad_util=None, nnz=None, n=None):
        gp = _contig(grad_p, np.float64)
        gu = _contig(grad_util, np.float64)
        grad_u = _empty_like_loc(gp, nnz, np.float64)
        grad_w = _empty_like_loc(gp, n, np.float64)
        st = capi.pdhcg_fisher_backward(self.h, _ptr(gp), _ptr(gu), _ptr(grad_u), _ptr(grad_w))
        if st:
            raise capi.PdhcgError(st, "pdhcg_fisher_backward")
        return grad_u, grad_w

    def row_prox(self, row_ptr, col, val, w, m, x_in, p, tau, precision="mixed"):
        mk = self.market(row_ptr, col, val, w, m)
        mixed = precision == "mixed"
        xi = _contig(x_in, np.float32 if mixed else np.float64)
        pp = _contig(p, np.float64)
        x_new = _empty_like_loc(xi, mk.nnz, np.float32 if mixed else np.float64)
        s = _empty_like_loc(xi, mk.n, np.float64)
        c = _empty_like_loc(xi, m, np.float64)
        st = capi.pdhcg_row_prox(self.h, mk, capi.PDHCG_MIXED if mixed else capi.PDHCG_FP64, _ptr(xi), _ptr(pp),
                                 tau, _ptr(x_new), _ptr(s), _ptr(c))
        if st:
            raise capi.PdhcgError(st, "pdhcg_row_prox")
        return x_new, s, c

    def kkt(self, row_ptr, col, val, w, m, x, p, precision="mixed"):
        mk = self.market(row_ptr, col, val, w, m)
        mixed = precision == "mixed"
        xx = _contig(x, np.float32 if mixed else np.float64)
        pp = _contig(p, np.float64)
        out = np.zeros(4)
        st = capi.pdhcg_kkt(self.h, mk, capi.PDHCG_MIXED if mixed else capi.PDHCG_FP64, _ptr(xx), _ptr(pp),
                            out.ctypes.data)
        if st:
            raise capi.PdhcgError(st, "pdhcg_kkt")
        return out


def fisher_solve(row_ptr, col, val, w, m, **kw) -> SolveOutput:
    s = Solver()
    try:
        return s.fisher_solve(row_ptr, col, val, w, m, **kw)
    finally:
        s.close()


if torch is not None:
    class FisherEquilibrium(torch.autograd.Function):
        """Equilibrium prices and utilities as a differentiable function of the
        utilities u (values of a fixed CSR pattern) and budgets w.  Forward runs
        pdhcg_fisher_solve, backward runs pdhcg_fisher_backward (implicit
        differentiation at the equilibrium)."""

        @staticmethod
        def forward(ctx, val, w, row_ptr, col, m, tol, precision):
            solver = Solver()
            out = solver.fisher_solve(row_ptr, col, val, w, m, tol=tol, precision=precision)
            ctx.solver = solver
            ctx.n = w.shape[0]
            ctx.m = int(m)
            ctx.nnz = val.shape[0]
            ctx.val_dtype = val.dtype
            return out.p, out.util

        @staticmethod
        def backward(ctx, grad_p, grad_util):
            gp = grad_p.contiguous() if grad_p is not None else None
            gu = grad_util.contiguous() if grad_util is not None else None
            if gp is None:
                gp = torch.zeros(ctx.m, dtype=torch.float64, device=gu.device if gu is not None else "cpu")
            grad_u, grad_w = ctx.solver.backward(gp, gu, nnz=ctx.nnz, n=ctx.n)
            ctx.solver.close()
            return grad_u.to(ctx.val_dtype), grad_w, None, None, None, None, None
