"""Arrow-Debreu fixed point in FP64 (TEST INFRASTRUCTURE ONLY).

Only tests/, __graft_entry__.smoke() and bench.py may import this module.

Alg. 4 (Section 4): starting from budgets w^0, repeat
    p^k = p(w^k)            Fisher equilibrium prices (Alg. 2, oracle.fisher)
    w^{k+1} = E p^k
until max_i |w^{k+1}_i - w^k_i| / max_i |w^k_i| < tol (relative form of the
paper's ||w^{k+1} - w^k|| <= eps).  E has unit column sums, so
sum_i w^{k+1}_i = sum_j p_j = sum_i w^k_i (Fact 1); w^{k+1} is rescaled to the
initial sum to remove the drift of inexact inner solves.  E = None means the
identity (agent i owns one unit of good i).  Each inner solve is warm-started
from the previous allocation and prices.
"""
from __future__ import annotations

import numpy as np

from . import fisher as F


def ad_fixed_point(row_ptr, col, val, w0, m, E=None, outer_tol=1e-6, max_outer=200, inner_tol=1e-10,
                   inner_max_iter=400000, x0=None, p0=None):
    w = np.asarray(w0, dtype=np.float64).copy()
    sum0 = w.sum()
    x, p = x0, p0
    hist = []
    res = None
    for k in range(1, max_outer + 1):
        res = F.pdhcg_solve(row_ptr, col, val, w, m, F.Params(tol=inner_tol, max_iter=inner_max_iter), x0=x, p0=p)
        x, p = res.x, res.p
        w_new = p.copy() if E is None else E @ p
        w_new *= sum0 / w_new.sum()
        change = np.max(np.abs(w_new - w)) / np.max(np.abs(w))
        hist.append(change)
        w = w_new
        if change < outer_tol:
            break
    return dict(p=p, w=w, outer=k, history=hist, x=x, t=res.t, converged=hist[-1] < outer_tol)
