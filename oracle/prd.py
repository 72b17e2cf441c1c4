"""Proportional-response dynamics for linear Fisher markets (TEST INFRASTRUCTURE ONLY).

Only tests/, __graft_entry__.smoke() and bench.py may import this module.

An independent published method (Zhang, "Proportional response dynamics in the
Fisher market", TCS 2011; Birnbaum, Devanur and Xiao, EC 2011) used solely to
cross-check the PDHCG oracle's equilibrium on small markets.  Each buyer splits
her budget in proportion to the utility she received from each good:

    p_j = sum_i b_ij,   x_ij = b_ij / p_j,   b_ij <- w_i u_ij x_ij / sum_k u_ik x_ik.

The bids converge to equilibrium spending, so p converges to the unique
equilibrium prices.
"""
from __future__ import annotations

import numpy as np

from . import fisher as F


def proportional_response(row_ptr, col, val, w, m, iters=200000, tol=1e-12):
    row_ptr = np.asarray(row_ptr, dtype=np.int64)
    col = np.asarray(col, dtype=np.int64)
    u = np.asarray(val, dtype=np.float64)
    w = np.asarray(w, dtype=np.float64)
    n = len(row_ptr) - 1
    rows = F.row_ids(row_ptr)
    deg = np.diff(row_ptr)
    b = (w / deg)[rows]                    # uniform initial bids
    p = np.bincount(col, weights=b, minlength=m)
    for it in range(iters):
        x = b / p[col]
        gain = u * x
        t = np.bincount(rows, weights=gain, minlength=n)
        b = w[rows] * gain / t[rows]
        p_new = np.bincount(col, weights=b, minlength=m)
        if np.max(np.abs(p_new - p) / p) < tol:
            p = p_new
            break
        p = p_new
    x = b / p[col]
    t = np.bincount(rows, weights=u * x, minlength=n)
    return p, t, x, it + 1
