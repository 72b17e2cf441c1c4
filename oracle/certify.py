"""Equilibrium certificate in FP64 (TEST INFRASTRUCTURE ONLY).

Only tests/, __graft_entry__.smoke() and bench.py may import this module.

Given any candidate allocation x (on supp U, CSR order) and prices p for the
ORIGINAL (unscaled) market, report how far it is from a Fisher equilibrium.
Each quantity is one of the conditions the paper fixes:

* clearing       max_j |sum_i x_ij - 1|                 (Eq. 1, KKT-system-8)
* budgets        max_i |sum_j p_j x_ij - w_i| / w_i      (follows from KKT-system-1,2,4,5)
* money          |sum p - sum w| / sum w                 (Fact 1(2), Eq. sum-pj)
* bang_per_buck  max_ij (u_ij y_i - p_j)_+ / p_j, y = w/t (KKT-system-7)
* complement     max_ij x_ij (p_j - u_ij y_i)_+ / p_j     (KKT-system-6)
* the relative KKT error of Section 5 on the row-scaled market.
"""
from __future__ import annotations

import numpy as np

from . import fisher as F


def certificate(row_ptr, col, val, w, m, x, p) -> dict:
    row_ptr = np.asarray(row_ptr, dtype=np.int64)
    col = np.asarray(col, dtype=np.int64)
    val = np.asarray(val, dtype=np.float64)
    w = np.asarray(w, dtype=np.float64)
    x = np.asarray(x, dtype=np.float64)
    p = np.asarray(p, dtype=np.float64)
    n = len(row_ptr) - 1
    rows = F.row_ids(row_ptr)
    c = np.bincount(col, weights=x, minlength=m)
    spend = np.bincount(rows, weights=p[col] * x, minlength=n)
    t = np.bincount(rows, weights=val * x, minlength=n)
    y = w / t
    uy = val * y[rows]
    sc = F.preprocess(row_ptr, col, val, w, m)
    k = F.kkt_error(sc, x, p)
    return {
        "clearing": float(np.max(np.abs(c - 1.0))),
        "budgets": float(np.max(np.abs(spend - w) / w)),
        "money": float(abs(p.sum() - w.sum()) / w.sum()),
        "bang_per_buck": float(np.max(np.maximum(uy - p[col], 0.0) / p[col])),
        "complement": float(np.max(x * np.maximum(p[col] - uy, 0.0) / p[col])),
        "r_primal": k.r_primal,
        "r_dual": k.r_dual,
        "r_gap": k.r_gap,
        "kkt": k.kkt,
        "t": t,
    }
