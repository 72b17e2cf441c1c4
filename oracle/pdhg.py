"""Restarted PDHG (Alg. 1) for the linear Fisher market in FP64.

TEST INFRASTRUCTURE ONLY: only tests/, __graft_entry__.smoke() and bench.py may
import this module.

The saddle-point form of Section 2 keeps the buyer utilities t as primal
variables beside x, and their defining constraints t_i = sum_j u_ij x_ij carry
dual variables y beside the prices p.  One PDHG step (Eq. update-rule) is
separable and closed-form:

  p_j <- p_j + sigma (sum_i (2 x^k - x^{k-1})_ij - 1)                 (Eq. update:py)
  y_i <- y_i + sigma (2 t^k_i - t^{k-1}_i - sum_j u_ij (2 x^k - x^{k-1})_ij)
  t_i <- positive root of t^2 + (tau y_i - t^k_i) t - tau w_i = 0       (Eq. update:t)
  x_ij <- [x^k_ij - tau (p_j - u_ij y_i)]_+                             (Eq. update:x)

Alg. 1 runs K such steps, averaging the iterates with weights 1/(k+1), and
restarts from the average.  Step sizes are constant: tau = eta / omega,
sigma = eta * omega with eta = 0.9 / ||K||_2 (K the constraint operator of
(x, t), its norm by power iteration) and omega = ||p^0|| / ||(x^0, t^0)||, the
primal weight of Section 5 held fixed.  The market is row-scaled first as in
oracle.fisher (Section 5, "Preprocessing"); the stopping test is the relative
KKT error of oracle.fisher.kkt_error on (x, p).
"""
from __future__ import annotations

import math
import time
from dataclasses import dataclass

import numpy as np

from . import fisher as F


@dataclass
class PdhgParams:
    tol: float = 1e-8
    max_iter: int = 400000
    restart_every: int = 1000      # K of Alg. 1
    check_every: int = 64          # KKT evaluation period
    eta_scale: float = 0.9
    power_iters: int = 200


def operator_norm(sc: F.Scaled, iters: int = 200, seed: int = 0) -> float:
    """||K||_2 for K(x, t) = (sum_i x_ij, t_i - sum_j u_ij x_ij), by power
    iteration on K^T K."""
    rng = np.random.default_rng(seed)
    x = rng.uniform(0.5, 1.5, len(sc.col))
    t = rng.uniform(0.5, 1.5, sc.n)
    lam = 0.0
    for _ in range(iters):
        nrm = math.sqrt(float(x @ x + t @ t))
        x, t = x / nrm, t / nrm
        q = F.column_sums(sc.col, x, sc.m)                 # C x
        z = t - F.row_dot(sc.row_ptr, sc.u, x)             # t - U x
        # K^T (q, z) = (C^T q - U^T z, z)
        x, t = q[sc.col] - sc.u * z[sc.rows], z
        lam = math.sqrt(float(x @ x + t @ t))
    return math.sqrt(lam)


def t_update(t_k, y, w, tau):
    """Eq. update:t: argmin_{t>0} -w log t + y t + (t - t_k)^2 / (2 tau), the
    positive root of t^2 + (tau y - t_k) t - tau w = 0 (cancellation-free)."""
    b = tau * y - t_k
    disc = np.sqrt(b * b + 4.0 * tau * w)
    return np.where(b <= 0.0, 0.5 * (disc - b), (2.0 * tau * w) / (disc + b))


def pdhg_solve(row_ptr, col, val, w, m, prm: PdhgParams | None = None) -> F.Result:
    prm = prm or PdhgParams()
    t_start = time.perf_counter()
    err = F.validate(row_ptr, col, val, w, m)
    if err:
        raise ValueError(err)
    sc = F.preprocess(row_ptr, col, val, w, m)
    x, p = F.initial_point(sc)
    t = F.row_dot(sc.row_ptr, sc.u, x)
    y = sc.w / t
    normK = operator_norm(sc, prm.power_iters) * 1.01
    eta = prm.eta_scale / normK
    omega = float(np.linalg.norm(p) / math.sqrt(float(x @ x + t @ t)))
    tau, sigma = eta / omega, eta * omega
    x_prev, t_prev = x.copy(), t.copy()
    xb, tb, pb, yb = x.copy(), t.copy(), p.copy(), y.copy()
    kk = F.kkt_error(sc, x, p)
    best = (kk.kkt, x.copy(), p.copy())
    total = inner = restarts = 0
    converged = kk.kkt <= prm.tol
    while not converged and total < prm.max_iter:
        # dual step at the extrapolated primal point (Eq. update:py)
        xe = 2.0 * x - x_prev
        te = 2.0 * t - t_prev
        p_new = p + sigma * (F.column_sums(sc.col, xe, sc.m) - 1.0)
        y_new = y + sigma * (te - F.row_dot(sc.row_ptr, sc.u, xe))
        # primal step (Eq. update:t, Eq. update:x)
        t_new = t_update(t, y_new, sc.w, tau)
        x_new = np.maximum(x - tau * (p_new[sc.col] - sc.u * y_new[sc.rows]), 0.0)
        x_prev, t_prev = x, t
        x, t, p, y = x_new, t_new, p_new, y_new
        inner += 1
        total += 1
        wgt = 1.0 / inner
        xb += wgt * (x - xb)
        tb += wgt * (t - tb)
        pb += wgt * (p - pb)
        yb += wgt * (y - yb)
        if total % prm.check_every == 0:
            for cx, cp in ((x, p), (xb, pb)):
                k = F.kkt_error(sc, cx, cp)
                if k.kkt < best[0]:
                    best = (k.kkt, cx.copy(), cp.copy())
            if best[0] <= prm.tol:
                converged = True
                break
        if inner == prm.restart_every:
            # restart from the average (Alg. 1)
            x, t, p, y = xb.copy(), tb.copy(), pb.copy(), yb.copy()
            x_prev, t_prev = x.copy(), t.copy()
            inner = 0
            restarts += 1
    _, xbest, pbest = best
    kb = F.kkt_error(sc, xbest, pbest)
    tt = F.row_dot(sc.row_ptr, sc.u, xbest) * sc.rowmax
    return F.Result(pbest, tt, xbest, kb, total, total, restarts, kb.kkt <= prm.tol,
                    time.perf_counter() - t_start, [])
