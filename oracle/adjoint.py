"""Derivatives of the Fisher / Arrow-Debreu equilibrium in FP64 (TEST INFRASTRUCTURE ONLY).

Only tests/, __graft_entry__.smoke() and bench.py may import this module.

Not in the paper; derived from its KKT system (Eq. KKT-system-6..9) and Fact 1.
At a non-degenerate equilibrium the tight graph G (edges with x_ij > 0, where
p_j = u_ij y_i, y_i = w_i / t_i) is a forest.  On a component C the log-prices
log p_j and log y_i are node potentials v with v_j - v_i = log u_ij on every
edge; one scale per component is left, fixed by sum_{j in C} p_j = sum_{i in C} w_i
(money conservation, Fact 1(2) per component).  For
    f = sum_j r_j p_j + sum_i g_i t_i      (t_i = w_i e^{-v_i})
with node weights h_j = r_j p_j, h_i = -g_i t_i, H_C = sum_C h, P_C = sum_C p:
    df/dlog u_e = lambda_e, where B^T lambda = h - H_C pi   (pi_j = p_j / P_C on
                  goods, 0 on buyers; B the edge-node incidence, +1 at the good,
                  -1 at the buyer), solved exactly by leaf peeling on a tree;
    df/du_ij    = lambda_e / u_ij on G, 0 elsewhere;
    df/dw_i     = g_i t_i / w_i + H_C / P_C.
Arrow-Debreu with E = I (w = p at a fixed point): mu = r~ + P_w^T mu
(P_w^T mu = H_C(mu)/P_C per agent), reduced exactly to a system over the
tight-graph components (see ad_backward); df/du = the Fisher derivative with
r replaced by mu.  Money is conserved per closed class of components, so the
derivative holds each class's money fixed.
"""
from __future__ import annotations

from collections import defaultdict

import numpy as np

from . import fisher as F


def tight_graph(row_ptr, col, val, w, x, p, t, kappa=1e-7, xrel=1e-9):
    """Edges (entry index, i, j) with x_ij > 0 and p_j <= u_ij y_i (1 + kappa)."""
    rows = F.row_ids(np.asarray(row_ptr))
    y = np.asarray(w) / np.asarray(t)
    uy = np.asarray(val) * y[rows]
    xmax = np.zeros(len(row_ptr) - 1)
    np.maximum.at(xmax, rows, x)
    tight = (x > xrel * xmax[rows]) & (np.asarray(p)[col] <= uy * (1 + kappa))
    idx = np.nonzero(tight)[0]
    return idx, rows[idx], np.asarray(col)[idx]


def _components(n, m, ei, ej):
    parent = list(range(n + m))

    def find(a):
        while parent[a] != a:
            parent[a] = parent[parent[a]]
            a = parent[a]
        return a
    for i, j in zip(ei, ej):
        a, b = find(int(i)), find(n + int(j))
        if a != b:
            parent[a] = b
    return np.array([find(k) for k in range(n + m)])


def fisher_backward(row_ptr, col, val, w, x, p, t, r, g=None, kappa=1e-7):
    """Returns (grad_u [nnz], grad_w [n], info)."""
    row_ptr = np.asarray(row_ptr, dtype=np.int64)
    col = np.asarray(col, dtype=np.int64)
    val = np.asarray(val, dtype=np.float64)
    w = np.asarray(w, dtype=np.float64)
    p = np.asarray(p, dtype=np.float64)
    t = np.asarray(t, dtype=np.float64)
    n, m = len(row_ptr) - 1, len(p)
    r = np.asarray(r, dtype=np.float64)
    g = np.zeros(n) if g is None else np.asarray(g, dtype=np.float64)
    idx, ei, ej = tight_graph(row_ptr, col, val, w, x, p, t, kappa)
    comp = _components(n, m, ei, ej)
    h = np.concatenate([-g * t, r * p])
    isgood = np.concatenate([np.zeros(n, bool), np.ones(m, bool)])
    pv = np.concatenate([np.zeros(n), p])
    HC = defaultdict(float)
    PC = defaultdict(float)
    for k in range(n + m):
        HC[comp[k]] += h[k]
        PC[comp[k]] += pv[k]
    rhs = np.array([h[k] - HC[comp[k]] * (pv[k] / PC[comp[k]]) for k in range(n + m)])
    # leaf peeling on the forest: B^T lambda = rhs
    adj = defaultdict(list)
    for e, (i, j) in enumerate(zip(ei, ej)):
        adj[int(i)].append(e)
        adj[n + int(j)].append(e)
    deg = {k: len(adj[k]) for k in range(n + m)}
    lam = np.zeros(len(idx))
    done = np.zeros(len(idx), bool)
    res = rhs.copy()
    stack = [k for k in range(n + m) if deg[k] == 1]
    cycles = False
    while stack:
        k = stack.pop()
        if deg[k] != 1:
            continue
        e = next(e for e in adj[k] if not done[e])
        # equation of node k: goods +lambda_e, buyers -lambda_e
        lam[e] = res[k] if isgood[k] else -res[k]
        done[e] = True
        deg[k] = 0
        q = (n + int(ej[e])) if k < n else int(ei[e])
        res[k] = 0.0
        res[q] -= lam[e] if isgood[q] else -lam[e]
        deg[q] -= 1
        if deg[q] == 1:
            stack.append(q)
    if not done.all():                      # cycles: least squares on the rest
        cycles = True
        rest = np.nonzero(~done)[0]
        Bt = np.zeros((n + m, len(rest)))
        for c, e in enumerate(rest):
            Bt[n + int(ej[e]), c] = 1.0
            Bt[int(ei[e]), c] = -1.0
        sol = np.linalg.lstsq(Bt, res, rcond=None)[0]
        lam[rest] = sol
        res = res - Bt @ sol
    grad_u = np.zeros(len(val))
    grad_u[idx] = lam / val[idx]
    grad_w = g * t / w + np.array([HC[comp[i]] / PC[comp[i]] for i in range(n)])
    info = dict(edges=len(idx), components=len(set(comp.tolist())), residual=float(np.max(np.abs(res))),
                cycles=cycles)
    return grad_u, grad_w, info


def ad_backward(row_ptr, col, val, x, p, t, r, kappa=1e-7):
    """Arrow-Debreu (E = I) derivative of f = r^T p at the normalised fixed
    point w = p.  With pi_j = p_j / P_C and A mapping agent i to the component
    of buyer i, P_w^T mu = A^T lambda with lambda_C = sum_{j in C} pi_j mu_j, so
    mu = r~ + A^T lambda and lambda solves the K x K system
        (I - Q) lambda = rho,  Q[C, C'] = sum_{j in C, cb(j) = C'} pi_j,
        rho_C = sum_{j in C} pi_j r~_j.
    Q is row-stochastic and every component is recurrent (money is conserved
    per component), so its closed classes are the weakly connected classes of
    the component graph C(good j) - C(buyer j).  Each class keeps its own money
    at a fixed point, so the fixed point is unique only up to the split of money
    between classes; the derivative holds every class's money fixed:
    r~_j = r_j - (sum_class r p / sum_class p), which makes the system
    consistent.  It is solved by least squares."""
    row_ptr = np.asarray(row_ptr, dtype=np.int64)
    col = np.asarray(col, dtype=np.int64)
    n = len(row_ptr) - 1
    m = len(p)
    p = np.asarray(p, dtype=np.float64)
    r = np.asarray(r, dtype=np.float64)
    idx, ei, ej = tight_graph(row_ptr, col, val, p, x, p, t, kappa)
    comp = _components(n, m, ei, ej)
    labels = {c: k for k, c in enumerate(sorted(set(comp.tolist())))}
    K = len(labels)
    cb = np.array([labels[comp[i]] for i in range(n)])          # component of buyer i
    cg = np.array([labels[comp[n + j]] for j in range(m)])      # component of good j
    # closed classes: weakly connected classes of the edges cg(j) - cb(j)
    parent = list(range(K))

    def find(a):
        while parent[a] != a:
            parent[a] = parent[parent[a]]
            a = parent[a]
        return a
    for j in range(m):
        a_, b_ = find(int(cg[j])), find(int(cb[j]))
        if a_ != b_:
            parent[a_] = b_
    cls = np.array([find(c) for c in range(K)])
    gcls = cls[cg]
    rp_cls = defaultdict(float)
    p_cls = defaultdict(float)
    for j in range(m):
        rp_cls[gcls[j]] += r[j] * p[j]
        p_cls[gcls[j]] += p[j]
    rt = np.array([r[j] - rp_cls[gcls[j]] / p_cls[gcls[j]] for j in range(m)])
    P = np.bincount(cg, weights=p, minlength=K)
    pi = p / P[cg]
    Q = np.zeros((K, K))
    np.add.at(Q, (cg, cb), pi)                                   # agent j = good j, its buyer comp
    rho = np.bincount(cg, weights=pi * rt, minlength=K)
    lam = np.linalg.lstsq(np.eye(K) - Q, rho, rcond=None)[0]
    mu = rt + lam[cb]
    gu, _, info = fisher_backward(row_ptr, col, val, p, x, p, t, mu, None, kappa)
    info["ad_components"] = K
    info["ad_classes"] = len(set(cls.tolist()))
    info["ad_residual"] = float(np.max(np.abs((np.eye(K) - Q) @ lam - rho)))
    return gu, mu, info
