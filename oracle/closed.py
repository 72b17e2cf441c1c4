"""Closed-form and brute-force Fisher equilibria (TEST INFRASTRUCTURE ONLY).

Only tests/, __graft_entry__.smoke() and bench.py may import this module.

These pin the PDHCG oracle to results that do not come from PDHCG:

* one buyer (n = 1): she receives every good, every good in her support is
  equally good per unit of money, so p_j = w u_j / sum_k u_k;
* one good (m = 1): p = sum_i w_i and x_i = w_i / sum w;
* rank-one utilities u_ij = a_i b_j: with p_j = b_j sum(w)/sum(b) every good has
  the same bang-per-buck a_i sum(b)/sum(w) for every buyer, and x_ij = w_i/sum(w)
  clears the market and exhausts budgets;
* 2 x 2 markets (all four utilities positive): the equilibrium is one of three
  regimes (each buyer buys only "her" good, or one buyer splits);
* tiny markets: enumeration of all spanning forests of supp(U) as candidate
  equilibrium supports (a basic equilibrium allocation has a forest support);
  on a forest the spending b_ij = p_j x_ij, prices and y_i = w_i/t_i solve a
  square linear system (budgets, good revenues, bang-per-buck equalities), and a
  candidate is the equilibrium iff b >= 0 and p_j >= u_ij y_i on all of supp(U)
  (the KKT conditions of the Eisenberg-Gale program, Section 3.2).
"""
from __future__ import annotations

import itertools
from typing import Optional

import numpy as np


def one_buyer(u: np.ndarray, w: float):
    u = np.asarray(u, dtype=np.float64)
    p = w * u / u.sum()
    t = float(u.sum())            # x_j = 1 for all j
    return p, np.array([t])


def one_good(w: np.ndarray, u: np.ndarray):
    w = np.asarray(w, dtype=np.float64)
    u = np.asarray(u, dtype=np.float64)
    p = np.array([w.sum()])
    x = w / w.sum()
    return p, u * x


def rank_one(a: np.ndarray, b: np.ndarray, w: np.ndarray):
    a, b, w = (np.asarray(z, dtype=np.float64) for z in (a, b, w))
    p = b * w.sum() / b.sum()
    t = a * w * b.sum() / w.sum()
    return p, t


def two_by_two(a: float, b: float, c: float, d: float, w1: float, w2: float):
    """u = [[a, b], [c, d]] with a d > b c (buyer 1 relatively prefers good 1).
    Regime 1: each buyer buys only her preferred good, p = (w1, w2), valid when
    buyer 1 does not want good 2 (a/w1 >= b/w2) and buyer 2 does not want good 1
    (d/w2 >= c/w1).  Regime 2 (a/w1 < b/w2): buyer 1 is indifferent and buys
    both goods, buyer 2 only good 2: p proportional to (a, b).  Regime 3: buyer 2
    buys both, p proportional to (c, d)."""
    assert a * d > b * c
    W = w1 + w2
    if a * w2 >= b * w1 and d * w1 >= c * w2:
        p = np.array([w1, w2])
    elif a * w2 < b * w1:
        p = np.array([a, b]) * W / (a + b)
    else:
        p = np.array([c, d]) * W / (c + d)
    # t_i = w_i * (best bang-per-buck max_j u_ij / p_j)
    bpb1 = max(a / p[0], b / p[1])
    bpb2 = max(c / p[0], d / p[1])
    t = np.array([w1 * bpb1, w2 * bpb2])
    return p, t


def _is_forest(edges, n, m):
    parent = list(range(n + m))

    def find(z):
        while parent[z] != z:
            parent[z] = parent[parent[z]]
            z = parent[z]
        return z
    for (i, j) in edges:
        ri, rj = find(i), find(n + j)
        if ri == rj:
            return False
        parent[ri] = rj
    return True


def brute_force(U: np.ndarray, w: np.ndarray, tol: float = 1e-10):
    """Enumerate spanning forests of supp(U) (every buyer and good covered) and
    return the equilibrium (p, t, b) found.  Raises if none or if two candidates
    disagree on prices (uniqueness, Fact 1)."""
    U = np.asarray(U, dtype=np.float64)
    w = np.asarray(w, dtype=np.float64)
    n, m = U.shape
    supp = [(i, j) for i in range(n) for j in range(m) if U[i, j] > 0]
    assert len(supp) <= 16, "brute force is for tiny markets"
    found = []
    for k in range(max(n, m), n + m):
        for S in itertools.combinations(supp, k):
            if {i for i, _ in S} != set(range(n)) or {j for _, j in S} != set(range(m)):
                continue
            if not _is_forest(S, n, m):
                continue
            # unknowns: b_e (k), p_j (m), y_i (n)
            N = k + m + n
            A = np.zeros((N, N))
            rhs = np.zeros(N)
            r = 0
            for i in range(n):                      # sum_j b_ij = w_i
                for e, (ii, _) in enumerate(S):
                    if ii == i:
                        A[r, e] = 1.0
                rhs[r] = w[i]
                r += 1
            for j in range(m):                      # sum_i b_ij - p_j = 0
                for e, (_, jj) in enumerate(S):
                    if jj == j:
                        A[r, e] = 1.0
                A[r, k + j] = -1.0
                r += 1
            for e, (i, j) in enumerate(S):          # p_j - u_ij y_i = 0
                A[r, k + j] = 1.0
                A[r, k + m + i] = -U[i, j]
                r += 1
            try:
                sol = np.linalg.solve(A, rhs)
            except np.linalg.LinAlgError:
                continue
            b, p, y = sol[:k], sol[k:k + m], sol[k + m:]
            if (b < -tol).any() or (p <= 0).any() or (y <= 0).any():
                continue
            ok = all(p[j] >= U[i, j] * y[i] * (1 - 1e-9) for (i, j) in supp)
            if ok:
                found.append((p, w / y, S, b))
    if not found:
        raise AssertionError("no equilibrium support found")
    p0 = found[0][0]
    for p, _, _, _ in found[1:]:
        assert np.allclose(p, p0, rtol=1e-9, atol=1e-12), "non-unique prices"
    p, t, S, b = found[0]
    return p, t, S, b
