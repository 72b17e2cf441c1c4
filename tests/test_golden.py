"""The stored C1 equilibrium (tests/golden/c1_equilibrium.txt) against the
equilibrium conditions themselves and against the oracle that wrote it.

The certificate is independent of any solver: market clearing (Eq. 1), budgets
spent, bang-per-buck optimality and complementarity (the KKT system of Section
2) on the stored point; a planted error in the stored prices must fail it."""
import numpy as np

from oracle import certify, fisher as F
from paper_2506_06258_gb300 import synth as S
from tests.golden_data import load_equilibrium


def _c1():
    return S.config1(), load_equilibrium()


def test_stored_point_is_an_equilibrium():
    mk, g = _c1()
    assert len(g["p"]) == mk.m and len(g["t"]) == mk.n and len(g["x"]) == mk.nnz
    c = certify.certificate(mk.row_ptr, mk.col, mk.val, mk.w, mk.m, g["x"], g["p"])
    for k in ("clearing", "budgets", "money", "bang_per_buck", "complement", "kkt"):
        assert c[k] <= 1e-11, (k, c[k])
    # stored utilities are u_i^T x_i of the stored allocation
    assert np.allclose(c["t"], g["t"], rtol=1e-12, atol=0.0)


def test_planted_price_error_fails_the_certificate():
    mk, g = _c1()
    p = g["p"].copy()
    j0, j1 = int(np.argmin(p)), int(np.argmax(p))
    p[j0], p[j1] = p[j1], p[j0]
    c = certify.certificate(mk.row_ptr, mk.col, mk.val, mk.w, mk.m, g["x"], p)
    assert c["bang_per_buck"] > 1e-3 or c["budgets"] > 1e-3


def test_oracle_reproduces_stored_prices():
    mk, g = _c1()
    r = F.pdhcg_solve(mk.row_ptr, mk.col, mk.val, mk.w, mk.m, F.Params(tol=1e-11))
    assert r.converged
    assert np.max(np.abs(r.p - g["p"]) / g["p"]) <= 1e-8
    assert np.max(np.abs(r.t - g["t"]) / g["t"]) <= 1e-8


def _c3law():
    import sys, os
    sys.path.insert(0, os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden"))
    from make_golden import c3law_market
    return c3law_market(), load_equilibrium("c3law_equilibrium.txt")


def test_stored_c3law_prices_satisfy_the_dual_equilibrium_conditions():
    """The stored benchmark-law equilibrium (p, t; no allocation is stored) meets
    the conditions that involve p and t alone: money is conserved (sum p =
    sum w, Fact 1), no buyer sees a bang-per-buck above y_i = w_i / t_i
    (p_j >= u_ij y_i, the KKT system of Section 2), and every buyer's best
    bang-per-buck is reached (each buyer spends on some good with p_j = u_ij y_i)."""
    mk, g = _c3law()
    p, t = g["p"], g["t"]
    assert len(p) == mk.m and len(t) == mk.n
    val = mk.val.astype(np.float64)
    rows = F.row_ids(mk.row_ptr)
    y = mk.w / t
    ratio = val * y[rows] / p[mk.col]                 # u_ij y_i / p_j <= 1, = 1 on the support
    best = np.full(mk.n, -np.inf)
    np.maximum.at(best, rows, ratio)
    assert abs(p.sum() - mk.w.sum()) / mk.w.sum() <= 1e-9
    assert np.max(ratio) <= 1 + 1e-7
    assert np.max(np.abs(best - 1.0)) <= 1e-7
    # a planted 1e-4 error in one price breaks the conditions
    j = int(np.argmax(p))
    p2 = p.copy()
    p2[j] *= 1 - 1e-4
    ratio2 = val * y[rows] / p2[mk.col]
    assert np.max(ratio2) > 1 + 1e-5
