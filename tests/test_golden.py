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
