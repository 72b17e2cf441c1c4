"""Pins for the oracle's Arrow-Debreu fixed point (Alg. 4)."""
import numpy as np
import pytest

from oracle import arrow, certify, closed
from paper_2506_06258_gb300 import synth as S


def test_two_agents_reach_closed_form_fixed_point():
    """u = [[a, b], [c, d]], E = I.  From budgets in the regime where agent 1
    splits her money, the 2x2 Fisher closed form gives p = (a, b) W/(a+b),
    independent of w, and at that point agent 1 is exactly indifferent, so
    p(w) = w there: the iteration must stop at w* = (a, b) W/(a+b)."""
    a, b, c, d = 0.9, 0.6, 0.3, 0.8
    U = np.array([[a, b], [c, d]])
    row_ptr = np.array([0, 2, 4], dtype=np.int64)
    col = np.array([0, 1, 0, 1], dtype=np.int32)
    w0 = np.array([1.8, 0.2])
    p_reg2, _ = closed.two_by_two(a, b, c, d, *w0)
    r = arrow.ad_fixed_point(row_ptr, col, U.ravel(), w0, 2, outer_tol=1e-9, inner_tol=1e-12)
    W = w0.sum()
    w_star = np.array([a, b]) * W / (a + b)
    assert np.allclose(p_reg2, w_star)
    assert np.allclose(r["w"], w_star, rtol=1e-7)
    assert np.allclose(r["p"], w_star, rtol=1e-7)


@pytest.mark.parametrize("seed", [0, 1])
def test_exchange_fixed_point_certificate(seed):
    mk = S.config4(n=40, d_other=5, seed=300 + seed)
    r = arrow.ad_fixed_point(mk.row_ptr, mk.col, mk.val, mk.w, mk.m, outer_tol=1e-8, inner_tol=1e-11)
    assert r["converged"]
    # fixed point: the budgets are the prices of the own goods
    assert np.max(np.abs(r["w"] - r["p"]) / r["p"]) < 1e-6
    # and the Fisher equilibrium conditions hold at those budgets
    cert = certify.certificate(mk.row_ptr, mk.col, mk.val, r["p"], mk.m, r["x"], r["p"])
    assert cert["clearing"] < 1e-7 and cert["bang_per_buck"] < 1e-6 and cert["budgets"] < 1e-5
    # money is conserved: sum p = sum w^0
    assert abs(r["p"].sum() - mk.w.sum()) < 1e-8 * mk.w.sum()


def test_random_endowments_general_E():
    """The paper's own setting (Section 5.3): random sparse endowments with unit
    column sums."""
    rng = np.random.default_rng(4)
    n, m = 30, 20
    mk = S.bernoulli_market(n, m, 0.3, seed=41)
    E = rng.uniform(0, 1, (n, m)) * (rng.uniform(size=(n, m)) < 0.5)
    E[rng.integers(0, n, m), np.arange(m)] += 0.1
    E /= E.sum(0, keepdims=True)
    r = arrow.ad_fixed_point(mk.row_ptr, mk.col, mk.val, np.ones(n), m, E=E, outer_tol=1e-8, inner_tol=1e-11)
    assert r["converged"]
    assert np.max(np.abs(E @ r["p"] - r["w"]) / r["w"]) < 1e-6


def test_generated_random_endowment_instance_reaches_a_certified_fixed_point():
    """synth.ad_random_instance (the law of Section 5.3) at a small size: the
    fixed point converges (inside Thm 2's random-E assumptions), budgets equal
    the value of the endowments at the final prices, and the final Fisher
    solve passes the equilibrium certificate."""
    from oracle import certify
    mk, (erp, ecol, ev) = S.ad_random_instance(40, 16, 0.3, 0.5, seed=12)
    E = np.zeros((mk.n, mk.m))
    E[np.repeat(np.arange(mk.n), np.diff(erp)), ecol] = ev
    r = arrow.ad_fixed_point(mk.row_ptr, mk.col, mk.val, mk.w, mk.m, E=E, outer_tol=1e-9, inner_tol=1e-11)
    assert r["converged"] and r["outer"] < 60
    assert np.max(np.abs(E @ r["p"] - r["w"]) / r["w"]) < 1e-6
    assert np.isclose(r["w"].sum(), mk.m)                     # sum of budgets = value of unit supplies at sum p = m
    c = certify.certificate(mk.row_ptr, mk.col, mk.val, E @ r["p"], mk.m, r["x"], r["p"])
    assert c["clearing"] < 1e-7 and c["bang_per_buck"] < 1e-7
