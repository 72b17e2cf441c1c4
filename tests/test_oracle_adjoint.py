"""Pins for the oracle's equilibrium derivatives: the 2x2 analytic derivative,
homogeneity (Euler) identities, and central finite differences of oracle solves."""
import numpy as np
import pytest

from oracle import adjoint as A, arrow, fisher as F
from paper_2506_06258_gb300 import synth as S


def _solve(row_ptr, col, val, w, m, tol=1e-13):
    return F.pdhcg_solve(row_ptr, col, val, w, m, F.Params(tol=tol, max_iter=500000))


def test_two_by_two_regime2_analytic():
    """Regime 2 (buyer 1 splits): p = (a, b) W/(a+b), so dp1/da = b W/(a+b)^2,
    dp1/db = -a W/(a+b)^2, dp1/dc = dp1/dd = 0, dp1/dw_i = a/(a+b)."""
    a, b, c, d, w1, w2 = 0.9, 0.6, 0.3, 0.8, 1.8, 0.4
    row_ptr = np.array([0, 2, 4]); col = np.array([0, 1, 0, 1]); val = np.array([a, b, c, d])
    w = np.array([w1, w2]); W = w1 + w2
    res = _solve(row_ptr, col, val, w, 2)
    gu, gw, info = A.fisher_backward(row_ptr, col, val, w, res.x, res.p, res.t, r=np.array([1.0, 0.0]))
    assert np.allclose(gu, [b * W / (a + b) ** 2, -a * W / (a + b) ** 2, 0.0, 0.0], atol=1e-7)
    assert np.allclose(gw, [a / (a + b)] * 2, atol=1e-7)


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_against_central_differences(seed):
    mk = S.bernoulli_market(14, 8, 0.45, seed=600 + seed)
    rng = np.random.default_rng(seed)
    r = rng.normal(size=mk.m)
    g = rng.normal(size=mk.n)
    res = _solve(mk.row_ptr, mk.col, mk.val, mk.w, mk.m)
    gu, gw, info = A.fisher_backward(mk.row_ptr, mk.col, mk.val, mk.w, res.x, res.p, res.t, r, g)
    assert info["residual"] < 1e-10

    def f(val, w):
        s = _solve(mk.row_ptr, mk.col, val, w, mk.m)
        return r @ s.p + g @ s.t

    tight = np.nonzero(gu)[0]
    off = np.nonzero(gu == 0)[0]
    picks = list(rng.choice(tight, size=min(6, len(tight)), replace=False)) + \
        list(rng.choice(off, size=min(4, len(off)), replace=False))
    for e in picks:
        hstep = 1e-6 * mk.val[e]
        vp, vm = mk.val.copy(), mk.val.copy()
        vp[e] += hstep; vm[e] -= hstep
        fd = (f(vp, mk.w) - f(vm, mk.w)) / (2 * hstep)
        assert abs(fd - gu[e]) <= 2e-5 * max(1.0, abs(fd)), (e, fd, gu[e])
    for i in rng.choice(mk.n, size=4, replace=False):
        hstep = 1e-6 * mk.w[i]
        wp, wm = mk.w.copy(), mk.w.copy()
        wp[i] += hstep; wm[i] -= hstep
        fd = (f(mk.val, wp) - f(mk.val, wm)) / (2 * hstep)
        assert abs(fd - gw[i]) <= 2e-5 * max(1.0, abs(fd))


def test_euler_identities():
    """Prices are degree-0 homogeneous in each buyer's utility row (t_i degree 1)
    and degree-1 in w (allocations, hence t, degree 0):
    sum_j u_ij df/du_ij = g_i t_i and sum_i w_i df/dw_i = r.p."""
    mk = S.bernoulli_market(30, 12, 0.3, seed=61)
    rng = np.random.default_rng(1)
    r, g = rng.normal(size=mk.m), rng.normal(size=mk.n)
    res = _solve(mk.row_ptr, mk.col, mk.val, mk.w, mk.m)
    gu, gw, _ = A.fisher_backward(mk.row_ptr, mk.col, mk.val, mk.w, res.x, res.p, res.t, r, g)
    rows = F.row_ids(mk.row_ptr)
    per_row = np.bincount(rows, weights=mk.val * gu, minlength=mk.n)
    assert np.allclose(per_row, g * res.t, atol=1e-8)
    assert abs(mk.w @ gw - r @ res.p) < 1e-8


def test_arrow_debreu_against_central_differences():
    """E = I exchange economies split into closed classes that each keep their
    money, so the fixed point is pinned down by where the iteration starts.  The
    derivative holds every class's money fixed; the finite differences do the
    same by restarting the perturbed iteration at the equilibrium."""
    mk = S.config4(n=40, d_other=5, seed=700)
    rng = np.random.default_rng(2)
    r = rng.normal(size=mk.m)
    kw = dict(outer_tol=1e-12, inner_tol=1e-13, max_outer=400)
    ad = arrow.ad_fixed_point(mk.row_ptr, mk.col, mk.val, mk.w, mk.m, **kw)
    gu, mu, info = A.ad_backward(mk.row_ptr, mk.col, mk.val, ad["x"], ad["p"], ad["t"], r)
    assert ad["converged"] and info["residual"] < 1e-9 and info["ad_residual"] < 1e-10
    assert info["ad_classes"] > 1
    picks = np.nonzero(gu)[0][:5]
    for e in picks:
        hstep = 1e-6 * mk.val[e]
        vp, vm = mk.val.copy(), mk.val.copy()
        vp[e] += hstep; vm[e] -= hstep
        start = dict(x0=ad["x"], p0=ad["p"])
        fp = r @ arrow.ad_fixed_point(mk.row_ptr, mk.col, vp, ad["w"], mk.m, **kw, **start)["p"]
        fm = r @ arrow.ad_fixed_point(mk.row_ptr, mk.col, vm, ad["w"], mk.m, **kw, **start)["p"]
        fd = (fp - fm) / (2 * hstep)
        assert abs(fd - gu[e]) <= 1e-4 * max(1.0, abs(fd)), (e, fd, gu[e])


def test_arrow_debreu_tiny_exchange_cycles():
    """With E = I (outside the random-endowment assumptions of Theorem 2) the
    plain fixed-point iteration need not converge: this 12-agent economy keeps
    a relative budget change of about 4e-3 forever, and the oracle says so."""
    mk = S.config4(n=12, d_other=3, seed=700)
    ad = arrow.ad_fixed_point(mk.row_ptr, mk.col, mk.val, mk.w, mk.m, outer_tol=1e-9, inner_tol=1e-11,
                              max_outer=60)
    assert not ad["converged"]
    assert 1e-3 < ad["history"][-1] < 1e-2
