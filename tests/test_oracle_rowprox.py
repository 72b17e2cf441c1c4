"""Pins for the oracle's row subproblem (Section 2.2) against independent checks:
brute force over active sets, the subproblem's own KKT conditions, a generic
bound-constrained optimiser, and the paper's bisection / 32-section searches."""
import itertools
import math

import numpy as np
import pytest

from oracle import fisher as F


def _random_row(rng, d, scale_tau=1.0):
    u = rng.uniform(0.05, 1.0, d)
    xk = rng.uniform(0.0, 1.0, d) * (rng.uniform(size=d) < 0.7)
    p = rng.uniform(0.1, 3.0, d)
    tau = scale_tau * rng.uniform(0.01, 2.0)
    w = rng.uniform(0.2, 2.0)
    a = xk - tau * p
    cc = tau * w * u
    return u, xk, p, tau, w, a, cc


def _brute(u, a, cc):
    """Scan every active set S: s solves s = A_S + C_S/s; keep the s whose own
    active set is S."""
    d = len(u)
    sols = []
    for r in range(1, d + 1):
        for S in itertools.combinations(range(d), r):
            S = list(S)
            A = float(np.sum(u[S] * a[S]))
            C = float(np.sum(u[S] * cc[S]))
            s = (A + math.sqrt(A * A + 4 * C)) / 2
            if s <= 0:
                continue
            act = set(np.nonzero(a + cc / s > 0)[0].tolist())
            if act == set(S):
                sols.append(s)
    return sols


@pytest.mark.parametrize("seed", range(40))
def test_exact_matches_active_set_brute_force(seed):
    rng = np.random.default_rng(seed)
    d = int(rng.integers(1, 11))
    u, xk, p, tau, w, a, cc = _random_row(rng, d)
    sols = _brute(u, a, cc)
    assert len(sols) >= 1
    s, x = F.row_prox_exact_single(u, a, cc)
    for sb in sols:  # all consistent active sets give the same root (uniqueness)
        assert abs(sb - s) <= 1e-12 * s
    assert abs(F.phi(s, u, a, cc)) <= 1e-13 * s


@pytest.mark.parametrize("seed", range(20))
def test_subproblem_kkt_conditions(seed):
    """x solves min_{x>=0} -w log(u^T x) + p^T x + |x - x^k|^2/(2 tau): for x_j > 0
    the gradient -w u_j/s + p_j + (x_j - x^k_j)/tau vanishes, for x_j = 0 it is >= 0."""
    rng = np.random.default_rng(100 + seed)
    d = int(rng.integers(1, 40))
    u, xk, p, tau, w, a, cc = _random_row(rng, d)
    s, x = F.row_prox_exact_single(u, a, cc)
    assert abs(np.dot(u, x) - s) <= 1e-12 * s
    g = -w * u / s + p + (x - xk) / tau
    scale = np.abs(w * u / s) + np.abs(p) + np.abs(xk / tau) + 1.0
    pos = x > 0
    assert np.all(np.abs(g[pos]) <= 1e-10 * scale[pos])
    assert np.all(g[~pos] >= -1e-10 * scale[~pos])


@pytest.mark.parametrize("seed", range(6))
def test_subproblem_against_generic_optimizer(seed):
    """Independent solver: scipy L-BFGS-B on the row objective as printed in
    Section 2.2 (with the utility factor inside the log's gradient)."""
    scipy_opt = pytest.importorskip("scipy.optimize")
    rng = np.random.default_rng(200 + seed)
    d = 8
    u, xk, p, tau, w, a, cc = _random_row(rng, d)

    def f(x):
        s = float(np.dot(u, x))
        return -w * math.log(s) + float(np.dot(p, x)) + float(np.dot(x - xk, x - xk)) / (2 * tau)

    def grad(x):
        s = float(np.dot(u, x))
        return -w * u / s + p + (x - xk) / tau

    x0 = np.maximum(xk, 0.0) + 0.1
    res = scipy_opt.minimize(f, x0, jac=grad, method="L-BFGS-B", bounds=[(0, None)] * d,
                             options=dict(ftol=1e-15, gtol=1e-12, maxiter=10000))
    s, x = F.row_prox_exact_single(u, a, cc)
    assert f(x) <= res.fun + 1e-10
    assert np.allclose(x, res.x, atol=2e-5)


def test_dropping_utility_factor_is_detectably_wrong():
    """The printed update tau w_i / s (no u_ij) does not satisfy the subproblem's
    optimality conditions when utilities differ, so the test above separates the
    two readings."""
    rng = np.random.default_rng(7)
    u, xk, p, tau, w, a, cc = _random_row(rng, 6)
    u = np.array([0.2, 0.4, 0.6, 0.8, 1.0, 0.3])
    cc_wrong = tau * w * np.ones_like(u)
    s, x = F.row_prox_exact_single(u, a, cc_wrong)
    g = -w * u / np.dot(u, x) + p + (x - xk) / tau
    assert np.max(np.abs(g[x > 0])) > 1e-3


@pytest.mark.parametrize("seed", range(10))
def test_vectorised_matches_single(seed):
    rng = np.random.default_rng(300 + seed)
    n = 30
    deg = rng.integers(1, 25, n)
    row_ptr = np.concatenate(([0], np.cumsum(deg))).astype(np.int64)
    nnz = int(row_ptr[-1])
    u = rng.uniform(0.05, 1, nnz)
    a = rng.normal(0, 1, nnz)
    cc = rng.uniform(0.01, 1, nnz)
    s, x = F.row_prox_exact(F.degree_groups(row_ptr), n, u, a, cc)
    for i in range(n):
        b, e = row_ptr[i], row_ptr[i + 1]
        si, xi = F.row_prox_exact_single(u[b:e], a[b:e], cc[b:e])
        assert abs(si - s[i]) <= 1e-12 * si
        assert np.allclose(xi, x[b:e], rtol=1e-12, atol=1e-15)


@pytest.mark.parametrize("seed", range(10))
def test_phi_monotone_and_bracket_property(seed):
    """phi is increasing; for s < s*, s~ > s* and for s > s*, s~ < s* (Section 2.2)."""
    rng = np.random.default_rng(400 + seed)
    u, xk, p, tau, w, a, cc = _random_row(rng, 20)
    s_star, _ = F.row_prox_exact_single(u, a, cc)
    grid = s_star * np.exp(np.linspace(-3, 3, 61))
    ph = np.array([F.phi(s, u, a, cc) for s in grid])
    assert np.all(np.diff(ph) > 0)
    for s in grid:
        st = float(np.dot(u, np.maximum(a + cc / s, 0)))
        if s < s_star * (1 - 1e-12):
            assert st >= s_star * (1 - 1e-12)
        elif s > s_star * (1 + 1e-12):
            assert st <= s_star * (1 + 1e-12)


@pytest.mark.parametrize("sections", [2, 4, 32])
def test_searches_reach_exact_root(sections):
    rng = np.random.default_rng(500 + sections)
    for _ in range(10):
        u, xk, p, tau, w, a, cc = _random_row(rng, 30)
        s_star, x_star = F.row_prox_exact_single(u, a, cc)
        s0 = max(float(np.dot(u, np.maximum(xk, 0))), 1e-3)
        s_b, _, _ = F.bisection_search(u, a, cc, s0, eps=1e-13)
        s_k, _, _ = F.section_search(u, a, cc, s0, sections=sections, eps=1e-13)
        assert abs(s_b - s_star) <= 1e-11 * s_star
        assert abs(s_k - s_star) <= 1e-11 * s_star
