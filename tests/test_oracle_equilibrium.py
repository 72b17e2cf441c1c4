"""Pins for the oracle's converged Fisher equilibrium (Alg. 2) against results
that do not come from PDHCG: closed forms, brute-force basic solutions,
proportional-response dynamics and the equilibrium certificate."""
import numpy as np
import pytest

from oracle import closed, certify, fisher as F, prd
from paper_2506_06258_gb300 import synth as S


def _csr_from_dense(U):
    n, m = U.shape
    rows, cols = np.nonzero(U > 0)
    row_ptr = np.zeros(n + 1, dtype=np.int64)
    np.add.at(row_ptr, rows + 1, 1)
    row_ptr = np.cumsum(row_ptr)
    return row_ptr, cols.astype(np.int32), U[rows, cols]


def _solve_dense(U, w, tol=1e-11, **kw):
    row_ptr, col, val = _csr_from_dense(U)
    return F.pdhcg_solve(row_ptr, col, val, w, U.shape[1], F.Params(tol=tol, max_iter=400000, **kw))


@pytest.mark.parametrize("m", [1, 2, 5, 17])
def test_one_buyer(m):
    rng = np.random.default_rng(m)
    u = rng.uniform(0.1, 1, m)
    w = 1.7
    r = _solve_dense(u[None, :], np.array([w]))
    p, t = closed.one_buyer(u, w)
    assert np.allclose(r.p, p, rtol=1e-8)
    assert np.allclose(r.t, t, rtol=1e-8)


@pytest.mark.parametrize("n", [1, 3, 50])
def test_one_good(n):
    rng = np.random.default_rng(10 + n)
    u = rng.uniform(0.1, 1, n)
    w = rng.uniform(0.5, 1.5, n)
    r = _solve_dense(u[:, None], w)
    p, t = closed.one_good(w, u)
    assert np.allclose(r.p, p, rtol=1e-8)
    assert np.allclose(r.t, t, rtol=1e-8)


@pytest.mark.parametrize("nm", [(3, 2), (20, 7), (60, 40)])
def test_rank_one(nm):
    n, m = nm
    mk = S.rank_one_market(n, m, seed=123 + n)
    r = F.pdhcg_solve(mk.row_ptr, mk.col, mk.val, mk.w, m, F.Params(tol=1e-10, max_iter=200000))
    p, t = closed.rank_one(mk.meta["a"], mk.meta["b"], mk.w)
    assert np.allclose(r.p, p, rtol=1e-7)
    assert np.allclose(r.t, t, rtol=1e-7)


@pytest.mark.parametrize("case", [
    (0.9, 0.2, 0.3, 0.8, 1.0, 1.0),    # regime 1: each buys her own good
    (0.9, 0.6, 0.3, 0.8, 1.8, 0.4),    # regime 2: buyer 1 splits
    (0.9, 0.2, 0.6, 0.8, 0.4, 1.9),    # regime 3: buyer 2 splits
    (0.5, 0.5, 0.1, 0.9, 1.0, 1.0),
])
def test_two_by_two(case):
    a, b, c, d, w1, w2 = case
    U = np.array([[a, b], [c, d]])
    w = np.array([w1, w2])
    r = _solve_dense(U, w)
    p, t = closed.two_by_two(a, b, c, d, w1, w2)
    assert np.allclose(r.p, p, rtol=1e-8)
    assert np.allclose(r.t, t, rtol=1e-8)
    pb, tb, _, _ = closed.brute_force(U, w)
    assert np.allclose(pb, p, rtol=1e-10)


@pytest.mark.parametrize("seed", range(12))
def test_tiny_markets_brute_force(seed):
    rng = np.random.default_rng(1000 + seed)
    n, m = int(rng.integers(1, 5)), int(rng.integers(1, 5))
    while True:
        U = rng.uniform(0.05, 1, (n, m)) * (rng.uniform(size=(n, m)) < 0.7)
        if (U > 0).sum() <= 12 and (U > 0).any(1).all() and (U > 0).any(0).all():
            break
    w = rng.uniform(0.5, 1.5, n)
    pb, tb, _, _ = closed.brute_force(U, w)
    r = _solve_dense(U, w)
    assert np.allclose(r.p, pb, rtol=1e-8)
    assert np.allclose(r.t, tb, rtol=1e-8)


@pytest.mark.parametrize("seed", range(3))
def test_proportional_response_agrees(seed):
    mk = S.bernoulli_market(25, 12, 0.4, seed=77 + seed)
    r = F.pdhcg_solve(mk.row_ptr, mk.col, mk.val, mk.w, mk.m, F.Params(tol=1e-10, max_iter=200000))
    pp, tp, xp, it = prd.proportional_response(mk.row_ptr, mk.col, mk.val, mk.w, mk.m, iters=200000, tol=1e-13)
    assert np.allclose(r.p, pp, rtol=1e-5)
    assert np.allclose(r.t, tp, rtol=1e-5)


def test_config1_certificate_and_uniqueness():
    """C1 to relative KKT 1e-8 (the config's tolerance): every condition the
    paper fixes holds, and a second solve from another start gives the same
    prices and utilities (uniqueness, Fact 1)."""
    mk = S.config1()
    r = F.pdhcg_solve(mk.row_ptr, mk.col, mk.val, mk.w, mk.m, F.Params(tol=1e-8))
    assert r.converged and r.kkt.kkt <= 1e-8
    cert = certify.certificate(mk.row_ptr, mk.col, mk.val, mk.w, mk.m, r.x, r.p)
    assert cert["clearing"] < 1e-7
    assert cert["budgets"] < 1e-6
    assert cert["money"] < 1e-7
    assert cert["bang_per_buck"] < 1e-6
    assert cert["complement"] < 1e-6
    rng = np.random.default_rng(5)
    x0 = rng.uniform(0, 2, mk.nnz)
    p0 = rng.uniform(0.5, 3, mk.m)
    r2 = F.pdhcg_solve(mk.row_ptr, mk.col, mk.val, mk.w, mk.m, F.Params(tol=1e-8), x0=x0, p0=p0)
    assert np.allclose(r.p, r2.p, rtol=1e-5)
    assert np.allclose(r.t, r2.t, rtol=1e-5)


def test_kkt_zero_at_exact_equilibrium_and_positive_off_it():
    U = np.array([[0.9, 0.6], [0.3, 0.8]])
    w = np.array([1.8, 0.4])
    pb, tb, S_, b = closed.brute_force(U, w)
    row_ptr, col, val = _csr_from_dense(U)
    x = np.zeros(len(val))
    lookup = {(i, j): k for k, (i, j) in enumerate(zip(np.repeat(np.arange(2), np.diff(row_ptr)), col))}
    for e, (i, j) in enumerate(S_):
        x[lookup[(i, j)]] = b[e] / pb[j]
    sc = F.preprocess(row_ptr, col, val, w, 2)
    k = F.kkt_error(sc, x, pb)
    assert k.kkt < 1e-14
    k2 = F.kkt_error(sc, x, pb * np.array([1.01, 0.99]))
    assert k2.kkt > 1e-4
    k3 = F.kkt_error(sc, x * 1.02, pb)
    assert k3.r_primal > 5e-3


def test_price_step_is_extrapolated_column_sum():
    rng = np.random.default_rng(3)
    mk = S.bernoulli_market(30, 10, 0.5, seed=3)
    xk = rng.uniform(0, 1, mk.nnz)
    xkm1 = rng.uniform(0, 1, mk.nnz)
    p = rng.uniform(0, 1, mk.m)
    sigma = 0.37
    U_k = np.zeros((mk.n, mk.m)); U_km1 = np.zeros((mk.n, mk.m))
    rows = np.repeat(np.arange(mk.n), np.diff(mk.row_ptr))
    U_k[rows, mk.col] = xk; U_km1[rows, mk.col] = xkm1
    expect = p + sigma * ((2 * U_k - U_km1).sum(0) - 1)
    got = F.price_step(p, F.column_sums(mk.col, xk, mk.m), F.column_sums(mk.col, xkm1, mk.m), sigma)
    assert np.allclose(got, expect, rtol=1e-14)
