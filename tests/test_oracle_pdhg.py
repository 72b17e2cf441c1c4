"""Pins for the restarted PDHG oracle (Alg. 1): the closed-form t step against a
scalar minimiser, the operator norm against a dense SVD, and the converged
equilibrium against closed forms, brute force and the PDHCG oracle."""
import numpy as np
import pytest

from oracle import closed, fisher as F, pdhg as P
from paper_2506_06258_gb300 import synth as S


def _csr_from_dense(U):
    n, m = U.shape
    rows, cols = np.nonzero(U > 0)
    row_ptr = np.zeros(n + 1, dtype=np.int64)
    np.add.at(row_ptr, rows + 1, 1)
    return np.cumsum(row_ptr), cols.astype(np.int32), U[rows, cols]


def _pdhg_dense(U, w, tol=1e-10):
    row_ptr, col, val = _csr_from_dense(U)
    return P.pdhg_solve(row_ptr, col, val, w, U.shape[1], P.PdhgParams(tol=tol, restart_every=400))


def test_t_step_is_the_scalar_prox():
    """Eq. update:t against bisection on the optimality condition of
    min_{t>0} -w log t + y t + (t - t_k)^2 / (2 tau), i.e. -w/t + y + (t - t_k)/tau = 0
    (increasing in t), including y tau >> t_k (the branch written without
    cancellation)."""
    rng = np.random.default_rng(0)
    for _ in range(200):
        tk = rng.uniform(0.01, 5.0)
        y = rng.choice([-1.0, 1.0]) * 10.0 ** rng.uniform(-3, 3)
        w = rng.uniform(0.1, 2.0)
        tau = 10.0 ** rng.uniform(-3, 2)
        t = float(P.t_update(np.array(tk), np.array(y), np.array(w), tau))

        def g(s):
            return -w / s + y + (s - tk) / tau

        a, b = 1e-300, 1.0
        while g(b) < 0.0:
            b *= 2.0
        for _ in range(2000):
            c = 0.5 * (a + b)
            if c in (a, b):
                break
            if g(c) < 0.0:
                a = c
            else:
                b = c
        assert abs(t - 0.5 * (a + b)) <= 1e-12 * t


def test_operator_norm_matches_dense_svd():
    mk = S.bernoulli_market(9, 6, 0.5, seed=4)
    sc = F.preprocess(mk.row_ptr, mk.col, mk.val, mk.w, mk.m)
    nnz = len(sc.col)
    K = np.zeros((mk.m + mk.n, nnz + mk.n))
    for q in range(nnz):
        K[sc.col[q], q] = 1.0                       # column sums
        K[mk.m + sc.rows[q], q] = -sc.u[q]          # - u_i^T x_i
    K[mk.m:, nnz:] = np.eye(mk.n)                   # + t_i
    assert np.isclose(P.operator_norm(sc, 2000), np.linalg.svd(K, compute_uv=False)[0], rtol=1e-6)


@pytest.mark.parametrize("m", [1, 3, 9])
def test_one_buyer(m):
    rng = np.random.default_rng(m)
    u = rng.uniform(0.1, 1, m)
    r = _pdhg_dense(u[None, :], np.array([1.3]))
    p, t = closed.one_buyer(u, 1.3)
    assert r.converged
    assert np.allclose(r.p, p, rtol=1e-7)
    assert np.allclose(r.t, t, rtol=1e-7)


@pytest.mark.parametrize("case", [
    (0.9, 0.2, 0.3, 0.8, 1.0, 1.0),
    (0.9, 0.6, 0.3, 0.8, 1.8, 0.4),
    (0.9, 0.2, 0.6, 0.8, 0.4, 1.9),
])
def test_two_by_two(case):
    a, b, c, d, w1, w2 = case
    r = _pdhg_dense(np.array([[a, b], [c, d]]), np.array([w1, w2]))
    p, t = closed.two_by_two(a, b, c, d, w1, w2)
    assert r.converged
    assert np.allclose(r.p, p, rtol=1e-7)
    assert np.allclose(r.t, t, rtol=1e-7)


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_same_equilibrium_as_pdhcg(seed):
    mk = S.bernoulli_market(30, 12, 0.4, seed=20 + seed)
    r = P.pdhg_solve(mk.row_ptr, mk.col, mk.val, mk.w, mk.m, P.PdhgParams(tol=1e-9, restart_every=500))
    ref = F.pdhcg_solve(mk.row_ptr, mk.col, mk.val, mk.w, mk.m, F.Params(tol=1e-11))
    assert r.converged
    assert np.max(np.abs(r.p - ref.p) / ref.p) <= 1e-6
    assert np.max(np.abs(r.t - ref.t) / ref.t) <= 1e-6


def test_restart_period():
    mk = S.bernoulli_market(12, 6, 0.5, seed=3)
    r = P.pdhg_solve(mk.row_ptr, mk.col, mk.val, mk.w, mk.m, P.PdhgParams(tol=1e-30, max_iter=1000,
                                                                           restart_every=300))
    assert r.iters == 1000 and r.restarts == 3
