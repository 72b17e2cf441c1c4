"""Degenerate and boundary cases of the GPU path against closed forms and the
FP64 oracle: one buyer, one good, the three regimes of the 2x2 market, buyers
with a single good, rows long enough for the chunked row path, and batches of
tiny markets (down to 1x1)."""
import numpy as np
import pytest

from oracle import closed, fisher as F
from paper_2506_06258_gb300 import synth as S
from tests.gpu_util import dev, host, torch_cuda

pytestmark = pytest.mark.gpu

# (precision, KKT tolerance of the solve, relative tolerance on p and t)
PRECS = [("fp64", 1e-9, 1e-7), ("mixed", 1e-7, 1e-5)]


@pytest.fixture(scope="module")
def solver():
    torch_cuda()
    from paper_2506_06258_gb300 import api
    s = api.Solver()
    yield s
    s.close()


def _dense(U, w):
    n, m = U.shape
    rows, cols = np.nonzero(U > 0)
    row_ptr = np.zeros(n + 1, dtype=np.int64)
    np.add.at(row_ptr, rows + 1, 1)
    return S.Market(n, m, np.cumsum(row_ptr), cols.astype(np.int32), U[rows, cols].astype(np.float64),
                    np.asarray(w, dtype=np.float64), "dense")


def _solve(solver, mk, prec, tol):
    val = mk.val.astype(np.float32) if prec == "mixed" else mk.val
    return solver.fisher_solve(dev(mk.row_ptr), dev(mk.col), dev(val), dev(mk.w), mk.m, tol=tol, precision=prec)


def _market_of(mk, prec):
    """The market the precision actually solves (FP32 utilities for MIXED)."""
    if prec == "mixed":
        return S.Market(mk.n, mk.m, mk.row_ptr, mk.col, mk.val.astype(np.float32).astype(np.float64), mk.w, mk.name)
    return mk


@pytest.mark.parametrize("prec,tol,rtol", PRECS)
@pytest.mark.parametrize("m", [1, 7, 300])
def test_one_buyer(solver, prec, tol, rtol, m):
    rng = np.random.default_rng(m)
    mk = _market_of(_dense(rng.uniform(0.1, 1.0, (1, m)), [1.7]), prec)
    out = _solve(solver, mk, prec, tol)
    p, t = closed.one_buyer(mk.val, 1.7)
    assert out.status == 0
    assert np.allclose(host(out.p), p, rtol=rtol)
    assert np.allclose(host(out.util), t, rtol=rtol)


@pytest.mark.parametrize("prec,tol,rtol", PRECS)
@pytest.mark.parametrize("n", [1, 5, 400])
def test_one_good(solver, prec, tol, rtol, n):
    rng = np.random.default_rng(10 + n)
    w = rng.uniform(0.5, 1.5, n)
    mk = _market_of(_dense(rng.uniform(0.1, 1.0, (n, 1)), w), prec)
    out = _solve(solver, mk, prec, tol)
    p, t = closed.one_good(w, mk.val)
    assert out.status == 0
    assert np.allclose(host(out.p), p, rtol=rtol)
    assert np.allclose(host(out.util), t, rtol=rtol)


@pytest.mark.parametrize("prec,tol,rtol", PRECS)
@pytest.mark.parametrize("case", [
    (0.9, 0.2, 0.3, 0.8, 1.0, 1.0),    # each buyer buys her own good
    (0.9, 0.6, 0.3, 0.8, 1.8, 0.4),    # buyer 1 splits
    (0.9, 0.2, 0.6, 0.8, 0.4, 1.9),    # buyer 2 splits
])
def test_two_by_two(solver, prec, tol, rtol, case):
    a, b, c, d, w1, w2 = case
    mk = _market_of(_dense(np.array([[a, b], [c, d]]), [w1, w2]), prec)
    u = mk.val
    out = _solve(solver, mk, prec, tol)
    p, t = closed.two_by_two(u[0], u[1], u[2], u[3], w1, w2)
    assert out.status == 0
    assert np.allclose(host(out.p), p, rtol=rtol)
    assert np.allclose(host(out.util), t, rtol=rtol)


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-8), ("mixed", 2e-7)])
def test_single_good_buyers_and_long_rows(solver, prec, tol):
    """Half the buyers want one good each; a few buyers want 300-900 goods
    (the chunked row path); the rest are ordinary.  On this market the price
    error is about 9x the relative KKT error even for the FP64 oracle (5.7e-6
    at KKT 6.2e-7), so both precisions are solved below 1e-6 to test a 1e-5
    price bound."""
    rng = np.random.default_rng(4)
    n, m = 600, 1000
    deg = np.where(np.arange(n) % 2 == 0, 1, rng.integers(2, 40, n))
    deg[:6] = rng.integers(300, 900, 6)
    row_ptr = np.concatenate(([0], np.cumsum(deg))).astype(np.int64)
    col = np.concatenate([np.sort(rng.choice(m, size=d, replace=False)) for d in deg]).astype(np.int32)
    val = rng.uniform(0.05, 1.0, len(col))
    mk = S.repair_assumption1(S.Market(n, m, row_ptr, col, val, rng.uniform(0.5, 1.5, n), "edge"), 4, 0, 0.05, 1.0)
    mk = _market_of(mk, prec)
    out = _solve(solver, mk, prec, tol)
    ref = F.pdhcg_solve(mk.row_ptr, mk.col, mk.val, mk.w, mk.m, F.Params(tol=1e-10, max_iter=400000))
    assert out.status == 0
    assert np.max(np.abs(host(out.p) - ref.p) / ref.p) <= 1e-5
    assert np.max(np.abs(host(out.util) - ref.t) / ref.t) <= 1e-5


def test_mixed_is_deterministic(solver):
    """Exact fixed-point column sums and counter-based rounding bits: two MIXED
    solves of the same market agree bit for bit."""
    mk = S.bernoulli_market(300, 90, 0.2, seed=12)
    a = _solve(solver, mk, "mixed", 1e-6)
    b = _solve(solver, mk, "mixed", 1e-6)
    assert np.array_equal(host(a.p), host(b.p))
    assert np.array_equal(host(a.util), host(b.util))
    assert a.info["iters"] == b.info["iters"]


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-9), ("mixed", 2e-7)])
def test_batch_of_tiny_markets(solver, prec, tol):
    """A batch mixing 1x1, 1xm, nx1 and 2x2 markets with ordinary ones."""
    rng = np.random.default_rng(8)
    mks = [_dense(np.array([[0.7]]), [1.3]),
           _dense(rng.uniform(0.1, 1, (1, 6)), [0.9]),
           _dense(rng.uniform(0.1, 1, (5, 1)), rng.uniform(0.5, 1.5, 5)),
           _dense(np.array([[0.9, 0.6], [0.3, 0.8]]), [1.8, 0.4])]
    mks += [S.bernoulli_market(40, 15, 0.3, seed=70 + k) for k in range(3)]
    mks = [_market_of(mk, prec) for mk in mks]
    bt = S.concat_markets(mks)
    if prec == "mixed":
        bt.val = bt.val.astype(np.float32)
    out = solver.solve_batched(bt, tol=tol, precision=prec)
    assert out.status == 0, [i["status"] for i in out.info]
    p = host(out.p)
    for b, mk in enumerate(mks):
        ref = F.pdhcg_solve(mk.row_ptr, mk.col, mk.val, mk.w, mk.m, F.Params(tol=1e-12, max_iter=400000))
        g0, g1 = bt.good_off[b], bt.good_off[b + 1]
        assert np.max(np.abs(p[g0:g1] - ref.p) / ref.p) <= 1e-5, b
