"""Batched persistent solver: every market of a batch matches the FP64 oracle
and the single-market GPU solve."""
import numpy as np
import pytest

from oracle import fisher as F
from paper_2506_06258_gb300 import synth as S
from tests.gpu_util import dev, host, torch_cuda

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def solver():
    torch_cuda()
    from paper_2506_06258_gb300 import api
    s = api.Solver()
    yield s
    s.close()


def _small_batch(B, seed, fp32):
    # the C5 law at reduced sizes (the oracle must finish in seconds)
    return S.config5(B=B, seed=seed, n_range=(20, 160), m_range=(5, 60), q_range=(0.05, 0.3), fp32=fp32)


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_batch_matches_oracle(solver, prec):
    bt = _small_batch(12, 77, fp32=(prec == "mixed"))
    # MIXED is solved a little below 1e-6: at KKT 1e-6 the price error bound
    # scales with 1 / (smallest price), and these small markets carry goods
    # priced at a few percent of the mean
    tol = 1e-8 if prec == "fp64" else 2e-7
    out = solver.solve_batched(bt, tol=tol, precision=prec)
    assert out.status == 0, [i["status"] for i in out.info]
    p = host(out.p)
    u = host(out.util)
    for b in range(bt.B):
        mk = bt.market(b)
        ref = F.pdhcg_solve(mk.row_ptr, mk.col, mk.val.astype(np.float64), mk.w, mk.m, F.Params(tol=1e-11))
        g0, g1 = bt.good_off[b], bt.good_off[b + 1]
        r0, r1 = bt.row_off[b], bt.row_off[b + 1]
        assert np.max(np.abs(p[g0:g1] - ref.p) / ref.p) <= 1e-5, b
        assert np.max(np.abs(u[r0:r1] - ref.t) / ref.t) <= 1e-5, b
        assert out.info[b]["kkt"] <= tol


def test_batch_equals_single_market_solves(solver):
    bt = _small_batch(6, 91, fp32=True)
    out = solver.solve_batched(bt, tol=1e-6, precision="mixed")
    p = host(out.p)
    for b in range(bt.B):
        mk = bt.market(b)
        one = solver.fisher_solve(dev(mk.row_ptr), dev(mk.col), dev(mk.val), dev(mk.w), mk.m, tol=1e-6,
                                  precision="mixed")
        g0, g1 = bt.good_off[b], bt.good_off[b + 1]
        assert np.max(np.abs(p[g0:g1] - host(one.p)) / host(one.p)) <= 2e-5


def test_batch_rejects_invalid_market(solver):
    from paper_2506_06258_gb300 import capi
    bt = _small_batch(4, 5, fp32=True)
    bt.val = bt.val.copy()
    bt.val[int(bt.nnz_off[2]) + 1] = -1.0
    out = solver.solve_batched(bt, tol=1e-6, precision="mixed", check=False)
    assert out.status == capi.PDHCG_ERR_INVALID


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_batch_long_rows_rank_one_closed_form(solver, prec):
    """Dense rank-one markets with 200-300 goods: every row takes the chunked
    warp-per-row path of the batched kernel; p_j = b_j sum(w) / sum(b) and
    t_i = a_i w_i sum(b) / sum(w) hold at any size."""
    from oracle import closed
    mks = [S.rank_one_market(n, m, seed=950 + k) for k, (n, m) in enumerate(((40, 300), (25, 200), (60, 260)))]
    bt = S.concat_markets(mks)
    if prec == "mixed":
        bt.val = bt.val.astype(np.float32)
    out = solver.solve_batched(bt, tol=1e-8 if prec == "fp64" else 2e-7, precision=prec)
    assert out.status == 0, [i["status"] for i in out.info]
    p, u = host(out.p), host(out.util)
    for b, mk in enumerate(mks):
        p_ref, t_ref = closed.rank_one(mk.meta["a"], mk.meta["b"], mk.w)
        g0, g1 = bt.good_off[b], bt.good_off[b + 1]
        r0, r1 = bt.row_off[b], bt.row_off[b + 1]
        assert np.max(np.abs(p[g0:g1] - p_ref) / p_ref) <= 1e-5, b
        assert np.max(np.abs(u[r0:r1] - t_ref) / t_ref) <= 1e-5, b
