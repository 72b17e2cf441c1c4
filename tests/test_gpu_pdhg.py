"""Restarted PDHG (Alg. 1) on the GPU, FP64: the paper's comparator for
PDHCG, and a second route to the same equilibrium.  Prices and utilities are
unique (Fact 1), so PDHG must reach the prices of the oracle (the stored C1
equilibrium of the oracle's PDHCG, and the oracle's own PDHG on a small
market) and the closed form of rank-one markets; its allocation must pass the
equilibrium certificate."""
import numpy as np
import pytest

from oracle import certify, closed, pdhg as OP
from paper_2506_06258_gb300 import synth as S
from tests.golden_data import load_equilibrium
from tests.gpu_util import dev, host, torch_cuda

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def solver():
    torch_cuda()
    from paper_2506_06258_gb300 import api
    s = api.Solver()
    yield s
    s.close()


def _solve(solver, mk, tol, **kw):
    return solver.fisher_solve_pdhg(dev(mk.row_ptr), dev(mk.col), dev(mk.val.astype(np.float64)), dev(mk.w), mk.m,
                                    tol=tol, return_x=True, max_iter=2_000_000, **kw)


def test_pdhg_c1_matches_stored_equilibrium(solver):
    mk = S.config1()
    g = load_equilibrium()
    out = _solve(solver, mk, 1e-8)
    assert out.status == 0 and out.info["kkt"] <= 1e-8
    assert np.max(np.abs(host(out.p) - g["p"]) / g["p"]) <= 1e-6
    assert np.max(np.abs(host(out.util) - g["t"]) / g["t"]) <= 1e-6
    c = certify.certificate(mk.row_ptr, mk.col, mk.val, mk.w, mk.m, host(out.x), host(out.p))
    assert c["clearing"] <= 1e-7 and c["bang_per_buck"] <= 1e-6 and c["complement"] <= 1e-7


def test_pdhg_matches_oracle_pdhg(solver):
    mk = S.bernoulli_market(60, 25, 0.3, seed=901)
    ref = OP.pdhg_solve(mk.row_ptr, mk.col, mk.val, mk.w, mk.m, OP.PdhgParams(tol=1e-10))
    assert ref.converged
    out = _solve(solver, mk, 1e-9, restart_every=1000)
    assert out.status == 0
    assert np.max(np.abs(host(out.p) - ref.p) / ref.p) <= 1e-6


@pytest.mark.parametrize("n,m", [(300, 40), (2000, 120)])
def test_pdhg_rank_one_closed_form(solver, n, m):
    rng = np.random.default_rng(n + m)
    a, bv = rng.uniform(0.2, 1.0, n), rng.uniform(0.2, 1.0, m)
    U = np.outer(a, bv)
    row_ptr = np.arange(0, n * m + 1, m, dtype=np.int64)
    col = np.tile(np.arange(m, dtype=np.int32), n)
    w = rng.uniform(0.5, 1.5, n)
    mk = S.Market(n, m, row_ptr, col, U.ravel(), w, "rank one")
    p_ref = closed.rank_one(a, bv, w)[0]
    out = _solve(solver, mk, 1e-8)
    assert out.status == 0
    assert np.max(np.abs(host(out.p) - p_ref) / p_ref) <= 1e-5


def test_pdhg_rejects_bad_restart_period(solver):
    from paper_2506_06258_gb300 import capi
    mk = S.config1()
    out = solver.fisher_solve_pdhg(dev(mk.row_ptr), dev(mk.col), dev(mk.val), dev(mk.w), mk.m, restart_every=0,
                                   check=False)
    assert out.status == capi.PDHCG_ERR_INVALID
