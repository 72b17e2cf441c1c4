"""GPU parity of the Fisher hot path against the FP64 oracle, through the C ABI.

Building blocks at sizes spanning several tiles and a ragged tail:
  row subproblem (Section 2.2) and column sums, KKT residuals (Section 5);
full solves (Alg. 2) against the oracle's converged equilibrium on C1 and
small markets, and against closed forms at larger sizes.
Tolerances: FP64 path 1e-10 relative on building blocks; MIXED path: x to
2e-6 relative to the row's largest entry (FP32 storage + float-float row
solve), s to 1e-6 relative; equilibrium prices 1e-5 relative at KKT <= 1e-6.
"""
import numpy as np
import pytest

from oracle import fisher as F
from paper_2506_06258_gb300 import synth as S
from tests.gpu_util import dev, host, ragged_market, torch_cuda
from tests.golden_data import load_equilibrium

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def solver():
    torch_cuda()
    from paper_2506_06258_gb300 import api
    s = api.Solver()
    yield s
    s.close()


def _oracle_prox(mk, x, p, tau):
    sc = F.preprocess(mk.row_ptr, mk.col, mk.val, mk.w, mk.m)
    xn, s = F.primal_step(sc, np.asarray(x, dtype=np.float64), p, tau)
    return sc, xn, s


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("seed", [0, 1])
def test_row_prox_parity(solver, prec, seed):
    mk = ragged_market(3000, 700, seed)
    rng = np.random.default_rng(seed)
    x = rng.uniform(0, 2.0 / 100, mk.nnz) * (rng.uniform(size=mk.nnz) < 0.8)
    if prec == "mixed":
        x = x.astype(np.float32).astype(np.float64)
    p = rng.uniform(0.2, 3.0, mk.m)
    tau = 0.01
    xg, sg, cg = solver.row_prox(dev(mk.row_ptr), dev(mk.col), dev(mk.val), dev(mk.w), mk.m,
                                 dev(x.astype(np.float32 if prec == "mixed" else np.float64)), dev(p), tau,
                                 precision=prec)
    sc, xo, so = _oracle_prox(mk, x, p, tau)
    xg, sg, cg = host(xg).astype(np.float64), host(sg), host(cg)
    rows = F.row_ids(mk.row_ptr)
    rowmaxx = np.zeros(mk.n)
    np.maximum.at(rowmaxx, rows, xo)
    if prec == "fp64":
        assert np.allclose(sg, so, rtol=1e-11)
        assert np.all(np.abs(xg - xo) <= 1e-11 * (rowmaxx[rows] + 1e-300))
        assert np.allclose(cg, F.column_sums(sc.col, xo, mk.m), rtol=1e-11, atol=1e-14)
    else:
        assert np.allclose(sg, so, rtol=1e-6)
        assert np.all(np.abs(xg - xo) <= 2e-6 * rowmaxx[rows] + 1e-30)
        # exact fixed-point column sums of the FP32 iterate (unit 2^-40, round
        # to nearest even per entry; integer work, compared bit for bit)
        q = np.rint(xg * 2.0 ** 40)
        assert np.array_equal(cg * 2.0 ** 40, np.bincount(mk.col, weights=q, minlength=mk.m))


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_kkt_parity(solver, prec):
    mk = ragged_market(2500, 500, 7)
    rng = np.random.default_rng(3)
    x = rng.uniform(0, 0.01, mk.nnz) * (rng.uniform(size=mk.nnz) < 0.6)
    x[mk.row_ptr[:-1]] = rng.uniform(1e-3, 0.01, mk.n)     # every buyer holds something: t_i > 0
    if prec == "mixed":
        x = x.astype(np.float32).astype(np.float64)
    p = rng.uniform(0.5, 2.0, mk.m)
    got = solver.kkt(dev(mk.row_ptr), dev(mk.col), dev(mk.val), dev(mk.w), mk.m,
                     dev(x.astype(np.float32 if prec == "mixed" else np.float64)), dev(p), precision=prec)
    sc = F.preprocess(mk.row_ptr, mk.col, mk.val, mk.w, mk.m)
    k = F.kkt_error(sc, x, p)
    ref = np.array([k.r_primal, k.r_dual, k.r_gap, k.kkt])
    rtol = 1e-12 if prec == "fp64" else 1e-6
    assert np.allclose(got, ref, rtol=rtol), (got, ref)


def _solve_dev(solver, mk, **kw):
    return solver.fisher_solve(dev(mk.row_ptr), dev(mk.col), dev(mk.val), dev(mk.w), mk.m, **kw)


def test_config1_fp64_matches_oracle(solver):
    mk = S.config1()
    out = _solve_dev(solver, mk, tol=1e-8, precision="fp64", return_x=True)
    assert out.status == 0 and out.info["kkt"] <= 1e-8
    ref = F.pdhcg_solve(mk.row_ptr, mk.col, mk.val, mk.w, mk.m, F.Params(tol=1e-11))
    p, t = host(out.p), host(out.util)
    assert np.max(np.abs(p - ref.p) / ref.p) <= 1e-5
    assert np.max(np.abs(t - ref.t) / ref.t) <= 1e-5
    g = load_equilibrium()          # the certified stored equilibrium of C1
    assert np.max(np.abs(p - g["p"]) / g["p"]) <= 1e-5
    assert np.max(np.abs(t - g["t"]) / g["t"]) <= 1e-5
    from oracle import certify
    cert = certify.certificate(mk.row_ptr, mk.col, mk.val, mk.w, mk.m, host(out.x), p)
    assert cert["kkt"] <= 1.5e-8


def test_config1_mixed_matches_oracle(solver):
    mk = S.config1()
    out = _solve_dev(solver, mk, tol=1e-6, precision="mixed")
    assert out.status == 0 and out.info["kkt"] <= 1e-6
    ref = F.pdhcg_solve(mk.row_ptr, mk.col, mk.val, mk.w, mk.m, F.Params(tol=1e-11))
    p = host(out.p)
    assert np.max(np.abs(p - ref.p) / ref.p) <= 1e-5
    g = load_equilibrium()
    assert np.max(np.abs(p - g["p"]) / g["p"]) <= 1e-5


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_rank_one_closed_form(solver, prec):
    from oracle import closed
    mk = S.rank_one_market(1500, 300, seed=5)
    out = _solve_dev(solver, mk, tol=1e-7, precision=prec)
    p_ref, t_ref = closed.rank_one(mk.meta["a"], mk.meta["b"], mk.w)
    assert out.status == 0
    assert np.max(np.abs(host(out.p) - p_ref) / p_ref) <= 1e-5
    assert np.max(np.abs(host(out.util) - t_ref) / t_ref) <= 1e-5


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_small_markets_both_precisions(solver, seed):
    mk = S.bernoulli_market(120, 50, 0.15, seed=100 + seed)
    ref = F.pdhcg_solve(mk.row_ptr, mk.col, mk.val, mk.w, mk.m, F.Params(tol=1e-11))
    for prec, tol in (("fp64", 1e-8), ("mixed", 1e-6)):
        out = _solve_dev(solver, mk, tol=tol, precision=prec)
        assert out.status == 0, (prec, out.info)
        assert np.max(np.abs(host(out.p) - ref.p) / ref.p) <= 1e-5, prec


def test_host_pointers_match_device(solver):
    """Host and device inputs give the same answer.  The MIXED path is
    deterministic (exact fixed-point column sums, ordered reductions), so its
    results are bit-identical; the FP64 path sums columns with FP64 atomics,
    whose order varies, so it agrees to rounding."""
    mk = S.bernoulli_market(80, 40, 0.3, seed=9)
    a = solver.fisher_solve(mk.row_ptr, mk.col, mk.val, mk.w, mk.m, tol=1e-6, precision="mixed")
    b = _solve_dev(solver, mk, tol=1e-6, precision="mixed")
    assert isinstance(a.p, np.ndarray)
    assert np.array_equal(a.p, host(b.p))
    a = solver.fisher_solve(mk.row_ptr, mk.col, mk.val, mk.w, mk.m, tol=1e-8, precision="fp64")
    b = _solve_dev(solver, mk, tol=1e-8, precision="fp64")
    assert np.allclose(a.p, host(b.p), rtol=1e-6)


def test_invalid_inputs_rejected(solver):
    from paper_2506_06258_gb300 import capi
    mk = S.bernoulli_market(30, 10, 0.5, seed=4)
    bad_val = mk.val.copy(); bad_val[3] = -1.0
    bad_w = mk.w.copy(); bad_w[2] = np.nan
    bad_col = mk.col.copy(); b0, b1 = mk.row_ptr[0], mk.row_ptr[1]
    bad_col[b0:b1] = bad_col[b0:b1][::-1] if b1 - b0 > 1 else bad_col[b0:b1]
    empty_col_m = mk.m + 1        # one good no buyer likes
    cases = [
        (mk.row_ptr, mk.col, bad_val, mk.w, mk.m),
        (mk.row_ptr, mk.col, mk.val, bad_w, mk.m),
        (mk.row_ptr, mk.col, mk.val, mk.w, empty_col_m),
    ]
    if mk.row_ptr[1] - mk.row_ptr[0] > 1:
        cases.append((mk.row_ptr, bad_col, mk.val, mk.w, mk.m))
    for args in cases:
        out = solver.fisher_solve(*[dev(a) if isinstance(a, np.ndarray) else a for a in args],
                                  tol=1e-6, check=False)
        assert out.status == capi.PDHCG_ERR_INVALID


def test_iteration_cap_reports_not_converged(solver):
    from paper_2506_06258_gb300 import capi
    mk = S.config1()
    out = _solve_dev(solver, mk, tol=1e-12, precision="fp64", max_iter=64, check=False)
    assert out.status == capi.PDHCG_ERR_NOT_CONVERGED
    assert out.info["iters"] >= 64
    assert np.all(np.isfinite(host(out.p)))
