"""JD-shaped Fisher markets (Section 5.2, Table tab:fisher): the two smallest
prefixes of the synthetic click log (n = 2,000 and 5,000 users), whose
click-count utilities span four orders of magnitude and whose prices span
six (goods clicked by one user with a small budget).

Reference: the single-market FP64 GPU solve to relative KKT 1e-8, whose
(x, p) must pass the oracle's equilibrium certificate (market clearing,
budgets, bang-per-buck, complementarity), which pins the unique p and t
(Fact 1).  The MIXED solve to 2e-7 must match it:
  - utilities to 1e-5 relative;
  - prices to 1e-5 relative on goods priced at least 1e-3 of the largest
    price, and to 1e-5 p_j + 1e-7 max p on every good.  The Section 5 KKT
    error scales its residuals by the largest entries, so it bounds a price
    error against max p, not against a price a million times smaller.
"""
import numpy as np
import pytest

from oracle import certify
from paper_2506_06258_gb300 import synth as S
from tests.gpu_util import dev, host, torch_cuda

pytestmark = pytest.mark.gpu

RTOL = 1e-5
ATOL_OF_MAX = 1e-7


@pytest.fixture(scope="module")
def solver():
    torch_cuda()
    from paper_2506_06258_gb300 import api
    s = api.Solver()
    yield s
    s.close()


@pytest.mark.parametrize("n", [2000, 5000])
def test_jd_prefix_mixed_matches_certified_fp64(solver, n):
    mk = S.jd_like_market(n, fp32=True)
    v64 = mk.val.astype(np.float64)
    ref = solver.fisher_solve(dev(mk.row_ptr), dev(mk.col), dev(v64), dev(mk.w), mk.m, tol=1e-8, precision="fp64",
                              return_x=True, max_iter=1_000_000)
    assert ref.status == 0, ref.info
    p64, x64, t64 = host(ref.p), host(ref.x), host(ref.util)
    cert = certify.certificate(mk.row_ptr, mk.col, v64, mk.w, mk.m, x64, p64)
    assert cert["clearing"] <= 1e-7 and cert["budgets"] <= 1e-7 and cert["money"] <= 1e-9, cert
    assert cert["bang_per_buck"] <= 1e-7 and cert["complement"] <= 1e-7, cert
    assert p64.max() / p64.min() > 1e5            # the wide price range this test is about

    out = solver.fisher_solve(dev(mk.row_ptr), dev(mk.col), dev(mk.val), dev(mk.w), mk.m, tol=2e-7,
                              precision="mixed", max_iter=1_000_000)
    assert out.status == 0, out.info
    assert out.info["kkt"] <= 2e-7
    p, t = host(out.p), host(out.util)
    assert np.max(np.abs(t - t64) / t64) <= RTOL
    big = p64 >= 1e-3 * p64.max()
    assert np.max(np.abs(p[big] - p64[big]) / p64[big]) <= RTOL
    assert np.all(np.abs(p - p64) <= RTOL * p64 + ATOL_OF_MAX * p64.max())
