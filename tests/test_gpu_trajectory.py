"""Trajectory parity of the FP64 GPU solver with the oracle before convergence.

Both run Alg. 2 with the Section 5 enhancements (adaptive step rule with
rejected steps, restarts checked every 64 accepted iterations, primal weight
updates) from the same initial point.  Stopped after K accepted iterations,
both return the candidate (current point or average, the one with the lower
relative KKT error) of the last check, so the two must agree iterate by
iterate: the same accepted iterations and passes (rejected steps included),
and the same point to rounding (atomic column sums on the GPU sum in another
order).  Restart counts may differ by one: the oracle takes the restart
decision of the last check before it stops, the GPU returns first.
"""
import numpy as np
import pytest

from oracle import fisher as F
from paper_2506_06258_gb300 import synth as S
from tests.gpu_util import dev, host, ragged_market, torch_cuda

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def solver():
    torch_cuda()
    from paper_2506_06258_gb300 import api
    s = api.Solver()
    yield s
    s.close()


@pytest.mark.parametrize("which", ["c1", "ragged"])
@pytest.mark.parametrize("K", [64, 128, 256, 512, 1024])
def test_fp64_trajectory_matches_oracle(solver, which, K):
    mk = S.config1() if which == "c1" else ragged_market(300, 120, 5, dmax=100)
    ref = F.pdhcg_solve(mk.row_ptr, mk.col, mk.val, mk.w, mk.m, F.Params(tol=1e-15, max_iter=K))
    out = solver.fisher_solve(dev(mk.row_ptr), dev(mk.col), dev(np.asarray(mk.val, np.float64)), dev(mk.w), mk.m,
                              tol=1e-15, precision="fp64", max_iter=K, check=False)
    assert out.info["iters"] == ref.iters == K
    assert out.info["passes"] == ref.passes
    assert ref.restarts - out.info["restarts"] in (0, 1)
    assert out.info["kkt"] == pytest.approx(ref.kkt.kkt, rel=1e-9)
    p, t = host(out.p), host(out.util)
    assert np.max(np.abs(p - ref.p) / ref.p) <= 1e-10
    assert np.max(np.abs(t - ref.t) / ref.t) <= 1e-10
