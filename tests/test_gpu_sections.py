"""The K-section row search of Section 2.2 (K = 32 in the paper) as the row
solve of the FP64 single-market solver: with any section count it must reach
the same equilibrium as the exact root (the stored C1 equilibrium of the
oracle) and, row by row, the oracle's K-section search reaches the oracle's
exact row solution it is compared with."""
import numpy as np
import pytest

from oracle import fisher as F
from paper_2506_06258_gb300 import synth as S
from tests.golden_data import load_equilibrium
from tests.gpu_util import dev, host, ragged_market, torch_cuda

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def solver():
    torch_cuda()
    from paper_2506_06258_gb300 import api
    s = api.Solver()
    yield s
    s.close()


@pytest.mark.parametrize("K", [2, 32])
def test_section_search_solver_reaches_the_equilibrium(solver, K):
    mk = S.config1()
    g = load_equilibrium()
    out = solver.fisher_solve(dev(mk.row_ptr), dev(mk.col), dev(mk.val), dev(mk.w), mk.m, tol=1e-8,
                              precision="fp64", section_count=K, section_tol=1e-11, max_iter=400000)
    assert out.status == 0
    assert np.max(np.abs(host(out.p) - g["p"]) / g["p"]) <= 1e-6
    assert np.max(np.abs(host(out.util) - g["t"]) / g["t"]) <= 1e-6


def test_section_search_on_ragged_rows_matches_the_exact_solver(solver):
    """Rows of every width (1 to 600 entries: register-resident and chunked):
    a K-section solve and an exact-root solve stop at the same equilibrium."""
    mk = ragged_market(600, 300, 11)
    args = (dev(mk.row_ptr), dev(mk.col), dev(mk.val), dev(mk.w), mk.m)
    a = solver.fisher_solve(*args, tol=1e-8, precision="fp64", max_iter=400000)
    b = solver.fisher_solve(*args, tol=1e-8, precision="fp64", section_count=8, section_tol=1e-11,
                            max_iter=400000)
    assert a.status == 0 and b.status == 0
    pa, pb = host(a.p), host(b.p)
    assert np.max(np.abs(pa - pb) / pa) <= 2e-6


def test_section_count_validation(solver):
    from paper_2506_06258_gb300 import capi
    mk = S.config1()
    out = solver.fisher_solve(dev(mk.row_ptr), dev(mk.col), dev(mk.val), dev(mk.w), mk.m, precision="fp64",
                              section_count=1, check=False)
    assert out.status == capi.PDHCG_ERR_INVALID
