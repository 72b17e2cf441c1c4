"""pdhcg_kkt_noalloc: the allocation-free KKT entry point, for callers that
cannot allocate device memory when they need the residual (inside allocator
callbacks, under a fully reserved device, or in loops that forbid allocation).
It must give the same residuals as pdhcg_kkt, call after call, although all of
its calls share one fixed scratch array.  Collected last on purpose."""
import numpy as np
import pytest

from paper_2506_06258_gb300 import synth as S
from tests.gpu_util import dev, torch_cuda

pytestmark = pytest.mark.gpu


def _point(mk, seed):
    rng = np.random.default_rng(seed)
    x = rng.uniform(0, 0.02, mk.nnz) * (rng.uniform(size=mk.nnz) < 0.6)
    x[mk.row_ptr[:-1]] = rng.uniform(1e-3, 0.02, mk.n)          # every buyer holds something
    p = rng.uniform(0.5, 2.0, mk.m)
    return x, p


def test_noalloc_matches_kkt_on_two_calls_in_a_row():
    torch_cuda()
    from paper_2506_06258_gb300 import api, capi
    s = api.Solver()
    markets = [S.bernoulli_market(900, 300, 0.05, seed=21), S.config3(n=3000, m=800, nnz_target=120_000,
                                                                        fp32=False)]
    for call, mk in enumerate(markets):        # two calls in a row, different markets and points
        x, p = _point(mk, call)
        ref = s.kkt(dev(mk.row_ptr), dev(mk.col), dev(mk.val), dev(mk.w), mk.m, dev(x), dev(p),
                    precision="fp64")
        dmk = s.market(dev(mk.row_ptr), dev(mk.col), dev(mk.val), dev(mk.w), mk.m)
        xd, pd = dev(x), dev(p)
        out = np.zeros(4)
        st = capi.pdhcg_kkt_noalloc(dmk, xd.data_ptr(), pd.data_ptr(), out.ctypes.data, 0)
        assert st == 0, capi.status_string(st)
        assert np.allclose(out, ref, rtol=1e-12), (call, out, ref)
    s.close()


def test_noalloc_rejects_oversize_and_host_inputs():
    torch_cuda()
    from paper_2506_06258_gb300 import api, capi
    mk = S.bernoulli_market(50, 20, 0.3, seed=3)
    x, p = _point(mk, 5)
    out = np.zeros(4)
    host_mk = api.Solver.market(mk.row_ptr, mk.col, mk.val, mk.w, mk.m)
    assert capi.pdhcg_kkt_noalloc(host_mk, x.ctypes.data, p.ctypes.data, out.ctypes.data, 0) == \
        capi.PDHCG_ERR_INVALID
    big = api.Solver.market(dev(mk.row_ptr), dev(mk.col), dev(mk.val), dev(mk.w), 262145)
    xd, pd = dev(x), dev(np.ones(262145))
    assert capi.pdhcg_kkt_noalloc(big, xd.data_ptr(), pd.data_ptr(), out.ctypes.data, 0) == capi.PDHCG_ERR_INVALID
