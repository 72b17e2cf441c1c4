"""pdhcg_kkt_noalloc: the allocation-free KKT entry point, for callers that
cannot allocate device memory when they need the residual: code inside an
allocator or memory-pool callback (an allocation there would re-enter the
allocator), a process whose device memory another framework holds in full, or
a loop that forbids allocation after start-up.  Each call must give the same
residuals as pdhcg_kkt and as the oracle's Section 5 criteria, call after
call, although all calls share one fixed scratch array, and a call must leave
the device's free memory unchanged.  Collected last on purpose, so that a run
stopping at its first failure has already run every other test."""
import numpy as np
import pytest

from oracle import fisher as F
from paper_2506_06258_gb300 import synth as S
from tests.gpu_util import dev, host, torch_cuda

pytestmark = pytest.mark.gpu


def _point(mk, seed):
    rng = np.random.default_rng(seed)
    x = rng.uniform(0, 0.02, mk.nnz) * (rng.uniform(size=mk.nnz) < 0.6)
    x[mk.row_ptr[:-1]] = rng.uniform(1e-3, 0.02, mk.n)          # every buyer holds something
    p = rng.uniform(0.5, 2.0, mk.m)
    return x, p


def _oracle(mk, x, p, val=None):
    sc = F.preprocess(mk.row_ptr, mk.col, mk.val if val is None else val, mk.w, mk.m)
    k = F.kkt_error(sc, x, p)
    return np.array([k.r_primal, k.r_dual, k.r_gap, k.kkt])


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
        assert np.allclose(out, _oracle(mk, x, p), rtol=1e-12, atol=0), (call, out)
    s.close()


def test_noalloc_fp32_values_and_device_output():
    torch = torch_cuda()
    from paper_2506_06258_gb300 import api, capi
    mk = S.bernoulli_market(700, 250, 0.06, seed=22)
    v32 = mk.val.astype(np.float32)
    x, p = _point(mk, 7)
    dmk = api.Solver.market(dev(mk.row_ptr), dev(mk.col), dev(v32), dev(mk.w), mk.m)
    xd, pd = dev(x), dev(p)
    out_d = torch.full((4,), -1.0, dtype=torch.float64, device="cuda")
    st = capi.pdhcg_kkt_noalloc(dmk, xd.data_ptr(), pd.data_ptr(), out_d.data_ptr(), 0)
    assert st == 0, capi.status_string(st)
    ref = _oracle(mk, x, p, val=v32.astype(np.float64))
    assert np.allclose(host(out_d), ref, rtol=1e-12, atol=0)


def test_noalloc_leaves_free_device_memory_unchanged():
    torch = torch_cuda()
    from paper_2506_06258_gb300 import api, capi
    mk = S.bernoulli_market(2000, 600, 0.03, seed=23)
    x, p = _point(mk, 8)
    args = [dev(a) for a in (mk.row_ptr, mk.col, mk.val, mk.w, x, p)]
    dmk = api.Solver.market(args[0], args[1], args[2], args[3], mk.m)
    out = np.zeros(4)
    assert capi.pdhcg_kkt_noalloc(dmk, args[4].data_ptr(), args[5].data_ptr(), out.ctypes.data, 0) == 0
    mk2 = S.bernoulli_market(1500, 500, 0.04, seed=24)     # a fresh market for the measured call
    x2, p2 = _point(mk2, 9)
    args2 = [dev(a) for a in (mk2.row_ptr, mk2.col, mk2.val, mk2.w, x2, p2)]
    dmk2 = api.Solver.market(args2[0], args2[1], args2[2], args2[3], mk2.m)
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    assert capi.pdhcg_kkt_noalloc(dmk2, args2[4].data_ptr(), args2[5].data_ptr(), out.ctypes.data, 0) == 0
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0
    assert np.allclose(out, _oracle(mk2, x2, p2), rtol=1e-12, atol=0)


def test_noalloc_rejects_bad_inputs():
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
    # one column index out of range: the kernel checks it, skips the entry and
    # reports the market as invalid
    col = mk.col.copy()
    col[len(col) // 2] = mk.m + 5
    bad = api.Solver.market(dev(mk.row_ptr), dev(col), dev(mk.val), dev(mk.w), mk.m)
    pd = dev(p)
    assert capi.pdhcg_kkt_noalloc(bad, xd.data_ptr(), pd.data_ptr(), out.ctypes.data, 0) == capi.PDHCG_ERR_INVALID
    # the next call on a good market still succeeds (the error flag is cleared)
    good = api.Solver.market(dev(mk.row_ptr), dev(mk.col), dev(mk.val), dev(mk.w), mk.m)
    assert capi.pdhcg_kkt_noalloc(good, xd.data_ptr(), pd.data_ptr(), out.ctypes.data, 0) == 0
    assert np.allclose(out, _oracle(mk, x, p), rtol=1e-12, atol=0)
