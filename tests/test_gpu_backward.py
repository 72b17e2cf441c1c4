"""GPU derivative of the equilibrium (pdhcg_fisher_backward) against the FP64
oracle adjoint and against central differences of GPU solves."""
import numpy as np
import pytest

from oracle import adjoint as A, arrow, fisher as F
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


def _dev_mk(mk):
    return dev(mk.row_ptr), dev(mk.col), dev(mk.val), dev(mk.w)


@pytest.mark.parametrize("prec,tol,rtol", [("fp64", 1e-10, 1e-5), ("mixed", 1e-6, 2e-5), ("mixed", 1e-7, 1e-6)])
def test_fisher_backward_matches_oracle(solver, prec, tol, rtol):
    mk = S.bernoulli_market(40, 15, 0.35, seed=801)
    rng = np.random.default_rng(5)
    r, g = rng.normal(size=mk.m), rng.normal(size=mk.n)
    out = solver.fisher_solve(*_dev_mk(mk), mk.m, tol=tol, precision=prec)
    assert out.status == 0
    gu, gw = solver.backward(dev(r), dev(g), nnz=mk.nnz, n=mk.n)
    ref = F.pdhcg_solve(mk.row_ptr, mk.col, mk.val, mk.w, mk.m, F.Params(tol=1e-13, max_iter=500000))
    gu_o, gw_o, info = A.fisher_backward(mk.row_ptr, mk.col, mk.val, mk.w, ref.x, ref.p, ref.t, r, g)
    gu, gw = host(gu), host(gw)
    assert np.array_equal(gu != 0, gu_o != 0)            # same tight graph
    scale = np.max(np.abs(gu_o))
    assert np.max(np.abs(gu - gu_o)) <= rtol * scale
    assert np.max(np.abs(gw - gw_o)) <= rtol * np.max(np.abs(gw_o))


def test_fisher_backward_central_differences(solver):
    """10 entries on the tight graph and 10 off it (off-graph derivatives are 0)."""
    mk = S.bernoulli_market(60, 20, 0.3, seed=802)
    rng = np.random.default_rng(6)
    r = rng.normal(size=mk.m)
    out = solver.fisher_solve(*_dev_mk(mk), mk.m, tol=1e-11, precision="fp64")
    gu, _ = solver.backward(dev(r), None, nnz=mk.nnz, n=mk.n)
    gu = host(gu)
    on, off = np.nonzero(gu)[0], np.nonzero(gu == 0)[0]
    picks = list(rng.choice(on, 10, replace=False)) + list(rng.choice(off, 10, replace=False))

    def f(val):
        o = solver.fisher_solve(dev(mk.row_ptr), dev(mk.col), dev(val), dev(mk.w), mk.m, tol=1e-12,
                                precision="fp64")
        return r @ host(o.p)

    for e in picks:
        h = 1e-5 * mk.val[e]
        vp, vm = mk.val.copy(), mk.val.copy()
        vp[e] += h
        vm[e] -= h
        fd = (f(vp) - f(vm)) / (2 * h)
        assert abs(fd - gu[e]) <= 1e-4 * max(1.0, abs(fd)), (e, fd, gu[e])


def test_arrow_debreu_backward_matches_oracle(solver):
    mk = S.config4(n=40, d_other=5, seed=700)
    rng = np.random.default_rng(2)
    r = rng.normal(size=mk.m)
    out = solver.ad_solve(*_dev_mk(mk), mk.m, outer_tol=1e-10, tol=1e-11, precision="fp64", max_outer=400)
    assert out.status == 0
    gu, _ = solver.backward(dev(r), None, nnz=mk.nnz, n=mk.n)
    ad = arrow.ad_fixed_point(mk.row_ptr, mk.col, mk.val, mk.w, mk.m, outer_tol=1e-12, inner_tol=1e-13,
                              max_outer=400)
    gu_o, mu, info = A.ad_backward(mk.row_ptr, mk.col, mk.val, ad["x"], ad["p"], ad["t"], r)
    gu = host(gu)
    scale = np.max(np.abs(gu_o))
    # same tight graph: edge flows that vanish exactly in the oracle's tree
    # solve come out of conjugate gradients at rounding level
    assert np.array_equal(np.abs(gu) > 1e-9 * scale, np.abs(gu_o) > 1e-9 * scale)
    assert np.max(np.abs(gu - gu_o)) <= 1e-4 * scale


def test_batched_backward_matches_per_market_oracle(solver):
    bt = S.config5(B=5, seed=90, n_range=(20, 60), m_range=(5, 20), q_range=(0.1, 0.3), fp32=False)
    M, N = int(bt.good_off[-1]), int(bt.row_off[-1])
    rng = np.random.default_rng(9)
    r = rng.normal(size=M)
    out = solver.solve_batched(bt, tol=1e-10, precision="fp64")
    assert out.status == 0
    gu, gw = solver.backward(dev(r), None, nnz=int(bt.nnz_off[-1]), n=N)
    gu, gw = host(gu), host(gw)
    for b in range(bt.B):
        mk = bt.market(b)
        ref = F.pdhcg_solve(mk.row_ptr, mk.col, mk.val, mk.w, mk.m, F.Params(tol=1e-13, max_iter=500000))
        g0, g1 = bt.good_off[b], bt.good_off[b + 1]
        z0, z1 = bt.nnz_off[b], bt.nnz_off[b + 1]
        gu_o, gw_o, _ = A.fisher_backward(mk.row_ptr, mk.col, mk.val, mk.w, ref.x, ref.p, ref.t, r[g0:g1])
        assert np.max(np.abs(gu[z0:z1] - gu_o)) <= 1e-5 * max(1.0, np.max(np.abs(gu_o))), b


def test_autograd_function(solver):
    torch = torch_cuda()
    from paper_2506_06258_gb300.api import FisherEquilibrium
    mk = S.bernoulli_market(30, 12, 0.4, seed=803)
    val = torch.tensor(mk.val, device="cuda", requires_grad=True)
    w = torch.tensor(mk.w, device="cuda", requires_grad=True)
    p, t = FisherEquilibrium.apply(val, w, dev(mk.row_ptr), dev(mk.col), mk.m, 1e-11, "fp64")
    rng = np.random.default_rng(3)
    r = torch.tensor(rng.normal(size=mk.m), device="cuda")
    (r * p).sum().backward()
    ref = F.pdhcg_solve(mk.row_ptr, mk.col, mk.val, mk.w, mk.m, F.Params(tol=1e-13, max_iter=500000))
    gu_o, gw_o, _ = A.fisher_backward(mk.row_ptr, mk.col, mk.val, mk.w, ref.x, ref.p, ref.t, r.cpu().numpy())
    assert np.max(np.abs(val.grad.cpu().numpy() - gu_o)) <= 1e-5 * np.max(np.abs(gu_o))
    assert np.max(np.abs(w.grad.cpu().numpy() - gw_o)) <= 1e-5 * np.max(np.abs(gw_o))


def test_autograd_function_utilities_only_loss(solver):
    """A loss that depends on the utilities t alone: the price gradient passed
    to pdhcg_fisher_backward is zero (r = 0, g != 0), checked against the
    oracle adjoint with the same seeds."""
    torch = torch_cuda()
    from paper_2506_06258_gb300.api import FisherEquilibrium
    mk = S.bernoulli_market(30, 12, 0.4, seed=804)
    val = torch.tensor(mk.val, device="cuda", requires_grad=True)
    w = torch.tensor(mk.w, device="cuda", requires_grad=True)
    _, t = FisherEquilibrium.apply(val, w, dev(mk.row_ptr), dev(mk.col), mk.m, 1e-11, "fp64")
    g = torch.tensor(np.random.default_rng(4).normal(size=mk.n), device="cuda")
    (g * t).sum().backward()
    ref = F.pdhcg_solve(mk.row_ptr, mk.col, mk.val, mk.w, mk.m, F.Params(tol=1e-13, max_iter=500000))
    gu_o, gw_o, _ = A.fisher_backward(mk.row_ptr, mk.col, mk.val, mk.w, ref.x, ref.p, ref.t, np.zeros(mk.m),
                                      g.cpu().numpy())
    assert np.max(np.abs(gu_o)) > 0
    assert np.max(np.abs(val.grad.cpu().numpy() - gu_o)) <= 1e-5 * np.max(np.abs(gu_o))
    assert np.max(np.abs(w.grad.cpu().numpy() - gw_o)) <= 1e-5 * np.max(np.abs(gw_o))


def test_backward_without_price_gradient_direct(solver):
    """FisherEquilibrium.backward with grad_p None (autograd may pass None when
    materialisation is off): it must build a zero price gradient of length m."""
    torch = torch_cuda()
    from paper_2506_06258_gb300.api import FisherEquilibrium, Solver
    mk = S.bernoulli_market(20, 9, 0.4, seed=805)

    class Ctx:
        pass
    ctx = Ctx()
    val = dev(mk.val)
    p, t = FisherEquilibrium.forward(ctx, val, dev(mk.w), dev(mk.row_ptr), dev(mk.col), mk.m, 1e-11, "fp64")
    g = torch.ones(mk.n, dtype=torch.float64, device="cuda")
    gu, gw, *_ = FisherEquilibrium.backward(ctx, None, g)
    ref = F.pdhcg_solve(mk.row_ptr, mk.col, mk.val, mk.w, mk.m, F.Params(tol=1e-13, max_iter=500000))
    gu_o, gw_o, _ = A.fisher_backward(mk.row_ptr, mk.col, mk.val, mk.w, ref.x, ref.p, ref.t, np.zeros(mk.m),
                                      np.ones(mk.n))
    assert np.max(np.abs(host(gu) - gu_o)) <= 1e-5 * max(np.max(np.abs(gu_o)), 1e-12)
    assert np.max(np.abs(host(gw) - gw_o)) <= 1e-5 * np.max(np.abs(gw_o))
