"""Multi-rank logic on CPU ranks (gloo, world size 2).

The single-market split exchanges only column sums and step scalars (Alg. 2:
buyers meet only in the price update); these tests run that split with the
FP64 oracle's steps on two gloo ranks and check that every rank reproduces the
unsplit iteration, and check the work splits and the max-over-ranks timing
reduction that the benchmark uses.
"""
import os
import socket
import sys

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

from paper_2506_06258_gb300 import shard, synth as S


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _run(fn, world, *args):
    port = _free_port()
    ctx = mp.get_context("spawn")
    procs = [ctx.Process(target=_entry, args=(fn, r, world, port, args)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
    codes = [p.exitcode for p in procs]
    for p in procs:
        if p.is_alive():
            p.kill()
    assert codes == [0] * world, codes


def _entry(fn, rank, world, port, args):
    if ROOT not in sys.path:
        sys.path.insert(0, ROOT)
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        fn(rank, world, *args)
    finally:
        dist.destroy_process_group()


# ---------------------------------------------------------------------------
# work splits (no process group)
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("parts", [1, 2, 3, 7, 64])
def test_partition_rows_balanced(parts):
    mk = S.skewed_market(20000, 500, 400000, seed=5)
    b = shard.partition_rows(mk.row_ptr, parts)
    assert b[0] == 0 and b[-1] == mk.n and len(b) == parts + 1
    assert (np.diff(b) >= 0).all()
    loads = mk.row_ptr[b[1:]] - mk.row_ptr[b[:-1]]
    assert loads.sum() == mk.nnz
    maxdeg = np.diff(mk.row_ptr).max()
    assert loads.max() <= mk.nnz / parts + maxdeg


def test_partition_rows_more_parts_than_rows():
    row_ptr = np.array([0, 3, 4, 9], dtype=np.int64)
    b = shard.partition_rows(row_ptr, 5)
    assert b[0] == 0 and b[-1] == 3 and (np.diff(b) >= 0).all()


@pytest.mark.parametrize("parts", [1, 2, 5, 8])
def test_partition_markets_cover_and_bound(parts):
    rng = np.random.default_rng(parts)
    sizes = rng.integers(100, 500000, 4096)
    owned = shard.partition_markets(sizes, parts)
    allm = np.sort(np.concatenate(owned))
    assert (allm == np.arange(len(sizes))).all()
    loads = np.array([sizes[o].sum() for o in owned])
    assert loads.max() <= sizes.sum() / parts + sizes.max()


# ---------------------------------------------------------------------------
# split iteration on two gloo ranks
# ---------------------------------------------------------------------------
def _split_iteration(rank, world, iters):
    from oracle import fisher as F
    mk = S.config1()
    b = shard.partition_rows(mk.row_ptr, world)
    lo, hi = int(b[rank]), int(b[rank + 1])
    e0, e1 = int(mk.row_ptr[lo]), int(mk.row_ptr[hi])

    # unsplit reference, run by every rank
    sc = F.preprocess(mk.row_ptr, mk.col, mk.val, mk.w, mk.m)
    x, p = F.initial_point(sc)
    tau = sigma = 0.9 / np.sqrt(sc.deg_col.max())
    c_prev = c = F.column_sums(sc.col, x, sc.m)

    # this rank's rows; column degrees (for x^0) are the first exchange
    rp_l = mk.row_ptr[lo:hi + 1] - mk.row_ptr[lo]
    sl = F.preprocess(rp_l, mk.col[e0:e1], mk.val[e0:e1], mk.w[lo:hi], mk.m)
    deg = shard.all_sum_(torch.from_numpy(np.bincount(sl.col, minlength=mk.m).astype(np.float64))).numpy()
    assert (deg == sc.deg_col).all()
    xl = 1.0 / deg[sl.col]
    pl = np.full(mk.m, shard.all_sum_(torch.tensor([sl.w.sum()], dtype=torch.float64)).item() / mk.m)
    cl_prev = cl = shard.all_sum_(torch.from_numpy(F.column_sums(sl.col, xl, mk.m))).numpy()

    for _ in range(iters):
        p_new = F.price_step(p, c, c_prev, sigma)
        x_new, _s = F.primal_step(sc, x, p_new, tau)
        dx2 = float(((x_new - x) ** 2).sum())
        c_prev, c = c, F.column_sums(sc.col, x_new, sc.m)
        x, p = x_new, p_new

        pl_new = F.price_step(pl, cl, cl_prev, sigma)
        xl_new, _sl = F.primal_step(sl, xl, pl_new, tau)
        dx2_l = shard.all_sum_(torch.tensor([((xl_new - xl) ** 2).sum()], dtype=torch.float64)).item()
        cl_prev, cl = cl, shard.all_sum_(torch.from_numpy(F.column_sums(sl.col, xl_new, mk.m))).numpy()
        xl, pl = xl_new, pl_new

        assert np.allclose(pl, p, rtol=1e-12, atol=1e-14)
        assert np.allclose(xl, x[e0:e1], rtol=1e-11, atol=1e-14)
        assert np.allclose(cl, c, rtol=1e-12, atol=1e-13)
        assert abs(dx2_l - dx2) <= 1e-11 * max(dx2, 1e-300)

    # KKT column maxima: max over ranks of the per-rank maxima
    y_l = sl.w / F.row_dot(sl.row_ptr, sl.u, xl)
    M_l = np.zeros(mk.m)
    np.maximum.at(M_l, sl.col, sl.u * y_l[sl.rows])
    M = shard.all_max_(torch.from_numpy(M_l)).numpy()
    y = sc.w / F.row_dot(sc.row_ptr, sc.u, x)
    M_ref = np.zeros(mk.m)
    np.maximum.at(M_ref, sc.col, sc.u * y[sc.rows])
    assert np.allclose(M, M_ref, rtol=1e-11)


def test_two_rank_row_split_matches_unsplit():
    _run(_split_iteration, 2, 12)


def _max_over(rank, world):
    v = shard.max_over_ranks(1.5 + rank)
    assert v == 0.5 + world
    t = torch.tensor([float(rank)])
    assert shard.all_sum_(t).item() == sum(range(world))


def test_two_rank_max_over_ranks():
    _run(_max_over, 2)


def _market_split(rank, world):
    mb = S.config5(B=32, seed=77, n_range=(20, 60), m_range=(10, 30))
    sizes = np.diff(mb.nnz_off)
    mine = shard.partition_markets(sizes, world)[rank]
    count = shard.all_sum_(torch.tensor([float(len(mine))])).item()
    assert count == 32
    mask = np.zeros(32)
    mask[mine] = 1
    assert (shard.all_sum_(torch.from_numpy(mask)).numpy() == 1).all()


def test_two_rank_market_split_covers_once():
    _run(_market_split, 2)
