"""Parity at the benchmark's full size (C3: n=1e7 buyers, m=1e5 goods,
nnz ~ 1e9, MIXED), in the launch configuration bench.py times.

The oracle cannot iterate a 1e9-entry market, so one row-subproblem pass
(Section 2.2) at full size is compared on sampled rows (random ones and the
longest ones) with the oracle's exact row solve of the same inputs, and the
column sums the kernel returns must equal the exact sums of its own x.
"""
import os

import numpy as np
import pytest

from oracle import fisher as F
from paper_2506_06258_gb300 import synth as S
from tests.gpu_util import host, torch_cuda

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

FULL = os.environ.get("PDHCG_FULLSIZE", "1") == "1"


@pytest.fixture(scope="module")
def c3():
    torch = torch_cuda()
    scale = 1.0 if FULL else 0.01
    mk = S.config3(n=int(1e7 * scale), m=100_000 if FULL else 20_000, nnz_target=int(1e9 * scale), fp32=True)
    d = {k: torch.from_numpy(getattr(mk, k)).cuda() for k in ("row_ptr", "col", "val", "w")}
    return mk, d


def test_row_prox_full_size_sampled_rows(c3):
    from paper_2506_06258_gb300 import api
    mk, d = c3
    torch = torch_cuda()
    rng = np.random.default_rng(0)
    # a mid-solve-like state: x with the column-clearing scale, prices around sum(w)/m
    deg = np.bincount(mk.col, minlength=mk.m)
    x = (1.0 / deg[mk.col]).astype(np.float32) * rng.uniform(0.5, 1.5, mk.nnz).astype(np.float32)
    p = mk.w.sum() / mk.m * rng.uniform(0.5, 2.0, mk.m)
    tau = 0.9 / np.sqrt(deg.max()) / 30.0
    s = api.Solver()
    xg, sg, cg = s.row_prox(d["row_ptr"], d["col"], d["val"], d["w"], mk.m, torch.from_numpy(x).cuda(),
                            torch.from_numpy(p).cuda(), tau, precision="mixed")
    xg = host(xg)
    sg = host(sg)
    cg = host(cg)
    s.close()
    # sampled rows (including the longest ones) against the oracle's exact solve
    degs = np.diff(mk.row_ptr)
    rows = np.concatenate([rng.choice(mk.n, 400, replace=False), np.argsort(degs)[-20:]])
    for i in rows:
        b, e = mk.row_ptr[i], mk.row_ptr[i + 1]
        u = mk.val[b:e].astype(np.float64)
        u = u / u.max()
        a = x[b:e].astype(np.float64) - tau * p[mk.col[b:e]]
        cc = tau * mk.w[i] * u
        s_ref, x_ref = F.row_prox_exact_single(u, a, cc)
        assert abs(sg[i] - s_ref) <= 1e-6 * s_ref, i
        assert np.max(np.abs(xg[b:e] - x_ref)) <= 2e-6 * max(np.max(x_ref), 1e-30), i
    # the returned column sums are the exact 64-bit fixed-point sums (unit
    # 2^-40, each x rounded to the nearest unit, ties to even) of the returned
    # x: integer work, so compared bit for bit.  Every rounded x and every
    # partial sum is an integer below 2^53, so float64 sums them exactly.
    q = np.rint(xg.astype(np.float64) * 2.0 ** 40)
    csum_q = np.bincount(mk.col, weights=q, minlength=mk.m)
    assert np.array_equal(cg * 2.0 ** 40, csum_q)
