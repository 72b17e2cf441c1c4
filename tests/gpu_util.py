"""Helpers shared by the GPU tests (inputs on cuda:0, results to numpy)."""
import numpy as np
import pytest


def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def dev(a):
    torch = torch_cuda()
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda:0")


def host(t):
    return t.detach().cpu().numpy() if hasattr(t, "detach") else np.asarray(t)


def ragged_market(n, m, seed, dmax=600, law=0):
    """Rows whose degrees span every bucket of the row kernel (1 .. dmax,
    log-uniform), goods drawn uniformly, so several tiles and a ragged tail."""
    from paper_2506_06258_gb300 import synth as S
    rng = np.random.default_rng(seed)
    deg = np.minimum(np.exp(rng.uniform(0, np.log(dmax), n)).astype(np.int64), m)
    deg = np.maximum(deg, 1)
    row_ptr = np.concatenate(([0], np.cumsum(deg))).astype(np.int64)
    cols = [np.sort(rng.choice(m, size=d, replace=False)) for d in deg]
    col = np.concatenate(cols).astype(np.int32)
    val = rng.uniform(0.05, 1.0, len(col)) if law == 0 else np.exp(rng.normal(0, 1, len(col)))
    w = rng.uniform(0.5, 1.5, n)
    mk = S.Market(n, m, row_ptr, col, val, w, f"ragged(n={n},m={m})")
    return S.repair_assumption1(mk, seed, 0, 0.05, 1.0)
