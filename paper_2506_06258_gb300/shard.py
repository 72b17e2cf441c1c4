"""Host-side work split for running the solver on several GPUs of one node.

Alg. 2 touches one buyer's entries only inside that buyer's row subproblem
(Section 2.2), and couples buyers only through the column sums
c_j = sum_i x_ij of the price update and a few global scalars (the step-size
and restart norms of Section 5).  Two splits follow:

* one market: contiguous blocks of buyers with about equal nnz; per iteration
  the ranks exchange the m-vector c (sum) and the step scalars (sum), and at a
  KKT check the per-good column maxima (max);
* many independent markets (the batched form): whole markets per rank,
  balanced by nnz, with no exchange at all.

The helpers below compute those splits and wrap the reductions; they are plain
host code (numpy + torch.distributed) and run with any process-group backend.
"""
from __future__ import annotations

import heapq

import numpy as np


def partition_rows(row_ptr, parts: int) -> np.ndarray:
    """Boundaries b[0..parts] of contiguous row blocks of about equal nnz.

    Rank r owns rows [b[r], b[r+1]).  Block r ends at the first row whose CSR
    offset reaches r * nnz / parts, so every block holds at most
    nnz / parts + (largest row degree) entries.  Blocks may be empty when
    parts exceeds the number of rows.
    """
    row_ptr = np.asarray(row_ptr, dtype=np.int64)
    if parts < 1:
        raise ValueError("parts must be >= 1")
    n = len(row_ptr) - 1
    nnz = int(row_ptr[-1])
    targets = (np.arange(1, parts, dtype=np.int64) * nnz) // parts
    cuts = np.searchsorted(row_ptr, targets, side="left")
    b = np.concatenate([[0], np.clip(cuts, 0, n), [n]]).astype(np.int64)
    return np.maximum.accumulate(b)


def partition_markets(nnz_per_market, parts: int) -> list:
    """Markets per rank by longest-processing-time-first on nnz.

    Returns `parts` sorted index arrays.  The heaviest rank carries at most
    total / parts + max(nnz_per_market) (the greedy bound).
    """
    sizes = np.asarray(nnz_per_market, dtype=np.int64)
    if parts < 1:
        raise ValueError("parts must be >= 1")
    heap = [(0, r) for r in range(parts)]
    owned = [[] for _ in range(parts)]
    for b in np.argsort(-sizes, kind="stable"):
        load, r = heapq.heappop(heap)
        owned[r].append(int(b))
        heapq.heappush(heap, (load + int(sizes[b]), r))
    return [np.array(sorted(o), dtype=np.int64) for o in owned]


def _dist():
    import torch.distributed as dist
    return dist if dist.is_available() and dist.is_initialized() else None


def all_sum_(t):
    """In-place sum over ranks of a tensor (identity without a process group):
    the exchange of column sums and step scalars."""
    dist = _dist()
    if dist is not None:
        dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return t


def all_max_(t):
    """In-place maximum over ranks (identity without a process group): the
    KKT column maxima and the wall time of the slowest rank."""
    dist = _dist()
    if dist is not None:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return t


def max_over_ranks(value: float, device=None) -> float:
    """The largest value of a host scalar over all ranks."""
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    return float(all_max_(t).item())
