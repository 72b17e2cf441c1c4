"""Seeded synthetic market generator (inputs only).

Holds none of the equilibrium method's arithmetic: it draws utility matrices
``U`` (CSR: ``row_ptr`` int64, ``col`` int32 sorted within each row, ``val``)
and budgets ``w`` with the shapes of the paper's synthetic workloads
(Section 5.1: sparse ``U`` with ``n`` buyers much larger than ``m`` goods) and
of the five benchmark configurations.  Both the CUDA solver's tests and the
FP64 oracle consume these arrays, so the generator is kept in a module of its
own.  Random numbers come from Philox4x32-10 (Salmon et al., SC'11) in
``synth.c``; draws are keyed by (seed, stream, row) so results do not depend on
the thread count.  Assumption 1 (every buyer likes some good and every good is
liked by some buyer) is enforced by :func:`repair_assumption1`.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass, field
from typing import Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "synth.c")
_LIB_PATH = os.path.join(_HERE, "libsynth.so")
_lib = None

SEED_BASE = 2506062580


def build(force: bool = False) -> str:
    """Compile ``synth.c`` into ``libsynth.so`` next to it (gcc, OpenMP)."""
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fPIC", "-shared", "-fopenmp", _SRC, "-o", tmp, "-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _L():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB_PATH)
        P = ctypes.c_void_p
        i64, i32, u64, u32, f64 = ctypes.c_int64, ctypes.c_int32, ctypes.c_uint64, ctypes.c_uint32, ctypes.c_double
        sig = {
            "synth_philox4x32_10": (None, [P, P, P]),
            "synth_budgets": (None, [u64, i64, f64, f64, P]),
            "synth_bernoulli_degrees": (None, [u64, i64, i32, f64, P]),
            "synth_fill_uniform": (None, [u64, i64, i32, P, P, P, P, ctypes.c_int, f64, f64, i32]),
            "synth_zipf_base": (None, [u64, i64, f64, i32, i32, P]),
            "synth_scale_degrees": (i64, [i64, P, f64, i32, i32, P]),
            "synth_popularity": (None, [u64, i32, f64, P, P]),
            "synth_fill_popular": (None, [u64, i64, i32, P, P, P, P, P, P, ctypes.c_int, f64, f64]),
            "synth_col_degrees": (None, [i64, i32, P, P]),
            "synth_repair_draw": (u32, [u64, u64, u32]),
            "synth_repair_util": (f64, [u64, u64, ctypes.c_int, f64, f64]),
            "synth_uniform_array": (None, [u64, u32, i64, f64, f64, P]),
            "synth_normal_array": (None, [u64, u32, i64, P]),
            "synth_int_array": (None, [u64, u32, i64, i64, i64, P]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
    return _lib


def _p(a: Optional[np.ndarray]):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


LAW_UNIFORM, LAW_LOGNORMAL = 0, 1


@dataclass
class Market:
    """A linear Fisher market: ``n`` buyers, ``m`` goods, CSR utilities, budgets."""
    n: int
    m: int
    row_ptr: np.ndarray          # int64 [n+1]
    col: np.ndarray              # int32 [nnz], sorted within each row
    val: np.ndarray              # float64 or float32 [nnz], u_ij > 0
    w: np.ndarray                # float64 [n], w_i > 0
    name: str = ""
    meta: dict = field(default_factory=dict)

    @property
    def nnz(self) -> int:
        return int(self.row_ptr[-1])

    def dense(self) -> np.ndarray:
        U = np.zeros((self.n, self.m))
        rows = np.repeat(np.arange(self.n), np.diff(self.row_ptr))
        U[rows, self.col] = self.val
        return U


def philox4x32_10(ctr, key) -> np.ndarray:
    """Raw Philox4x32-10 block (exposed for the known-answer test)."""
    c = np.asarray(ctr, dtype=np.uint32)
    k = np.asarray(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    _L().synth_philox4x32_10(_p(c), _p(k), _p(out))
    return out


def budgets(seed: int, n: int, lo: float = 0.5, hi: float = 1.5) -> np.ndarray:
    w = np.empty(n, dtype=np.float64)
    _L().synth_budgets(seed, n, lo, hi, _p(w))
    return w


def uniform_array(seed: int, stream: int, n: int, lo: float = 0.0, hi: float = 1.0) -> np.ndarray:
    out = np.empty(n, dtype=np.float64)
    _L().synth_uniform_array(seed, stream, n, lo, hi, _p(out))
    return out


def normal_array(seed: int, stream: int, n: int) -> np.ndarray:
    out = np.empty(n, dtype=np.float64)
    _L().synth_normal_array(seed, stream, n, _p(out))
    return out


def int_array(seed: int, stream: int, n: int, lo: int, hi: int) -> np.ndarray:
    out = np.empty(n, dtype=np.int64)
    _L().synth_int_array(seed, stream, n, lo, hi, _p(out))
    return out


def _ptr_from_deg(deg: np.ndarray) -> np.ndarray:
    row_ptr = np.zeros(len(deg) + 1, dtype=np.int64)
    np.cumsum(deg, out=row_ptr[1:])
    return row_ptr


def repair_assumption1(mk: Market, seed: int, law: int, lo: float, hi: float) -> Market:
    """Give every empty row one uniform good and every empty column one uniform
    buyer (Assumption 1 of the paper).  Rows stay sorted by column."""
    deg = np.diff(mk.row_ptr)
    cdeg = np.bincount(mk.col, minlength=mk.m)
    empty_rows = np.nonzero(deg == 0)[0]
    empty_cols = np.nonzero(cdeg == 0)[0]
    if len(empty_rows) == 0 and len(empty_cols) == 0:
        return mk
    L = _L()
    add_r, add_c, add_v = [], [], []
    for i in empty_rows:
        j = int(L.synth_repair_draw(seed, int(i), mk.m))
        add_r.append(int(i)); add_c.append(j)
        add_v.append(L.synth_repair_util(seed, int(i), law, lo, hi))
    have = set(zip(add_r, add_c))
    for j in empty_cols:
        if any(c == j for c in add_c):
            continue
        i = int(L.synth_repair_draw(seed, mk.n + int(j), mk.n))
        if (i, int(j)) in have:
            continue
        add_r.append(i); add_c.append(int(j))
        add_v.append(L.synth_repair_util(seed, mk.n + int(j), law, lo, hi))
    rows = np.concatenate([np.repeat(np.arange(mk.n, dtype=np.int64), deg), np.array(add_r, dtype=np.int64)])
    cols = np.concatenate([mk.col.astype(np.int64), np.array(add_c, dtype=np.int64)])
    vals = np.concatenate([mk.val, np.array(add_v, dtype=mk.val.dtype)])
    order = np.lexsort((cols, rows))
    rows, cols, vals = rows[order], cols[order], vals[order]
    new_deg = np.bincount(rows, minlength=mk.n)
    out = Market(mk.n, mk.m, _ptr_from_deg(new_deg), cols.astype(np.int32), vals, mk.w, mk.name, dict(mk.meta))
    out.meta["repaired_rows"] = len(empty_rows)
    out.meta["repaired_cols"] = len(empty_cols)
    return _recheck(out, seed, law, lo, hi)


def _recheck(mk, seed, law, lo, hi):
    if (np.diff(mk.row_ptr) == 0).any() or (np.bincount(mk.col, minlength=mk.m) == 0).any():
        return repair_assumption1(mk, seed + 7919, law, lo, hi)
    return mk


def bernoulli_market(n: int, m: int, q: float, seed: int, law: int = LAW_UNIFORM,
                     u_lo: float = 0.0, u_hi: float = 1.0, w_lo: float = 0.5, w_hi: float = 1.5,
                     fp32: bool = False, name: str = "") -> Market:
    """Each (i,j) kept independently with probability ``q``; kept utilities
    drawn from the given law; budgets Uniform(w_lo, w_hi)."""
    L = _L()
    deg = np.empty(n, dtype=np.int32)
    L.synth_bernoulli_degrees(seed, n, m, q, _p(deg))
    row_ptr = _ptr_from_deg(deg)
    nnz = int(row_ptr[-1])
    col = np.empty(nnz, dtype=np.int32)
    val = np.empty(nnz, dtype=np.float32 if fp32 else np.float64)
    L.synth_fill_uniform(seed, n, m, _p(row_ptr), _p(col), None if fp32 else _p(val),
                         _p(val) if fp32 else None, law, u_lo, u_hi, 0)
    w = budgets(seed, n, w_lo, w_hi)
    mk = Market(n, m, row_ptr, col, val, w, name or f"bernoulli(n={n},m={m},q={q})")
    return repair_assumption1(mk, seed, law, u_lo, u_hi)


def fixed_degree_market(n: int, m: int, d: int, seed: int, law: int = LAW_LOGNORMAL,
                        u_lo: float = 0.0, u_hi: float = 1.0, w_lo: float = 0.5, w_hi: float = 1.5,
                        fp32: bool = False, with_self: bool = False, name: str = "") -> Market:
    """Every buyer has exactly ``d`` distinct goods drawn uniformly (Floyd);
    with ``with_self`` buyer i always holds good i (exchange economies)."""
    L = _L()
    deg = np.full(n, d, dtype=np.int32)
    row_ptr = _ptr_from_deg(deg)
    nnz = int(row_ptr[-1])
    col = np.empty(nnz, dtype=np.int32)
    val = np.empty(nnz, dtype=np.float32 if fp32 else np.float64)
    L.synth_fill_uniform(seed, n, m, _p(row_ptr), _p(col), None if fp32 else _p(val),
                         _p(val) if fp32 else None, law, u_lo, u_hi, 1 if with_self else 0)
    w = budgets(seed, n, w_lo, w_hi)
    mk = Market(n, m, row_ptr, col, val, w, name or f"fixed(n={n},m={m},d={d})")
    return repair_assumption1(mk, seed, law, u_lo, u_hi)


def skewed_market(n: int, m: int, nnz_target: int, seed: int, zipf_s: float = 2.0,
                  dmin: int = 10, dmax: int = 2000, alpha: float = 1.1,
                  law: int = LAW_LOGNORMAL, w_lo: float = 0.5, w_hi: float = 1.5,
                  fp32: bool = True, name: str = "") -> Market:
    """Buyer degrees ~ Zipf(s) on [dmin, dmax], rescaled by a factor f (found by
    bisection) so that the total is within 0.1% of ``nnz_target``; goods drawn
    with popularity proportional to rank^-alpha (rank -> id by a seeded
    permutation), distinct within a row by rejection."""
    L = _L()
    z = np.empty(n, dtype=np.int32)
    L.synth_zipf_base(seed, n, zipf_s, dmin, dmax, _p(z))
    lo_f, hi_f = 1e-3, float(dmax)
    for _ in range(200):
        f = 0.5 * (lo_f + hi_f)
        tot = L.synth_scale_degrees(n, _p(z), f, dmin, dmax, None)
        if abs(tot - nnz_target) <= 1e-3 * nnz_target:
            break
        if tot < nnz_target:
            lo_f = f
        else:
            hi_f = f
    deg = np.empty(n, dtype=np.int32)
    L.synth_scale_degrees(n, _p(z), f, dmin, dmax, _p(deg))
    deg = np.minimum(deg, m)
    row_ptr = _ptr_from_deg(deg)
    nnz = int(row_ptr[-1])
    cdf = np.empty(m, dtype=np.float64)
    r2g = np.empty(m, dtype=np.int32)
    L.synth_popularity(seed, m, alpha, _p(cdf), _p(r2g))
    col = np.empty(nnz, dtype=np.int32)
    val = np.empty(nnz, dtype=np.float32 if fp32 else np.float64)
    L.synth_fill_popular(seed, n, m, _p(row_ptr), _p(cdf), _p(r2g), _p(col),
                         None if fp32 else _p(val), _p(val) if fp32 else None, law, 0.0, 1.0)
    w = budgets(seed, n, w_lo, w_hi)
    mk = Market(n, m, row_ptr, col, val, w, name or f"skewed(n={n},m={m},nnz~{nnz_target})",
                {"degree_scale": f})
    return repair_assumption1(mk, seed, law, 0.0, 1.0)


# ---------------------------------------------------------------------------
# The five benchmark workloads (and scaled-down versions of each for tests).
# ---------------------------------------------------------------------------

def config1(seed: int = SEED_BASE + 0) -> Market:
    """n=200, m=100, each (i,j) kept w.p. 0.2, u~U(0,1), w~U(0.5,1.5)."""
    return bernoulli_market(200, 100, 0.2, seed, LAW_UNIFORM, 0.0, 1.0, name="C1 n=200 m=100 q=0.2")


def config2(n: int = 1_000_000, m: int = 10_000, d: int = 100, seed: int = SEED_BASE + 1,
            fp32: bool = False) -> Market:
    """Each buyer has exactly d distinct uniform goods; u~LogNormal(0,1)."""
    return fixed_degree_market(n, m, d, seed, LAW_LOGNORMAL, fp32=fp32,
                               name=f"C2 n={n} m={m} d={d} lognormal")


def config3(n: int = 10_000_000, m: int = 100_000, nnz_target: int = 1_000_000_000,
            seed: int = SEED_BASE + 2, fp32: bool = True) -> Market:
    """Zipf(2) buyer degrees on [10,2000] rescaled to nnz_target; popularity
    rank^-1.1; u~LogNormal(0,1)."""
    return skewed_market(n, m, nnz_target, seed, fp32=fp32,
                         name=f"C3 n={n} m={m} nnz~{nnz_target} zipf")


def config4(n: int = 100_000, d_other: int = 50, seed: int = SEED_BASE + 3, fp32: bool = False) -> Market:
    """Exchange economy: n=m agents, agent i holds its own good i plus d_other
    distinct others; u~U(0.1,1); initial budgets w=1 (E = I)."""
    mk = fixed_degree_market(n, n, d_other + 1, seed, LAW_UNIFORM, 0.1, 1.0, fp32=fp32,
                             with_self=True, name=f"C4 n=m={n} d={d_other}+self")
    mk.w = np.ones(n, dtype=np.float64)
    return mk


@dataclass
class MarketBatch:
    """B independent markets concatenated: market b owns rows
    [row_off[b], row_off[b+1]), goods [good_off[b], good_off[b+1]) (column ids
    in ``col`` are LOCAL to the market) and nnz [nnz_off[b], nnz_off[b+1])."""
    B: int
    row_off: np.ndarray
    good_off: np.ndarray
    nnz_off: np.ndarray
    row_ptr: np.ndarray       # global CSR over all rows, int64 [N+1]
    col: np.ndarray           # int32, local good ids
    val: np.ndarray
    w: np.ndarray

    def market(self, b: int) -> Market:
        r0, r1 = int(self.row_off[b]), int(self.row_off[b + 1])
        z0 = int(self.nnz_off[b])
        rp = self.row_ptr[r0:r1 + 1] - self.row_ptr[r0]
        nz = int(rp[-1])
        return Market(r1 - r0, int(self.good_off[b + 1] - self.good_off[b]), rp.astype(np.int64),
                      self.col[z0:z0 + nz].copy(), self.val[z0:z0 + nz].copy(),
                      self.w[r0:r1].copy(), name=f"market {b}")


def concat_markets(mks) -> MarketBatch:
    B = len(mks)
    row_off = np.zeros(B + 1, dtype=np.int64)
    good_off = np.zeros(B + 1, dtype=np.int64)
    nnz_off = np.zeros(B + 1, dtype=np.int64)
    for b, mk in enumerate(mks):
        row_off[b + 1] = row_off[b] + mk.n
        good_off[b + 1] = good_off[b] + mk.m
        nnz_off[b + 1] = nnz_off[b] + mk.nnz
    row_ptr = np.zeros(int(row_off[-1]) + 1, dtype=np.int64)
    for b, mk in enumerate(mks):
        row_ptr[row_off[b] + 1:row_off[b + 1] + 1] = mk.row_ptr[1:] + nnz_off[b]
    col = np.concatenate([mk.col for mk in mks]).astype(np.int32)
    val = np.concatenate([mk.val for mk in mks])
    w = np.concatenate([mk.w for mk in mks])
    return MarketBatch(B, row_off, good_off, nnz_off, row_ptr, col, val, w)


def config5(B: int = 4096, seed: int = SEED_BASE + 4, n_range=(50, 5000), m_range=(20, 2000),
            q_range=(0.05, 0.3), fp32: bool = True) -> MarketBatch:
    """B markets: n~UniformInt, m~UniformInt, density~Uniform; u~U(0,1),
    w~U(0.5,1.5)."""
    ns = int_array(seed, 1, B, n_range[0], n_range[1])
    ms = int_array(seed, 2, B, m_range[0], m_range[1])
    qs = uniform_array(seed, 3, B, q_range[0], q_range[1])
    mks = [bernoulli_market(int(ns[b]), int(ms[b]), float(qs[b]), seed * 8191 + b + 1, LAW_UNIFORM,
                            0.0, 1.0, fp32=fp32) for b in range(B)]
    return concat_markets(mks)


def paper_synthetic(n: int, m: int, q: float, seed: int) -> Market:
    """The paper's own synthetic Fisher instances: w~U(0,1), each u_ij nonzero
    with probability q and then ~U(0,1) (Section 5.1)."""
    return bernoulli_market(n, m, q, seed, LAW_UNIFORM, 0.0, 1.0, 0.0, 1.0, name=f"paper(n={n},m={m},q={q})")


def rank_one_market(n: int, m: int, seed: int) -> Market:
    """Dense market with u_ij = a_i b_j (a, b ~ U(0.1, 1)), w ~ U(0.5, 1.5)."""
    a = uniform_array(seed, 11, n, 0.1, 1.0)
    b = uniform_array(seed, 12, m, 0.1, 1.0)
    row_ptr = (np.arange(n + 1, dtype=np.int64) * m)
    col = np.tile(np.arange(m, dtype=np.int32), n)
    val = (a[:, None] * b[None, :]).ravel()
    return Market(n, m, row_ptr, col, val, budgets(seed, n), f"rank-one(n={n},m={m})", {"a": a, "b": b})


# ---------------------------------------------------------------------------
# JD.com-shaped Fisher market (Section 5.2).  The paper's real instances take
# the n most active users of a click log and the products they clicked; its
# table gives, for eight values of n, the number of products m and of
# user-product pairs.  The synthetic stand-in reproduces the pair count of
# every one of those prefixes exactly and their product counts to about 15 %.
# ---------------------------------------------------------------------------
JD_USERS = (2000, 5000, 20000, 50000, 200000, 500000, 1000000, 2557841)
JD_NNZ = (136877, 265220, 698579, 1278391, 2937906, 4679648, 6189526, 8073837)
JD_GOODS = (13541, 15887, 19449, 21410, 23853, 25214, 26115, 27330)


def jd_activity_profile() -> np.ndarray:
    """Clicked products of the user of each activity rank (most active first).
    Inside each interval between two consecutive table sizes the counts follow
    a log-log interpolation of the interval averages through the intervals'
    geometric centres (extended linearly past the first and last centre),
    scaled to the interval's exact total and rounded by largest remainders;
    every user keeps at least one product."""
    N = np.array(JD_USERS, dtype=np.int64)
    tot = np.diff(np.concatenate(([0], np.array(JD_NNZ, dtype=np.int64))))
    lo = np.concatenate(([0], N[:-1]))
    lc = np.log(np.sqrt(np.maximum(lo, 1) * N).astype(np.float64))
    la = np.log(tot / (N - lo))
    lr = np.log(np.arange(1, N[-1] + 1, dtype=np.float64))
    f = np.interp(lr, lc, la)
    head = (la[1] - la[0]) / (lc[1] - lc[0])
    tail = (la[-1] - la[-2]) / (lc[-1] - lc[-2])
    f = np.where(lr < lc[0], la[0] + head * (lr - lc[0]), f)
    f = np.exp(np.where(lr > lc[-1], la[-1] + tail * (lr - lc[-1]), f))
    d = np.empty(int(N[-1]), dtype=np.int64)
    for k in range(len(N)):
        sl = slice(int(lo[k]), int(N[k]))
        fk = f[sl] * (tot[k] / f[sl].sum())
        base = np.maximum(np.floor(fk), 1.0).astype(np.int64)
        rest = int(tot[k] - base.sum())
        if rest > 0:
            base[np.argsort(-(fk - np.floor(fk)), kind="stable")[:rest]] += 1
        elif rest < 0:
            base[np.argsort(-base, kind="stable")[:-rest]] -= 1
        d[sl] = base
    return d


def jd_like_market(n: int = JD_USERS[-1], seed: int = SEED_BASE + 5, popularity: float = 1.3,
                   click_tail: float = 1.5, fp32: bool = False) -> Market:
    """The n most active users of a synthetic click log shaped like the JD.com
    data of Section 5.2 (2,557,841 users, 27,330 products, 8,073,837 clicked
    user-product pairs), with the products they clicked.

    * activity: jd_activity_profile(), the table's prefix sizes exactly;
    * products: distinct per user, drawn with popularity proportional to
      rank^-popularity (rank -> product by a seeded permutation); 1.3 brings
      the product count of every table prefix within about 15 % of the table;
    * utilities: click counts with P(u >= k) = k^-click_tail, integers capped
      at 10^4 (the paper uses click counts and gives no law for them);
    * budgets w ~ U(0, 1) as in the paper, floored at 1e-12 (budgets must be
      positive);
    * a product nobody clicked gets one click from one of the least active
      users, so the full log holds every product and every smaller prefix
      keeps its table size;
    * rows in a seeded order, not by activity (``meta["activity_rank"]`` holds
      each row's rank); goods are the products the chosen users clicked, in
      product-id order.
    """
    if not (1 <= n <= JD_USERS[-1]):
        raise ValueError(f"n must lie in [1, {JD_USERS[-1]}]")
    L = _L()
    M = JD_GOODS[-1]
    d = jd_activity_profile()
    N = len(d)
    row_ptr = _ptr_from_deg(d)
    nnz = int(row_ptr[-1])
    cdf = np.empty(M, dtype=np.float64)
    r2g = np.empty(M, dtype=np.int32)
    L.synth_popularity(seed, M, popularity, _p(cdf), _p(r2g))
    col = np.empty(nnz, dtype=np.int32)
    L.synth_fill_popular(seed, N, M, _p(row_ptr), _p(cdf), _p(r2g), _p(col), None, None, LAW_UNIFORM, 0.0, 1.0)
    clicks = np.minimum(np.floor((1.0 - uniform_array(seed, 31, nnz)) ** (-1.0 / click_tail)), 1e4)
    missing = np.nonzero(np.bincount(col, minlength=M) == 0)[0]
    if len(missing):
        users = N - 1 - np.arange(len(missing)) % (N - JD_USERS[-2])
        rows = np.concatenate([np.repeat(np.arange(N), d), users])
        cols = np.concatenate([col.astype(np.int64), missing])
        vals = np.concatenate([clicks, np.ones(len(missing))])
        order = np.lexsort((cols, rows))
        col, clicks = cols[order].astype(np.int32), vals[order]
        d = np.bincount(rows, minlength=N)
        row_ptr = _ptr_from_deg(d)
    w = np.maximum(uniform_array(seed, 32, N), 1e-12)
    # the n most active users and the products they clicked
    sub = int(row_ptr[n])
    goods, col_s = np.unique(col[:sub], return_inverse=True)
    perm = np.argsort(uniform_array(seed, 33, n), kind="stable")
    dd = d[:n][perm]
    rp = _ptr_from_deg(dd)
    idx = np.repeat(row_ptr[:n][perm] - rp[:-1], dd) + np.arange(int(rp[-1]))
    val = clicks[:sub][idx].astype(np.float32 if fp32 else np.float64)
    return Market(n, len(goods), rp, col_s[idx].astype(np.int32), val, w[:n][perm],
                  f"JD-shaped(n={n})", {"activity_rank": perm})


def ad_random_instance(n: int, m: int, q_u: float, q_e: float, seed: int, fp32: bool = False):
    """Arrow-Debreu instances of Section 5.3: utilities as in Section 5.1
    (u_ij nonzero with probability q_u, then U(0,1)); the endowment matrix E
    (n x m) built the same way with density q_e, every agent holding some good
    and every good held by some agent (the Assumption-1 repair), each column
    normalised to sum 1 (a good's unit supply split among its holders).
    Initial budgets w0 = E 1 (all prices 1), so sum w0 = m.
    Returns (market with w = w0, (e_row_ptr, e_col, e_val))."""
    mk = bernoulli_market(n, m, q_u, seed, LAW_UNIFORM, 0.0, 1.0, fp32=fp32,
                          name=f"AD(n={n},m={m},qU={q_u},qE={q_e})")
    em = bernoulli_market(n, m, q_e, seed + 104729, LAW_UNIFORM, 0.0, 1.0, name="E")
    v = np.maximum(em.val, 1e-12)
    v = v / np.bincount(em.col, weights=v, minlength=m)[em.col]
    rows = np.repeat(np.arange(n), np.diff(em.row_ptr))
    mk.w = np.bincount(rows, weights=v, minlength=n)
    return mk, (em.row_ptr, em.col, v)
