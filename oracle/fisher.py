"""FP64 oracle: restarted PDHCG for the linear Fisher market (TEST INFRASTRUCTURE).

Only tests/, __graft_entry__.smoke() and bench.py's cpu_baseline / reference arm
may import this module.  It shares no code with the CUDA path.

Problem (Eisenberg-Gale, Eq. 1 and its PDHCG saddle form, Eq. pdhcg:primal-dual):
    min_{x >= 0} max_p  -sum_i w_i log(u_i^T x_i) + sum_j p_j (sum_i x_ij - 1)
with x stored on the support of U (CSR order).  Notation follows the paper:
n buyers, m goods, budgets w, prices p, step sizes tau (primal), sigma (dual).

Readings of the paper taken here (each is listed in the design notes):
  R1  The row subproblem of Section 2.2 has gradient -w_i u_ij / (u_i^T x_i);
      the printed update omits u_ij.  We use
          x_ij(s) = [x^k_ij - tau p_j + tau w_i u_ij / s]_+          (Eq. bisection, corrected)
      which agrees with the paper's KKT system (Eq. KKT-system-6/7).
  R2  "CG" names the inner solver of PDHCG; for this problem the primal
      subproblem is solved exactly per row (scalar root of phi(s)).
  R4  p is updated first with the extrapolated column sums, then x with the new
      p (Alg. 2).  After a restart there is no extrapolation (x^{-1} := x^0).
  R5  Averages are weighted by the step size eta_k (PDLP convention); this is
      the 1/(k+1) average of Alg. 2 when eta is constant.
  R6  Restarts follow PDLP/PDHCG adaptive restarts with the paper's
      beta_sufficient=0.2, beta_necessary=0.8, beta_artificial=0.2, evaluated
      every ``check_every`` iterations on the relative KKT error.
  R7  Primal weight: omega <- exp(theta log(dp/dx) + (1-theta) log omega),
      theta = 0.2, at each restart; every 3 restarts omega is reset to omega_0
      when it has left [omega_0/100, 100 omega_0].
  R8  Step size: PDLP adaptive rule; eta kept in [0.01 eta_0, 3 eta_0]; a step
      taken at the lower bound is always accepted.
  R9  eta_0 = 0.9/||K||_2 with ||K||_2 = sqrt(max_j deg_j) (K K^T = diag(deg)).
  R10 x^0_ij = 1/deg_j (clears the market), p^0_j = sum(w)/m (so sum p = sum w),
      omega_0 = ||p^0||_2 / ||x^0||_2.
  R12 Relative KKT error of Section 5 with t_i = u_i^T x_i, y = w/t; maxima run
      over the support of U.
  R14 Preprocessing divides each row of U by its maximum (Section 5,
      "Preprocessing"); prices are invariant, utilities are scaled back.
"""
from __future__ import annotations

import math
import time
from dataclasses import dataclass, field
from typing import Optional

import numpy as np


# ---------------------------------------------------------------------------
# Sparse helpers (plain definitions)
# ---------------------------------------------------------------------------

def row_ids(row_ptr: np.ndarray) -> np.ndarray:
    """Row index of every stored entry."""
    n = len(row_ptr) - 1
    return np.repeat(np.arange(n, dtype=np.int64), np.diff(row_ptr))


def column_sums(col: np.ndarray, x: np.ndarray, m: int) -> np.ndarray:
    """c_j = sum_i x_ij (the market-clearing left-hand side, Eq. 1)."""
    return np.bincount(col, weights=x, minlength=m).astype(np.float64)


def row_dot(row_ptr: np.ndarray, u: np.ndarray, x: np.ndarray) -> np.ndarray:
    """t_i = u_i^T x_i (buyer utility, the SpMV of the row subproblem)."""
    n = len(row_ptr) - 1
    return np.bincount(row_ids(row_ptr), weights=u * x, minlength=n).astype(np.float64)


# ---------------------------------------------------------------------------
# Preprocessing (Section 5, "Preprocessing")
# ---------------------------------------------------------------------------

@dataclass
class Scaled:
    n: int
    m: int
    row_ptr: np.ndarray
    col: np.ndarray
    u: np.ndarray          # row-scaled utilities, max of each row = 1
    w: np.ndarray
    rowmax: np.ndarray
    rows: np.ndarray       # row id of each entry
    deg_col: np.ndarray
    groups: list           # rows grouped by degree (see degree_groups)


def preprocess(row_ptr, col, val, w, m) -> Scaled:
    """Divide each buyer's utilities by their maximum so that they lie in (0,1].
    Scaling one buyer's utility function does not change her demand, so prices
    are unchanged; utilities t_i are multiplied back by the row maximum."""
    row_ptr = np.asarray(row_ptr, dtype=np.int64)
    col = np.asarray(col, dtype=np.int64)
    val = np.asarray(val, dtype=np.float64)
    w = np.asarray(w, dtype=np.float64)
    n = len(row_ptr) - 1
    rows = row_ids(row_ptr)
    rowmax = np.zeros(n)
    np.maximum.at(rowmax, rows, val)
    u = val / rowmax[rows]
    deg_col = np.bincount(col, minlength=m).astype(np.int64)
    return Scaled(n, m, row_ptr, col, u, w, rowmax, rows, deg_col, degree_groups(row_ptr))


def validate(row_ptr, col, val, w, m) -> Optional[str]:
    """Assumption 1 plus basic CSR sanity; returns an error message or None."""
    row_ptr = np.asarray(row_ptr)
    n = len(row_ptr) - 1
    if n <= 0 or m <= 0:
        return "empty market"
    if row_ptr[0] != 0 or (np.diff(row_ptr) < 0).any():
        return "row_ptr not monotone"
    nnz = int(row_ptr[-1])
    if len(col) != nnz or len(val) != nnz or len(w) != n:
        return "array lengths"
    if (np.diff(row_ptr) == 0).any():
        return "empty row (Assumption 1)"
    col = np.asarray(col)
    if nnz and (col.min() < 0 or col.max() >= m):
        return "column index out of range"
    if (np.bincount(col, minlength=m) == 0).any():
        return "empty column (Assumption 1)"
    if not np.all(np.isfinite(val)) or (np.asarray(val) <= 0).any():
        return "utility not positive finite"
    if not np.all(np.isfinite(w)) or (np.asarray(w) <= 0).any():
        return "budget not positive finite"
    rows = row_ids(row_ptr)
    same_row = rows[1:] == rows[:-1]
    if (np.diff(col.astype(np.int64))[same_row] <= 0).any():
        return "columns not strictly increasing within a row"
    return None


# ---------------------------------------------------------------------------
# Row subproblem (Section 2.2): exact solution
# ---------------------------------------------------------------------------

def degree_groups(row_ptr):
    """Rows grouped by degree: list of (row ids, entry-index matrix [rows x d])
    so that per-row prefix sums are plain row-wise cumsums."""
    deg = np.diff(row_ptr)
    groups = []
    for d in np.unique(deg):
        r = np.nonzero(deg == d)[0]
        E = row_ptr[r][:, None] + np.arange(d)[None, :]
        groups.append((r, E))
    return groups


def row_prox_exact(groups, n, u, a, cc):
    """Solve, for every row i, the scalar equation of Section 2.2

        s = sum_j u_ij [a_ij + cc_ij / s]_+ ,   a_ij = x^k_ij - tau p_j,
                                                cc_ij = tau w_i u_ij > 0,

    exactly.  With v = 1/s, entry j is active iff v > beta_ij = -a_ij/cc_ij, so on
    the interval between consecutive sorted breakpoints the active set is fixed
    and the equation is the quadratic  C v^2 + A v - 1 = 0  with
    A = sum_active u a, C = sum_active u cc.  F(v) = sum_j u_j[a_j + cc_j v]_+ - 1/v
    is increasing, so the root lies in the first interval whose right end has
    F >= 0.  Returns (s, x_new)."""
    s = np.empty(n)
    x_new = np.empty_like(a)
    for r, E in groups:
        aE, cE, uE = a[E], cc[E], u[E]
        beta = -aE / cE
        order = np.argsort(beta, axis=1, kind="stable")
        b_s = np.take_along_axis(beta, order, axis=1)
        A = np.cumsum(np.take_along_axis(uE * aE, order, axis=1), axis=1)
        C = np.cumsum(np.take_along_axis(uE * cE, order, axis=1), axis=1)
        nxt = np.empty_like(b_s)
        nxt[:, :-1] = b_s[:, 1:]
        nxt[:, -1] = np.inf
        with np.errstate(over="ignore", invalid="ignore"):
            ok = np.isinf(nxt) | ((nxt > 0) & ((A + C * nxt) * nxt >= 1.0))
        k = np.argmax(ok, axis=1)
        idx = np.arange(len(r))
        Ak, Ck = A[idx, k], C[idx, k]
        disc = np.sqrt(Ak * Ak + 4.0 * Ck)
        # positive root of C v^2 + A v - 1 = 0 in the cancellation-free form
        v = np.where(Ak >= 0, 2.0 / (Ak + disc), (disc - Ak) / (2.0 * Ck))
        s[r] = 1.0 / v
        x_new[E] = np.maximum(aE + cE * v[:, None], 0.0)
    return s, x_new


def row_prox_exact_single(u, a, cc):
    """Same as :func:`row_prox_exact` for one row, written as a loop over active
    sets in breakpoint order (used by the brute-force tests)."""
    u, a, cc = (np.asarray(z, dtype=np.float64) for z in (u, a, cc))
    beta = -a / cc
    order = np.argsort(beta, kind="stable")
    A = C = 0.0
    for k, j in enumerate(order):
        A += u[j] * a[j]
        C += u[j] * cc[j]
        right = beta[order[k + 1]] if k + 1 < len(order) else math.inf
        if math.isinf(right) or (right > 0 and (A + C * right) * right >= 1.0):
            disc = math.sqrt(A * A + 4 * C)
            v = 2.0 / (A + disc) if A >= 0 else (disc - A) / (2 * C)
            return 1.0 / v, np.maximum(a + cc * v, 0.0)
    raise AssertionError("unreachable")


def phi(s, u, a, cc):
    """phi(s) = s - sum_j u_j [a_j + cc_j/s]_+  (Section 2.2; increasing in s)."""
    return s - np.sum(u * np.maximum(a + cc / s, 0.0))


def bisection_search(u, a, cc, s0, eps=1e-12, max_rounds=200):
    """Alg. 3 (enhanced bisection) for one row: bracket from s = u^T x^k and the
    image s~ of s, then midpoints, tightening with each image."""
    def image(s):
        xt = np.maximum(a + cc / s, 0.0)
        return float(np.dot(u, xt)), xt
    s = s0
    st, xt = image(s)
    U, L = max(s, st), min(s, st)
    rounds = 0
    while U - L > eps * U and rounds < max_rounds:
        s = 0.5 * (U + L)
        st, xt = image(s)
        U = min(U, max(s, st))
        L = max(L, min(s, st))
        rounds += 1
    return 0.5 * (U + L), xt, rounds


def section_search(u, a, cc, s0, sections=32, eps=1e-12, max_rounds=200):
    """The K-section search of Section 2.2 (K = 32 in the paper): candidates
    s_l = (1 - l/(K+1)) L + l/(K+1) U, l = 1..K; each candidate and its image
    s~_l bracket the root, so U <- min(U, min_l max(s_l, s~_l)) and
    L <- max(L, max_l min(s_l, s~_l))."""
    def img(s):
        return float(np.dot(u, np.maximum(a + cc / s, 0.0)))
    s = s0
    st = img(s)
    U, L = max(s, st), min(s, st)
    rounds = 0
    while U - L > eps * U and rounds < max_rounds:
        ls = np.arange(1, sections + 1) / (sections + 1.0)
        cand = (1 - ls) * L + ls * U
        imgs = np.array([img(c) for c in cand])
        U = min(U, np.min(np.maximum(cand, imgs)))
        L = max(L, np.max(np.minimum(cand, imgs)))
        rounds += 1
    s = 0.5 * (U + L)
    return s, np.maximum(a + cc / s, 0.0), rounds


# ---------------------------------------------------------------------------
# Relative KKT error (Section 5, "Criteria")
# ---------------------------------------------------------------------------

@dataclass
class KKT:
    r_primal: float
    r_dual: float
    r_gap: float

    @property
    def kkt(self) -> float:
        return max(self.r_primal, self.r_dual, self.r_gap)


def kkt_error(sc: Scaled, x: np.ndarray, p: np.ndarray) -> KKT:
    """Relative primal residual, dual residual and primal-dual gap of Section 5
    with t_i = u_i^T x_i and y = w/t (so ||w/t - y|| = |t - u^T x| = 0)."""
    t = row_dot(sc.row_ptr, sc.u, x)
    with np.errstate(divide="ignore"):
        y = sc.w / t
    c = column_sums(sc.col, x, sc.m)
    r_primal = np.max(np.abs(c - 1.0)) / (1.0 + max(np.max(c), 1.0))
    uy = sc.u * y[sc.rows]
    M = np.full(sc.m, -np.inf)
    np.maximum.at(M, sc.col, uy)
    dual_gap = p - M                                 # p_j - max_i u_ij y_i
    num_d = np.max(np.maximum(-dual_gap, 0.0))       # (.)_- = negative part
    den_d = 1.0 + max(np.max(y), np.max(dual_gap))
    r_dual = num_d / den_d
    g = np.maximum(p[sc.col] - uy, 0.0)              # (p_j - u_ij y_i)_+
    r_gap = np.max(x * g) / (1.0 + max(np.max(x), np.max(g)))
    return KKT(float(r_primal), float(r_dual), float(r_gap))


# ---------------------------------------------------------------------------
# Restarted PDHCG (Alg. 2 with the Section 5 enhancements)
# ---------------------------------------------------------------------------

@dataclass
class Params:
    tol: float = 1e-8
    max_iter: int = 200000
    check_every: int = 64
    beta_suff: float = 0.2
    beta_nec: float = 0.8
    beta_art: float = 0.2
    theta: float = 0.2
    eta_lo: float = 0.01
    eta_hi: float = 3.0
    eta0_scale: float = 0.9
    omega_reset_every: int = 3
    omega_range: float = 100.0
    time_limit: float = 1e30


@dataclass
class Result:
    p: np.ndarray            # equilibrium prices (original units)
    t: np.ndarray            # buyer utilities u_i^T x_i (original utilities)
    x: np.ndarray            # allocation on supp U (CSR order)
    kkt: KKT
    iters: int
    passes: int
    restarts: int
    converged: bool
    seconds: float
    history: list = field(default_factory=list)


def initial_point(sc: Scaled):
    """R10: x^0_ij = 1/deg_j, p^0_j = sum(w)/m."""
    x0 = 1.0 / sc.deg_col[sc.col]
    p0 = np.full(sc.m, sc.w.sum() / sc.m)
    return x0, p0


def price_step(p, c_k, c_km1, sigma):
    """Eq. update:py (first line): p_j + sigma (sum_i (2 x^k_ij - x^{k-1}_ij) - 1),
    written with the column sums c^k = sum_i x^k_ij (linearity)."""
    return p + sigma * (2.0 * c_k - c_km1 - 1.0)


def primal_step(sc: Scaled, x, p_new, tau):
    """Alg. 2 line 'parallel update each row': the exact row prox of Section 2.2
    with reading R1.  Returns (x_new, s) with s_i = u_i^T x_new_i."""
    a = x - tau * p_new[sc.col]
    cc = tau * sc.w[sc.rows] * sc.u
    s, x_new = row_prox_exact(sc.groups, sc.n, sc.u, a, cc)
    return x_new, s


def step_size_limit(omega, dx2, dp2, interaction):
    """PDLP adaptive step: eta_max = ||dz||_omega^2 / (2 |dp^T K dx|)."""
    movement = omega * dx2 + dp2 / omega
    if interaction <= 0.0:
        return math.inf
    return movement / (2.0 * interaction)


def next_step_size(eta, eta_max, k):
    """PDLP: eta' = min((1 - (k+1)^-0.3) eta_max, (1 + (k+1)^-0.6) eta); an
    unbounded eta_max (no interaction) leaves only the growth term."""
    grow = (1.0 + (k + 1) ** -0.6) * eta
    if math.isinf(eta_max):
        return grow
    return min((1.0 - (k + 1) ** -0.3) * eta_max, grow)


def restart_decision(kkt_cand, kkt_last_restart, kkt_prev_cand, inner, total, prm: Params):
    """R6: sufficient decay, necessary decay without local progress, or
    artificial restart after a long inner loop."""
    if kkt_cand <= prm.beta_suff * kkt_last_restart:
        return True
    if kkt_cand <= prm.beta_nec * kkt_last_restart and kkt_cand > kkt_prev_cand:
        return True
    if inner >= prm.beta_art * total:
        return True
    return False


def primal_weight_update(omega, dx, dp, theta):
    """R7: exponential smoothing of log(dp/dx)."""
    if dx > 1e-300 and dp > 1e-300:
        return math.exp(theta * math.log(dp / dx) + (1.0 - theta) * math.log(omega))
    return omega


def pdhcg_solve(row_ptr, col, val, w, m, prm: Optional[Params] = None,
                x0: Optional[np.ndarray] = None, p0: Optional[np.ndarray] = None,
                record: bool = False) -> Result:
    """Alg. 2 (restarted PDHCG) in FP64 with the exact row subproblem."""
    prm = prm or Params()
    t_start = time.perf_counter()
    err = validate(row_ptr, col, val, w, m)
    if err:
        raise ValueError(err)
    sc = preprocess(row_ptr, col, val, w, m)
    normK = math.sqrt(float(sc.deg_col.max()))
    eta0 = prm.eta0_scale / normK
    xi, pi = initial_point(sc)
    x = xi if x0 is None else np.asarray(x0, dtype=np.float64).copy()
    p = pi if p0 is None else np.asarray(p0, dtype=np.float64).copy()
    omega0 = float(np.linalg.norm(pi) / np.linalg.norm(xi))
    omega, eta = omega0, eta0
    c_k = column_sums(sc.col, x, m)
    c_km1 = c_k.copy()
    xbar, pbar, sum_eta = x.copy(), p.copy(), 0.0
    x_rs, p_rs = x.copy(), p.copy()
    kk = kkt_error(sc, x, p)
    kkt_rs = kk.kkt
    kkt_prev_cand = math.inf
    total = inner = passes = restarts = 0
    history = []
    best = (kk.kkt, x, p)
    converged = kk.kkt <= prm.tol
    while not converged and total < prm.max_iter:
        # ---- one accepted PDHCG step with the adaptive step-size rule ----
        while True:
            tau, sigma = eta / omega, eta * omega
            p_new = price_step(p, c_k, c_km1, sigma)
            x_new, _ = primal_step(sc, x, p_new, tau)
            c_new = column_sums(sc.col, x_new, m)
            dx = x_new - x
            dp = p_new - p
            interaction = abs(float(np.dot(dp, c_new - c_k)))
            eta_max = step_size_limit(omega, float(np.dot(dx, dx)), float(np.dot(dp, dp)), interaction)
            eta_next = next_step_size(eta, eta_max, total)
            eta_next = min(max(eta_next, prm.eta_lo * eta0), prm.eta_hi * eta0)
            passes += 1
            if eta <= eta_max or eta <= prm.eta_lo * eta0 * (1 + 1e-12):
                break
            eta = eta_next
        eta_used = eta
        eta = eta_next
        x, p, c_km1, c_k = x_new, p_new, c_k, c_new
        sum_eta += eta_used
        wgt = eta_used / sum_eta
        xbar = xbar + wgt * (x - xbar)
        pbar = pbar + wgt * (p - pbar)
        total += 1
        inner += 1
        if total % prm.check_every == 0:
            k_cur = kkt_error(sc, x, p)
            k_avg = kkt_error(sc, xbar, pbar)
            use_avg = k_avg.kkt < k_cur.kkt
            cand_k = k_avg if use_avg else k_cur
            cand_x, cand_p = (xbar, pbar) if use_avg else (x, p)
            if cand_k.kkt < best[0]:
                best = (cand_k.kkt, cand_x.copy(), cand_p.copy())
            if record:
                history.append(dict(iter=total, passes=passes, kkt_cur=k_cur.kkt, kkt_avg=k_avg.kkt,
                                    eta=eta_used, omega=omega))
            if cand_k.kkt <= prm.tol:
                converged = True
                break
            if time.perf_counter() - t_start > prm.time_limit:
                break
            if restart_decision(cand_k.kkt, kkt_rs, kkt_prev_cand, inner, total, prm):
                x, p = cand_x.copy(), cand_p.copy()
                c_k = column_sums(sc.col, x, m)
                c_km1 = c_k.copy()
                restarts += 1
                omega = primal_weight_update(omega, float(np.linalg.norm(x - x_rs)),
                                             float(np.linalg.norm(p - p_rs)), prm.theta)
                if restarts % prm.omega_reset_every == 0:
                    if not (omega0 / prm.omega_range <= omega <= omega0 * prm.omega_range):
                        omega = omega0
                x_rs, p_rs = x.copy(), p.copy()
                xbar, pbar, sum_eta = x.copy(), p.copy(), 0.0
                kkt_rs = cand_k.kkt
                kkt_prev_cand = math.inf
                inner = 0
            else:
                kkt_prev_cand = cand_k.kkt
    _, xb, pb = best
    kb = kkt_error(sc, xb, pb)
    t = row_dot(sc.row_ptr, sc.u, xb) * sc.rowmax
    return Result(pb, t, xb, kb, total, passes, restarts, kb.kkt <= prm.tol,
                  time.perf_counter() - t_start, history)


def solve_market(mk, **kw) -> Result:
    """Convenience wrapper for a ``synth.Market``."""
    prm = Params(**kw)
    return pdhcg_solve(mk.row_ptr, mk.col, mk.val, mk.w, mk.m, prm)
