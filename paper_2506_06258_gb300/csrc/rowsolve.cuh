// Row subproblem of Section 2.2 solved by G lanes of a warp (shared by the
// single-market row kernel and the batched persistent kernel).
//
// FP64 form: phi(s) = s - sum_j u_j [a_j + c_j / s]_+ (a = x - tau p,
// c = tau w u) is increasing.  Freezing the active set S at the current s turns
// the equation into s^2 - A s - C = 0 (A = sum_S u a, C = sum_S u c); its
// positive root is a lower bound of s* (the frozen sum is a minorant that
// touches at s), and iterating "active set -> root" climbs monotonically to
// s*, ending when the active set no longer changes, at which point the root is
// exact.  MIXED form: the same iteration written in y = w/s, on
// cancellation-free residuals (see row_mixed_core).
#pragma once
#include "common.cuh"

namespace pdhcg {

// ---------------------------------------------------------------------------
// positive root of s^2 - A s - C = 0 (C >= 0), cancellation free
// ---------------------------------------------------------------------------
__device__ __forceinline__ double root64(double A, double C) {
    double D = fma(A, A, 4.0 * C);
    double sq = sqrt(fmax(D, 0.0));
    return A >= 0.0 ? 0.5 * (A + sq) : (2.0 * C) / (sq - A);
}

// ---------------------------------------------------------------------------
// column-sum accumulation
// ---------------------------------------------------------------------------
// s: shared-memory accumulators of the hot goods [0, hot); g: global ones
__device__ __forceinline__ void acc_add_fixed(unsigned long long* s, unsigned long long* g, int hot, int j, float x) {
    if (x > 0.0f) {
        unsigned long long v = (unsigned long long)__float2ll_rn(x * kFixScaleF);
        if (j < hot) shared_add_u64(&s[j], v);
        else atomicAdd(&g[j], v);
    }
}
__device__ __forceinline__ void acc_add_f64(unsigned long long* s, unsigned long long* g, int hot, int j, double x) {
    if (x > 0.0) {
        if (j < hot) shared_add_f64(&s[j], x);
        else atomicAdd((double*)&g[j], x);
    }
}

struct RowCtx {
    float tau_hi, tau_lo;
    double tau;
    float fold_w;
    double fold_wd;
    bool fold;
    int cap;
    unsigned seed;      // pass counter mixed into the stochastic-rounding bits
    int sections = 0;   // FP64: 0 = exact active-set root, K >= 2 = K-section search
    double sec_tol = 1e-8;
};

// ---------------------------------------------------------------------------
// MIXED row solve: G lanes per row, row data in registers (d <= G*kSlots;
// longer rows: row_mixed_long below).  Every lane of the warp calls this
// together; `valid` marks real rows.
//
// Unknown y = w / s (the buyer's price of utility).  With d_j = p_j - u_j y the
// row equation of Section 2.2 reads
//     F(y) = sum_j u_j [x_j - tau d_j]_+ - w / y = 0,
// F strictly increasing, F'(y) = tau sum_active u_j^2 + w / y^2 > 0.
// The cancellation of the method sits in d_j (p_j and u_j y agree closely on
// the support near equilibrium, and tau p_j can dwarf x_j), so p is carried in
// float-float, y = y_h + y_l likewise, and
//     d_j = fma(-u, y_l, fma(-u, y_h, p_h) + p_l)
// is exact up to rounding relative to d_j itself.  The sum is split as
//     sum_j u_j [x_j - tau d_j]_+ = s0 - C(y),  s0 = u^T x^k,
//     C(y) = sum_j u_j min(tau d_j, x_j),
// with s0 and w / y in float-float and only the correction C in FP32: its
// rounding error scales with sum_j u_j |min(tau d_j, x_j)|, which shrinks with
// the step x^{k+1} - x^k, so the root is resolved far below the FP32 noise of
// sum u x itself.
// Iteration: with the active set of y_k frozen, C is affine in y
// (slope -tau Q, Q = sum_active u^2), and the frozen equation
//     F_k + tau Q delta + w delta / (y_k (y_k + delta)) = 0
// is a quadratic in delta whose root is taken in cancellation-free form.
// min(tau d_j, x_j) is concave in y, so the frozen model lies below F and its
// root is an upper bound of y*: after the first step the iterates decrease
// monotonically to y* and stop once the active set no longer changes (the
// same finite active-set iteration as the FP64 form, written in y).  Each row
// starts from y_0 = w / t of the previous pass, so s0 and the evaluation at
// y_0 share one sweep; after a frozen-model step whose own rounding error is
// within the final tolerance, a sweep without reductions checks that no entry
// changed activity, which makes the model exact at the new y.  A bracket
// [lo, hi] on the sign of F guards against rounding; stop when |F| is below
// the rounding bound of its evaluation or y no longer moves.
// ---------------------------------------------------------------------------
// Entries of one row held by one lane (register-resident rows).
struct RowRegs {
    long long b, e;
    float u[kSlots], x[kSlots];
    int j[kSlots];
};

template <int G>
__device__ __forceinline__ void row_load(const DevMarket& mk, const float* __restrict__ U,
                                         const float* __restrict__ Xin, int row, bool valid, RowRegs& R) {
    const int tl = (threadIdx.x & 31) & (G - 1);
    R.b = valid ? mk.rp[row] : 0;
    R.e = valid ? mk.rp[row + 1] : 0;
#pragma unroll
    for (int k = 0; k < kSlots; k++) {
        const long long idx = R.b + k * G + tl;
        if (idx < R.e) {
            R.j[k] = __ldg(mk.cj + idx);
            R.u[k] = __ldg(U + idx);
            R.x[k] = __ldcs(Xin + idx);
        } else {
            R.j[k] = -1;
            R.u[k] = 0.0f;
            R.x[k] = 0.0f;
        }
    }
}

// price of good j as float-float: hot goods from shared memory
__device__ __forceinline__ float2 price_ff(const float2* __restrict__ pff, const float2* sp, int hot, int j) {
    return j < hot ? sp[j] : __ldg(pff + j);
}

template <int G>
__device__ void row_mixed_core(const DevMarket& mk, const float* __restrict__ U, const float* __restrict__ Xin,
                               float* __restrict__ Xout, float* __restrict__ Xb, const float2* __restrict__ pff,
                               const float2* sp, unsigned long long* acc_s, unsigned long long* acc_g,
                               double* __restrict__ t_out, const RowCtx& rc, int row, bool valid, float& dx2,
                               int& capped, int& evals, RowRegs& R) {
    const int tl = (threadIdx.x & 31) & (G - 1);
    const long long b = R.b;
    const float tau = rc.tau_hi;
    const double wd = valid ? mk.w[row] : 1.0;

    float rph[kSlots], rpl[kSlots], rtd[kSlots];
    float* ru = R.u;
    float* rx = R.x;
    int* rj = R.j;

#pragma unroll
    for (int k = 0; k < kSlots; k++) {
        if (rj[k] >= 0) {
            const float2 p = price_ff(pff, sp, mk.hot, rj[k]);
            rph[k] = p.x;
            rpl[k] = p.y;
        } else {
            rph[k] = 0.0f;
            rpl[k] = 0.0f;
        }
    }
    // at (yh, yl): C = sum u min(tau d, x), A = sum u |min(tau d, x)|,
    // Q = sum_active u^2, the activity bits (tau d < x, one per entry of this
    // lane); with S: also s0 = u^T x^k
    auto eval = [&](float yh, float yl, float& C, float& A, float& Q, unsigned& act, bool S, ff& s0) {
#pragma unroll
        for (int k = 0; k < kSlots; k++) {
            const float u = ru[k];
            if (S) s0 = ff_add(s0, two_prod(u, rx[k]));
            const float d = fmaf(-u, yl, fmaf(-u, yh, rph[k]) + rpl[k]);
            const float td = tau * d;
            rtd[k] = td;
            const float cr = fminf(td, rx[k]);
            C = fmaf(u, cr, C);
            A = fmaf(u, fabsf(cr), A);
            if (td < rx[k] && rj[k] >= 0) {
                Q = fmaf(u, u, Q);
                act |= 1u << k;
            }
        }
    };

    // ---- start y_0 = w / t of the previous pass (any y > 0 is a valid start) ----
    const ff wff = ff_from_double(wd);
    float yh = 1.0f, yl = 0.0f;
    if (valid) {
        const double tp = t_out[row];
        if (tp > 0.0 && tp < 1e300) {
            const ff y0 = ff_div(wff, ff_from_double(tp));
            if (y0.hi > 0.0f && isfinite(y0.hi)) { yh = y0.hi; yl = y0.lo; }
        }
    }
    // ---- first sweep: s0 and the evaluation at y_0 ----
    ff s0 = ff_make(0.0f, 0.0f);
    float C = 0.0f, A = 0.0f, Q = 0.0f;
    unsigned act = 0u;
    eval(yh, yl, C, A, Q, act, true, s0);
    s0 = group_sum<G>(s0);
    C = group_sum<G>(C);
    A = group_sum<G>(A);
    Q = group_sum<G>(Q);
    // rounding bound of C: a lane adds kSlots terms, then log2(G) levels
    const float cnoise = 1.2e-7f * (sqrtf((float)kSlots) + 3.0f);
    ff lo = ff_make(0.0f, 0.0f), hi = ff_make(INFINITY, 0.0f);   // bracket, in float-float
    float Cf = 0.0f;
    bool done = !valid;
    int steps = 0, nev = 0;
    // every lane of a group holds the group's identical sums, so the lanes of a
    // row take identical decisions; rows of one warp may differ (any-loop)
    while (__any_sync(0xffffffffu, !done)) {
        bool check = false;
        float Cm = 0.0f, aQm = 0.0f;
        ff ym = ff_make(yh, yl);
        if (!done) {
            nev++;
            const ff ws = ff_div(wff, ff_make(yh, yl));    // w / y
            const ff D = ff_sub(s0, ws);
            const float F = (D.hi - C) + D.lo;
            // rounding bound of F: C's FP32 sum, plus the float-float
            // resolution of p and y seen through tau sum u p ~ tau Q y
            const float aQ = tau * Q;
            const float floor = fmaf(cnoise, A, fmaf(3e-14f, aQ * yh, 2e-8f * ws.hi));
            if (fabsf(F) <= floor || ++steps >= rc.cap) {
                done = true;
                Cf = C;
                if (steps >= rc.cap && fabsf(F) > floor && tl == 0 && valid) capped++;
            } else {
                if (F > 0.0f) hi = ff_make(yh, yl); else lo = ff_make(yh, yl);
                // root of the frozen-active-set quadratic a d^2 + b d + c = 0,
                // b = sum u x_new + tau Q y >= 0
                const float bq = fmaf(aQ, yh, F + ws.hi);
                const float cq = F * yh;
                const float disc = fmaf(bq, bq, -4.0f * aQ * cq);
                const float delta = (-2.0f * cq) / (bq + sqrtf(fmaxf(disc, 0.0f)));
                ff yn = ff_add_f(ff_make(yh, yl), delta);
                // the frozen model may replace an evaluation at the new y when
                // its own rounding error is as small as the final tolerance
                check = cnoise * A <= 2e-8f * ws.hi;
                if (!(ff_gt(yn, lo) && ff_gt(hi, yn))) {     // rounding left the bracket
                    yn = isinf(hi.hi) ? ff_make(2.0f * yh, 0.0f) : ff_mul_f(ff_add(lo, hi), 0.5f);
                    check = false;
                }
                if (yn.hi == yh && yn.lo == yl) {
                    done = true;                              // no representable progress
                    Cf = C;
                } else {
                    Cm = C;
                    aQm = aQ;
                    yh = yn.hi;
                    yl = yn.lo;
                }
            }
        }
        // rows that took a model step: does any entry change activity at y?
        if (__any_sync(0xffffffffu, check)) {
            bool chg = false;
#pragma unroll
            for (int k = 0; k < kSlots; k++) {
                const float u = ru[k];
                const float td = tau * fmaf(-u, yl, fmaf(-u, yh, rph[k]) + rpl[k]);
                if (check) {
                    rtd[k] = td;
                    const bool a = td < rx[k] && rj[k] >= 0;
                    chg |= a != ((act >> k) & 1u);
                }
            }
            chg = group_any<G>(chg);
            if (check && !chg) {
                done = true;
                const float dy = (yh - ym.hi) + (yl - ym.lo);
                Cf = Cm - aQm * dy;
            }
        }
        // evaluation at the current y for rows still open
        if (__any_sync(0xffffffffu, !done)) {
            C = A = Q = 0.0f;
            unsigned an = 0u;
            ff dummy = ff_make(0.0f, 0.0f);
            if (!done) eval(yh, yl, C, A, Q, an, false, dummy);
            C = group_sum<G>(C);
            A = group_sum<G>(A);
            Q = group_sum<G>(Q);
            if (!done) act = an;
        }
    }
    if (valid && tl == 0) {
        t_out[row] = ((double)s0.hi + (double)s0.lo) - (double)Cf;
        evals += nev;
    }

    // ---- new iterate (at the final y), average fold, column sums ----
    const float fw = rc.fold_w;
#pragma unroll
    for (int k = 0; k < kSlots; k++) {
        if (rj[k] < 0) continue;
        const long long idx = b + k * G + tl;
        const float td = rtd[k];
        const unsigned rb = sr_bits(idx, rc.seed);
        // x^{k+1} = [x^k - tau d]_+, stochastically rounded
        const float xn = td < rx[k] ? sr_add(rx[k], -td, rb) : 0.0f;
        __stcs(Xout + idx, xn);
        const float d = xn - rx[k];
        dx2 = fmaf(d, d, dx2);
        if (rc.fold) {
            const float xb = Xb[idx];
            Xb[idx] = (fw == 1.0f) ? rx[k] : sr_add(xb, fw * (rx[k] - xb), rb >> 16);
        }
        acc_add_fixed(acc_s, acc_g, mk.hot, rj[k], xn);
    }
}

// ---------------------------------------------------------------------------
// MIXED row solve for rows longer than 32*kSlots entries: one warp per row,
// the row streamed in chunks of 32*kSlots entries and re-read (from L2) on
// every sweep.  Iteration, stopping rule and rounding are those of
// row_mixed_core, entry for entry; what differs is the number of sweeps:
//  - x-bar is folded during the first sweep (the fold needs x^k only);
//  - the first activity check (after a frozen-model step) writes x^{k+1}, its
//    column sums and ||dx||^2 at the new y chunk by chunk behind the check.
//    When no entry changes activity that y is final and no separate write
//    sweep follows; at the first chunk that shows a change the check stops,
//    the column-sum contributions of the chunks already written are
//    subtracted again (exact: the sums are fixed-point integers), ||dx||^2 is
//    restored, and the iteration continues without further speculation.
// Every lane of the warp calls this with the same row.
// ---------------------------------------------------------------------------
__device__ inline void row_mixed_long(const DevMarket& mk, const float* __restrict__ U, const float* __restrict__ Xin,
                               float* __restrict__ Xout, float* __restrict__ Xb, const float2* __restrict__ pff,
                               const float2* sp, unsigned long long* acc_s, unsigned long long* acc_g,
                               double* __restrict__ t_out, const RowCtx& rc, int row, bool valid, float& dx2,
                               int& capped, int& evals) {
    if (!valid) return;
    const int lane = threadIdx.x & 31;
    constexpr int span = 32 * kSlots;
    const long long b = mk.rp[row];
    const long long e = mk.rp[row + 1];
    const int nch = (int)((e - b + span - 1) / span);
    const float tau = rc.tau_hi;

    float ru[kSlots], rx[kSlots], rph[kSlots], rpl[kSlots], rtd[kSlots];
    int rj[kSlots];
    auto load_chunk = [&](int c) {
#pragma unroll
        for (int k = 0; k < kSlots; k++) {
            const long long idx = b + (long long)c * span + k * 32 + lane;
            if (idx < e) {
                rj[k] = __ldg(mk.cj + idx);
                ru[k] = __ldg(U + idx);
                rx[k] = Xin[idx];
            } else {
                rj[k] = -1; ru[k] = 0.0f; rx[k] = 0.0f;
            }
        }
#pragma unroll
        for (int k = 0; k < kSlots; k++) {
            if (rj[k] >= 0) {
                const float2 p = price_ff(pff, sp, mk.hot, rj[k]);
                rph[k] = p.x;
                rpl[k] = p.y;
            } else {
                rph[k] = 0.0f;
                rpl[k] = 0.0f;
            }
        }
    };
    auto td_at = [&](int k, float yh, float yl) -> float {
        return tau * fmaf(-ru[k], yl, fmaf(-ru[k], yh, rph[k]) + rpl[k]);
    };
    // x^{k+1} of the loaded chunk from rtd: store, ||dx||^2, column sums; with
    // undo, subtract the column-sum contributions written by the same call
    auto write_chunk = [&](int c, bool undo) {
#pragma unroll
        for (int k = 0; k < kSlots; k++) {
            if (rj[k] < 0) continue;
            const long long idx = b + (long long)c * span + k * 32 + lane;
            const float td = rtd[k];
            const float xn = td < rx[k] ? sr_add(rx[k], -td, sr_bits(idx, rc.seed)) : 0.0f;
            if (!undo) {
                __stcs(Xout + idx, xn);
                const float d = xn - rx[k];
                dx2 = fmaf(d, d, dx2);
                acc_add_fixed(acc_s, acc_g, mk.hot, rj[k], xn);
            } else if (xn > 0.0f) {
                const unsigned long long v = 0ull - (unsigned long long)__float2ll_rn(xn * kFixScaleF);
                if (rj[k] < mk.hot) shared_add_u64(&acc_s[rj[k]], v);
                else atomicAdd(&acc_g[rj[k]], v);
            }
        }
    };
    auto undo_chunks = [&](int cw, float yh, float yl) {
        for (int c = 0; c < cw; c++) {
            load_chunk(c);
#pragma unroll
            for (int k = 0; k < kSlots; k++) rtd[k] = td_at(k, yh, yl);
            write_chunk(c, true);
        }
    };
    auto bit = [&](int c, int k) -> unsigned long long { return 1ull << ((c * kSlots + k) & 63); };
    const bool track = nch * kSlots <= 64;

    // ---- start y_0 = w / t of the previous pass ----
    const ff wff = ff_from_double(mk.w[row]);
    float yh = 1.0f, yl = 0.0f;
    {
        const double tp = t_out[row];
        if (tp > 0.0 && tp < 1e300) {
            const ff y0 = ff_div(wff, ff_from_double(tp));
            if (y0.hi > 0.0f && isfinite(y0.hi)) { yh = y0.hi; yl = y0.lo; }
        }
    }
    // ---- first sweep: s0, the evaluation at y_0, the x-bar fold ----
    const float fw = rc.fold_w;
    ff s0 = ff_make(0.0f, 0.0f);
    float C = 0.0f, A = 0.0f, Q = 0.0f;
    unsigned long long act = 0ull;
    for (int c = 0; c < nch; c++) {
        load_chunk(c);
#pragma unroll
        for (int k = 0; k < kSlots; k++) {
            const float u = ru[k];
            s0 = ff_add(s0, two_prod(u, rx[k]));
            const float td = td_at(k, yh, yl);
            const float cr = fminf(td, rx[k]);
            C = fmaf(u, cr, C);
            A = fmaf(u, fabsf(cr), A);
            if (td < rx[k] && rj[k] >= 0) {
                Q = fmaf(u, u, Q);
                act |= bit(c, k);
            }
            if (rc.fold && rj[k] >= 0) {
                const long long idx = b + (long long)c * span + k * 32 + lane;
                const float xb = Xb[idx];
                Xb[idx] = (fw == 1.0f) ? rx[k] : sr_add(xb, fw * (rx[k] - xb), sr_bits(idx, rc.seed) >> 16);
            }
        }
    }
    s0 = group_sum<32>(s0);
    C = group_sum<32>(C);
    A = group_sum<32>(A);
    Q = group_sum<32>(Q);
    const float cnoise = 1.2e-7f * (sqrtf((float)(nch * kSlots)) + 3.0f);
    ff lo = ff_make(0.0f, 0.0f), hi = ff_make(INFINITY, 0.0f);
    float Cf = 0.0f;
    int steps = 0, nev = 0;
    bool spec = true;        // the next activity check may write x^{k+1} behind it
    bool written = false;    // x^{k+1} written at the final y
    while (true) {
        nev++;
        const ff ws = ff_div(wff, ff_make(yh, yl));
        const ff D = ff_sub(s0, ws);
        const float F = (D.hi - C) + D.lo;
        const float aQ = tau * Q;
        const float floor = fmaf(cnoise, A, fmaf(3e-14f, aQ * yh, 2e-8f * ws.hi));
        if (fabsf(F) <= floor || ++steps >= rc.cap) {
            Cf = C;
            if (steps >= rc.cap && fabsf(F) > floor && lane == 0) capped++;
            break;
        }
        if (F > 0.0f) hi = ff_make(yh, yl); else lo = ff_make(yh, yl);
        const float bq = fmaf(aQ, yh, F + ws.hi);
        const float cq = F * yh;
        const float disc = fmaf(bq, bq, -4.0f * aQ * cq);
        const float delta = (-2.0f * cq) / (bq + sqrtf(fmaxf(disc, 0.0f)));
        ff yn = ff_add_f(ff_make(yh, yl), delta);
        bool check = track && cnoise * A <= 2e-8f * ws.hi;
        if (!(ff_gt(yn, lo) && ff_gt(hi, yn))) {
            yn = isinf(hi.hi) ? ff_make(2.0f * yh, 0.0f) : ff_mul_f(ff_add(lo, hi), 0.5f);
            check = false;
        }
        if (yn.hi == yh && yn.lo == yl) {                    // no representable progress
            Cf = C;
            break;
        }
        const float Cm = C, aQm = aQ;
        const ff ym = ff_make(yh, yl);
        yh = yn.hi;
        yl = yn.lo;
        if (check) {
            // does any entry change activity at y?  Chunk by chunk, writing
            // x^{k+1} behind the check while nothing has changed
            const bool wr = spec;
            spec = false;
            const float dsave = dx2;
            bool chg = false;
            int cw = 0;
            for (int c = 0; c < nch; c++) {
                load_chunk(c);
                bool cc = false;
#pragma unroll
                for (int k = 0; k < kSlots; k++) {
                    rtd[k] = td_at(k, yh, yl);
                    const bool a = rtd[k] < rx[k] && rj[k] >= 0;
                    cc |= a != ((act & bit(c, k)) != 0ull);
                }
                if (__any_sync(0xffffffffu, cc)) {
                    chg = true;
                    break;
                }
                if (wr) {
                    write_chunk(c, false);
                    cw = c + 1;
                }
            }
            if (!chg) {
                const float dy = (yh - ym.hi) + (yl - ym.lo);
                Cf = Cm - aQm * dy;
                written = wr;
                break;
            }
            if (wr) {
                undo_chunks(cw, yh, yl);
                dx2 = dsave;
            }
        }
        // evaluation at y
        C = A = Q = 0.0f;
        act = 0ull;
        for (int c = 0; c < nch; c++) {
            load_chunk(c);
#pragma unroll
            for (int k = 0; k < kSlots; k++) {
                const float u = ru[k];
                const float td = td_at(k, yh, yl);
                rtd[k] = td;
                const float cr = fminf(td, rx[k]);
                C = fmaf(u, cr, C);
                A = fmaf(u, fabsf(cr), A);
                if (td < rx[k] && rj[k] >= 0) {
                    Q = fmaf(u, u, Q);
                    act |= bit(c, k);
                }
            }
        }
        C = group_sum<32>(C);
        A = group_sum<32>(A);
        Q = group_sum<32>(Q);
    }
    if (lane == 0) {
        t_out[row] = ((double)s0.hi + (double)s0.lo) - (double)Cf;
        evals += nev;
    }
    if (written) return;
    // ---- new iterate at the final y, column sums ----
    for (int c = 0; c < nch; c++) {
        load_chunk(c);
#pragma unroll
        for (int k = 0; k < kSlots; k++) rtd[k] = td_at(k, yh, yl);
        write_chunk(c, false);
    }
}

// Convenience form (loads the row itself): used by the batched kernel.
template <int G, bool LONG>
__device__ void row_mixed(const DevMarket& mk, const float* __restrict__ U, const float* __restrict__ Xin,
                          float* __restrict__ Xout, float* __restrict__ Xb, const float2* __restrict__ pff,
                          unsigned long long* acc_s, unsigned long long* acc_g, double* __restrict__ t_out,
                          const RowCtx& rc, int row, bool valid, float& dx2, int& capped, int& evals) {
    if (LONG) {
        row_mixed_long(mk, U, Xin, Xout, Xb, pff, pff, acc_s, acc_g, t_out, rc, row, valid, dx2, capped, evals);
    } else {
        RowRegs R;
        row_load<G>(mk, U, Xin, row, valid, R);
        row_mixed_core<G>(mk, U, Xin, Xout, Xb, pff, pff, acc_s, acc_g, t_out, rc, row, valid, dx2, capped, evals, R);
    }
}

// ---------------------------------------------------------------------------
// FP64 row solve (plain form): the same active-set iteration in double.
// ---------------------------------------------------------------------------
template <int G, bool LONG>
__device__ void row_fp64(const DevMarket& mk, const double* __restrict__ U, const double* __restrict__ Xin,
                         double* __restrict__ Xout, double* __restrict__ Xb, const double* __restrict__ pc,
                         unsigned long long* acc_s, unsigned long long* acc_g, double* __restrict__ t_out,
                         const RowCtx& rc, int row, bool valid, double& dx2, int& capped) {
    const int tl = (threadIdx.x & 31) & (G - 1);
    const long long b = valid ? mk.rp[row] : 0;
    const long long e = valid ? mk.rp[row + 1] : 0;
    const double wi = valid ? mk.w[row] : 1.0;
    const double tw = rc.tau * wi;
    const int span = G * kSlots;
    const int nch = LONG ? (int)((e - b + span - 1) / span) : 1;
    double ru[kSlots], rx[kSlots], ra[kSlots];
    int rj[kSlots];
    bool rin[kSlots];
    auto load_chunk = [&](int c) {
#pragma unroll
        for (int k = 0; k < kSlots; k++) {
            long long idx = b + (long long)c * span + k * G + tl;
            rin[k] = idx < e;
            if (rin[k]) {
                int j = __ldg(mk.cj + idx);
                double u = __ldg(U + idx);
                double x = Xin[idx];
                rj[k] = j; ru[k] = u; rx[k] = x; ra[k] = x - rc.tau * pc[j];   // pc may live in shared memory
            } else {
                rj[k] = 0; ru[k] = 0.0; rx[k] = 0.0; ra[k] = 0.0;
            }
        }
    };
    double s0 = 0.0, qall = 0.0;
    for (int c = 0; c < nch; c++) {
        if (LONG || c == 0) load_chunk(c);
#pragma unroll
        for (int k = 0; k < kSlots; k++) { s0 = fma(ru[k], rx[k], s0); qall = fma(ru[k], ru[k], qall); }
    }
    s0 = group_sum<G>(s0);
    qall = group_sum<G>(qall);
    if (!(s0 > 0.0)) s0 = sqrt(tw * qall);
    if (!(s0 > 0.0)) s0 = 1.0;
    double s = s0, s_last = -1.0;
    bool gdone = !valid;
    int rounds = 0;
    if (rc.sections > 0) {
        // K-section search of Section 2.2: s* lies between any s and its image
        // s~(s) = sum_j u_j [a_j + tw u_j / s]_+ (s~ is decreasing), so each of
        // the K candidates s_l = L + l (U - L) / (K + 1) with its image brackets
        // the root: U <- min_l max(s_l, s~_l), L <- max_l min(s_l, s~_l); stop
        // when U - L <= sec_tol U; s = (L + U) / 2
        auto img = [&](double sv) -> double {
            const double R = tw / sv;
            double acc = 0.0;
            for (int c = 0; c < nch; c++) {
                if (LONG) load_chunk(c);
#pragma unroll
                for (int k = 0; k < kSlots; k++)
                    if (rin[k]) acc = fma(ru[k], fmax(fma(ru[k], R, ra[k]), 0.0), acc);
            }
            return group_sum<G>(acc);
        };
        const double st0 = img(s0);
        double U = fmax(s0, st0), L = fmin(s0, st0);
        if (!(U - L > rc.sec_tol * U)) gdone = true;
        const int K = rc.sections;
        while (__any_sync(0xffffffffu, !gdone)) {
            double nU = U, nL = L;
            for (int l = 1; l <= K; l++) {
                const double sl = fmax(L + (U - L) * ((double)l / (double)(K + 1)), 1e-300);
                const double st = img(sl);
                nU = fmin(nU, fmax(sl, st));
                nL = fmax(nL, fmin(sl, st));
            }
            if (!gdone) {
                U = nU;
                L = nL;
                if (!(U - L > rc.sec_tol * U)) gdone = true;
                else if (++rounds >= rc.cap) { gdone = true; if (tl == 0 && valid) capped++; }
            }
        }
        s = 0.5 * (U + L);
        gdone = true;
    }
    while (__any_sync(0xffffffffu, !gdone)) {
        const double R = tw / s;
        double A = 0.0, Q = 0.0;
        for (int c = 0; c < nch; c++) {
            if (LONG) load_chunk(c);
#pragma unroll
            for (int k = 0; k < kSlots; k++) {
                if (rin[k] && fma(ru[k], R, ra[k]) > 0.0) {
                    A = fma(ru[k], ra[k], A);
                    Q = fma(ru[k], ru[k], Q);
                }
            }
        }
        A = group_sum<G>(A);
        Q = group_sum<G>(Q);
        if (!gdone) {
            double sn = root64(A, tw * Q);
            if (sn == s_last) {
                gdone = true;
            } else {
                s = (rounds == 0) ? sn : fmax(s, sn);
                s_last = sn;
                if (++rounds >= rc.cap) { gdone = true; if (tl == 0 && valid) capped++; }
            }
        }
    }
    const double R = tw / s;
    const double fw = rc.fold_wd;
    for (int c = 0; c < nch; c++) {
        if (LONG) load_chunk(c);
#pragma unroll
        for (int k = 0; k < kSlots; k++) {
            if (!rin[k]) continue;
            long long idx = b + (long long)c * span + k * G + tl;
            double xn = fmax(fma(ru[k], R, ra[k]), 0.0);
            Xout[idx] = xn;
            double d = xn - rx[k];
            dx2 = fma(d, d, dx2);
            if (rc.fold) Xb[idx] = (fw == 1.0) ? rx[k] : fma(fw, rx[k] - Xb[idx], Xb[idx]);
            acc_add_f64(acc_s, acc_g, mk.hot, rj[k], xn);
        }
    }
    if (valid && tl == 0) t_out[row] = s;
}

}  // namespace pdhcg
