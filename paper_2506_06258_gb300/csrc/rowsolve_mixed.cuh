// MIXED row subproblem of Section 2.2 for the single-market row kernel.
//
// Unknown y = w / s (the buyer's price of utility).  With d_j = p_j - u_j y the
// row equation of Section 2.2 (utility factor u_ij restored, as in Eq.
// KKT-system-6) is S(y) = w / y with
//     S(y) = sum_j u_j [x_j - tau d_j]_+ ,
// S convex and nondecreasing in y.  The root is found on
//     G(y) = y S(y) - w ,
// strictly increasing for y > 0, with no division anywhere: with the active
// set of y_k frozen, S is its tangent s0 - C_k + tau Q (y - y_k) (a minorant,
// as S is convex), so the frozen G is the quadratic
//     H(delta) = tau Q delta^2 + b delta + G(y_k),   b = s0 - C_k + tau Q y_k,
// whose root lies above the root of G: after the first step the iterates
// decrease monotonically to y*, and stop once the active set no longer
// changes (the model is then exact).
//   Cancellation: near equilibrium p_j ~ u_j y on the support and tau p_j can
// dwarf x_j.  p and y are float-float and d_j = fma(-u, y_lo, fma(-u, y_hi,
// p_hi) + p_lo) is exact up to rounding relative to d_j itself.  The sum is
// split as S = s0 - C(y), s0 = u^T x^k exactly in float-float and only the
// small correction C(y) = sum_j u_j min(tau d_j, x_j) in FP32, so G(y) =
// y (s0 - C) - w is resolved far below the FP32 noise of u^T x itself.
//   Activity is monotone in y for every entry (tau d_j falls as y rises), so
// after a step in y the active set is unchanged exactly when every lane's
// count of active entries is unchanged: the activity check compares counts.
//   Warm start: y_0 of each row is the y of the previous pass (stored per row
// as float-float, no conversion).  After a frozen-model step whose result is
// accurate to the final tolerance (small step, small rounding noise in C), a
// sweep without reductions checks the activity and then the model is exact;
// otherwise a new evaluation follows.  A float-float bracket on the sign of G
// guards against rounding.
//   No FP64 instruction runs here (FP64 is a slow pipe on this GPU): budgets
// and y live in float-float, reductions are float-float or FP32.
#pragma once
#include "common.cuh"
#include "rowsolve.cuh"

namespace pdhcg {

// Upper limit of y = w / s: beyond it the row is reported as capped rather
// than letting y, and with it x = [x - tau (p - u y)]_+, overflow.
constexpr float kYMax = 1e30f;

struct RowCtxM {
    float tau;
    int cap;
    unsigned seed;      // pass counter mixed into the stochastic-rounding bits
};

// A row's entries, G lanes per row: lane tl holds entries tl, tl + G, ...
// Addresses are formed once per row (64-bit base + lane); the slots then
// differ by compile-time offsets, and bounds are 32-bit.
struct RowRegsM {
    long long b;        // first entry of the row
    int d;              // entries in the row
    float u[kSlots], x[kSlots];
    int j[kSlots];
};

template <int G>
__device__ __forceinline__ void rowm_load(const DevMarket& mk, const float* __restrict__ U,
                                          const float* __restrict__ Xin, int row, bool valid, RowRegsM& R) {
    const int tl = (threadIdx.x & 31) & (G - 1);
    const long long b = valid ? mk.rp[row] : 0;
    R.b = b;
    R.d = valid ? (int)(mk.rp[row + 1] - b) : 0;
    const int* __restrict__ cp = mk.cj + b + tl;
    const float* __restrict__ up = U + b + tl;
    const float* __restrict__ xp = Xin + b + tl;
#pragma unroll
    for (int k = 0; k < kSlots; k++) {
        if (k * G + tl < R.d) {
            R.j[k] = __ldg(cp + k * G);
            R.u[k] = __ldg(up + k * G);
            R.x[k] = __ldcs(xp + k * G);
        } else {
            R.j[k] = -1;
            R.u[k] = 0.0f;
            R.x[k] = 0.0f;
        }
    }
}

// G(y) = y (s0 - C) - w in float-float
__device__ __forceinline__ float rowm_G(ff s0, float C, ff y, ff w, float& sc_hi) {
    const ff sc = ff_add_f(s0, -C);
    sc_hi = sc.hi;
    const ff g = ff_sub(ff_mul(sc, y), w);
    return g.hi + g.lo;
}

// Root of the frozen model: delta (FP32; approximate reciprocal and square
// root, a few ulp, which the acceptance test of the caller allows for).
// Returns false when the model has no root: with no active entry (Q = 0)
// every term of S is zero, so S = 0 exactly (s0 - C is then rounding noise)
// and the frozen G is the constant -w; the caller doubles y or bisects.
__device__ __forceinline__ bool rowm_delta(float Gf, float sc_hi, float aQ, float yh, float& delta) {
    if (!(aQ > 0.0f)) return false;
    const float b = fmaf(aQ, yh, sc_hi);
    const float disc = fmaf(b, b, -4.0f * aQ * Gf);
    const float sq = disc > 0.0f ? disc * rsqrtf(disc) : 0.0f;
    const float den = b + sq;
    if (!(den > 0.0f)) return false;
    delta = __fdividef(-2.0f * Gf, den);
    return isfinite(delta);
}

// Column-sum contribution of a stored x (exact 64-bit fixed point); sign -1 undoes it.
__device__ __forceinline__ void rowm_acc(unsigned long long* s, unsigned long long* g, int hot, int j, float x,
                                         bool undo) {
    if (x > 0.0f) {
        unsigned long long v = (unsigned long long)__float2ll_rn(x * kFixScaleF);
        if (undo) v = 0ull - v;
        if (j < hot) shared_add_u64(&s[j], v);
        else atomicAdd(&g[j], v);
    }
}

// ---------------------------------------------------------------------------
// register-resident rows: G lanes per row, d <= G * kSlots
// ---------------------------------------------------------------------------
template <int G>
__device__ void rowm_core(const DevMarket& mk, float* __restrict__ Xout, const float2* __restrict__ pff, const float2* sp, unsigned long long* acc_s,
                          unsigned long long* acc_g, float2* __restrict__ yst, const RowCtxM& rc, int row, bool valid,
                          float& dx2, int& capped, int& evals, RowRegsM& R) {
    const int tl = (threadIdx.x & 31) & (G - 1);
    const float tau = rc.tau;
    float rph[kSlots], rpl[kSlots], rtd[kSlots];
    const float* ru = R.u;
    const float* rx = R.x;
    const int* rj = R.j;
#pragma unroll
    for (int k = 0; k < kSlots; k++) {
        // selects, not a branch per slot: padding slots gather good 0 and zero it
        const bool ok = rj[k] >= 0;
        const float2 p = price_ff(pff, sp, mk.hot, ok ? rj[k] : 0);
        rph[k] = ok ? p.x : 0.0f;
        rpl[k] = ok ? p.y : 0.0f;
    }
    const float2 wv = valid ? mk.wff[row] : make_float2(1.0f, 0.0f);
    float2 y0 = valid ? yst[row] : make_float2(1.0f, 0.0f);
    if (!(y0.x > 0.0f) || !isfinite(y0.x)) y0 = make_float2(1.0f, 0.0f);
    const ff W = ff_make(wv.x, wv.y);
    float yh = y0.x, yl = y0.y;

    // ---- first sweep: s0 = u^T x^k (float-float) and the evaluation at y_0 ----
    // padding slots have u = x = p = 0: they are never active and add nothing
    float s0h = 0.0f, s0l = 0.0f, C = 0.0f, A = 0.0f, Q = 0.0f;
    int cnt = 0;
#pragma unroll
    for (int k = 0; k < kSlots; k++) {
        const float u = ru[k], x = rx[k];
        const ff pr = two_prod(u, x);
        const ff t = two_sum(s0h, pr.hi);
        s0h = t.hi;
        s0l += t.lo + pr.lo;
        const float td = tau * fmaf(-u, yl, fmaf(-u, yh, rph[k]) + rpl[k]);
        rtd[k] = td;
        const float cr = fminf(td, x);
        C = fmaf(u, cr, C);
        A = fmaf(u, fabsf(cr), A);
        if (td < x) {
            Q = fmaf(u, u, Q);
            cnt++;
        }
    }
    ff s0 = group_sum<G>(ff_make(s0h, s0l));
    C = group_sum<G>(C);
    A = group_sum<G>(A);
    Q = group_sum<G>(Q);
    const float cnoise = 1.2e-7f * (sqrtf((float)kSlots) + 3.0f);   // rounding bound of C per unit of A
    ff lo = ff_make(0.0f, 0.0f), hi = ff_make(INFINITY, 0.0f);
    bool done = !valid;
    int steps = 0, nev = 0;
    // every lane of a group holds the group's sums, so the lanes of a row take
    // identical decisions; rows of one warp may differ (any-loops)
    while (__any_sync(0xffffffffu, !done)) {
        bool check = false;
        if (!done) {
            nev++;
            const ff Y = ff_make(yh, yl);
            float sch;
            const float Gf = rowm_G(s0, C, Y, W, sch);
            const float aQ = tau * Q;
            // rounding bound of G: y times (C's FP32 sum + the float-float
            // resolution of p and y seen through tau Q y + that of s0 and w/y)
            const float floor = fmaf(cnoise * A, yh, fmaf(3e-14f * aQ * yh, yh, 2e-8f * W.hi));
            if (fabsf(Gf) <= floor || ++steps >= rc.cap || !(yh < kYMax)) {
                done = true;
                if (!(fabsf(Gf) <= floor) && tl == 0 && valid) capped++;
            } else {
                // G increases with y; a non-finite G comes from overflow at a
                // far too large y
                if (!(Gf <= 0.0f)) hi = Y; else lo = Y;
                float delta = 0.0f;
                const bool root = rowm_delta(Gf, sch, aQ, yh, delta);
                ff yn = root ? ff_add_f(Y, delta) : Y;
                // the model root replaces an evaluation at yn when both the
                // step (FP32, a few ulp) and C's rounding are within tolerance
                check = cnoise * A * yh <= 2e-8f * W.hi && fabsf(delta) <= 0.0625f * yh;
                if (!root || !(ff_gt(yn, lo) && ff_gt(hi, yn))) {     // no model root, or outside the bracket
                    yn = isinf(hi.hi) ? ff_make(2.0f * yh, 0.0f) : ff_mul_f(ff_add(lo, hi), 0.5f);
                    check = false;
                }
                if (yn.hi == yh && yn.lo == yl) {
                    done = true;                              // no representable progress
                } else {
                    yh = yn.hi;
                    yl = yn.lo;
                }
            }
        }
        // rows that took a model step: does any entry change activity at y?
        if (__any_sync(0xffffffffu, check)) {
            int cn = 0;
            float ntd[kSlots];
#pragma unroll
            for (int k = 0; k < kSlots; k++) {
                const float u = ru[k];
                ntd[k] = tau * fmaf(-u, yl, fmaf(-u, yh, rph[k]) + rpl[k]);
                cn += ntd[k] < rx[k] ? 1 : 0;
            }
            const bool chg = group_any<G>(check && cn != cnt);
            if (check && !chg) {
                done = true;
#pragma unroll
                for (int k = 0; k < kSlots; k++) rtd[k] = ntd[k];
            }
        }
        // evaluation at the current y for rows still open
        if (__any_sync(0xffffffffu, !done)) {
            float Cn = 0.0f, An = 0.0f, Qn = 0.0f;
            int cn = 0;
            if (!done) {
#pragma unroll
                for (int k = 0; k < kSlots; k++) {
                    const float u = ru[k], x = rx[k];
                    const float td = tau * fmaf(-u, yl, fmaf(-u, yh, rph[k]) + rpl[k]);
                    rtd[k] = td;
                    const float cr = fminf(td, x);
                    Cn = fmaf(u, cr, Cn);
                    An = fmaf(u, fabsf(cr), An);
                    if (td < x) {
                        Qn = fmaf(u, u, Qn);
                        cn++;
                    }
                }
            }
            Cn = group_sum<G>(Cn);
            An = group_sum<G>(An);
            Qn = group_sum<G>(Qn);
            if (!done) {
                C = Cn;
                A = An;
                Q = Qn;
                cnt = cn;
            }
        }
    }
    if (valid && tl == 0) {
        yst[row] = make_float2(yh, yl);
        evals += nev;
    }

    // ---- new iterate at the final y, column sums ----
    const unsigned rh = row_hash(row, rc.seed);
    float* __restrict__ xo = Xout + R.b + tl;
#pragma unroll
    for (int k = 0; k < kSlots; k++) {
        if (rj[k] < 0) continue;
        const unsigned hb = entry_hash(rh, (unsigned)(k * G + tl));
        const float td = rtd[k];
        // x^{k+1} = [x^k - tau d]_+, stochastically rounded
        const float xn = td < rx[k] ? sr_add_rd(rx[k], -td, rand01_lo(hb)) : 0.0f;
        __stcs(xo + k * G, xn);
        const float d = xn - rx[k];
        dx2 = fmaf(d, d, dx2);
        rowm_acc(acc_s, acc_g, mk.hot, rj[k], xn, false);
    }
}

// ---------------------------------------------------------------------------
// rows longer than 32 * kSlots entries: one warp per row, the row streamed in
// chunks of 32 * kSlots entries and re-read (from L2) on every sweep.  The
// iteration and its stopping rule are those of rowm_core; what differs:
//  - the first activity check (after a frozen-model step) writes x^{k+1}, its
//    column sums and ||dx||^2 at the new y behind the check.  When the counts
//    are unchanged that y is final and no write sweep follows; otherwise the
//    column-sum contributions just written are subtracted again (exact: the
//    sums are fixed-point integers, and the same random bits give the same
//    rounded values), ||dx||^2 is restored, and the iteration continues
//    without further write-behind.
// Every lane of the warp calls this with the same row.
// ---------------------------------------------------------------------------
__device__ inline void rowm_long(const DevMarket& mk, const float* __restrict__ U, const float* __restrict__ Xin,
                                 float* __restrict__ Xout, const float2* __restrict__ pff,
                                 const float2* sp, unsigned long long* acc_s, unsigned long long* acc_g,
                                 float2* __restrict__ yst, const RowCtxM& rc, int row, float& dx2, int& capped,
                                 int& evals) {
    const int lane = threadIdx.x & 31;
    constexpr int span = 32 * kSlots;
    const long long b = mk.rp[row];
    const long long e = mk.rp[row + 1];
    const int dr = (int)(e - b);
    const int nch = (dr + span - 1) / span;
    const int* __restrict__ cjr = mk.cj + b + lane;      // this lane's entries: + c * span + k * 32
    const float* __restrict__ ur = U + b + lane;
    const float* __restrict__ xr = Xin + b + lane;
    float* __restrict__ xw = Xout + b + lane;
    const float tau = rc.tau;
    const unsigned rh = row_hash(row, rc.seed);

    float ru[kSlots], rx[kSlots], rph[kSlots], rpl[kSlots], rtd[kSlots];
    int rj[kSlots];
    auto load_chunk = [&](int c) {
        const int o = c * span;
#pragma unroll
        for (int k = 0; k < kSlots; k++) {
            if (o + k * 32 + lane < dr) {
                rj[k] = __ldg(cjr + o + k * 32);
                ru[k] = __ldg(ur + o + k * 32);
                rx[k] = xr[o + k * 32];
            } else {
                rj[k] = -1; ru[k] = 0.0f; rx[k] = 0.0f;
            }
        }
#pragma unroll
        for (int k = 0; k < kSlots; k++) {
            const bool ok = rj[k] >= 0;
            const float2 p = price_ff(pff, sp, mk.hot, ok ? rj[k] : 0);
            rph[k] = ok ? p.x : 0.0f;
            rpl[k] = ok ? p.y : 0.0f;
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
            const int pos = c * span + k * 32;
            const float td = rtd[k];
            const float xn = td < rx[k] ? sr_add_rd(rx[k], -td, rand01_lo(entry_hash(rh, (unsigned)(pos + lane)))) : 0.0f;
            if (!undo) {
                __stcs(xw + pos, xn);
                const float d = xn - rx[k];
                dx2 = fmaf(d, d, dx2);
            }
            rowm_acc(acc_s, acc_g, mk.hot, rj[k], xn, undo);
        }
    };

    // the row's arrays into L2 ahead of the chunk loads (one bulk prefetch per
    // array; 16-byte aligned window, the arrays carry slack after their end)
    if (lane < 3) {
        const char* base = lane == 0 ? (const char*)(mk.cj + b) : lane == 1 ? (const char*)(U + b) : (const char*)(Xin + b);
        const unsigned long long a0 = (unsigned long long)base & ~15ull;
        const unsigned long long a1 = ((unsigned long long)base + (unsigned long long)(e - b) * 4ull + 15ull) & ~15ull;
        asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(a0), "r"((unsigned)(a1 - a0)) : "memory");
    }
    const float2 wv = mk.wff[row];
    const ff W = ff_make(wv.x, wv.y);
    float2 y0 = yst[row];
    if (!(y0.x > 0.0f) || !isfinite(y0.x)) y0 = make_float2(1.0f, 0.0f);
    float yh = y0.x, yl = y0.y;

    // ---- first sweep: s0 and the evaluation at y_0 ----
    float s0h = 0.0f, s0l = 0.0f, C = 0.0f, A = 0.0f, Q = 0.0f;
    int cnt = 0;
    for (int c = 0; c < nch; c++) {
        load_chunk(c);
#pragma unroll
        for (int k = 0; k < kSlots; k++) {
            const float u = ru[k], x = rx[k];
            const ff pr = two_prod(u, x);
            const ff t = two_sum(s0h, pr.hi);
            s0h = t.hi;
            s0l += t.lo + pr.lo;
            const float td = td_at(k, yh, yl);
            const float cr = fminf(td, x);
            C = fmaf(u, cr, C);
            A = fmaf(u, fabsf(cr), A);
            if (td < x) {
                Q = fmaf(u, u, Q);
                cnt++;
            }
        }
    }
    ff s0 = group_sum<32>(ff_make(s0h, s0l));
    C = group_sum<32>(C);
    A = group_sum<32>(A);
    Q = group_sum<32>(Q);
    const float cnoise = 1.2e-7f * (sqrtf((float)(nch * kSlots)) + 3.0f);
    ff lo = ff_make(0.0f, 0.0f), hi = ff_make(INFINITY, 0.0f);
    int steps = 0, nev = 0;
    bool spec = true;        // the next activity check may write x^{k+1} behind it
    bool written = false;    // x^{k+1} written at the final y
    while (true) {
        nev++;
        const ff Y = ff_make(yh, yl);
        float sch;
        const float Gf = rowm_G(s0, C, Y, W, sch);
        const float aQ = tau * Q;
        const float floor = fmaf(cnoise * A, yh, fmaf(3e-14f * aQ * yh, yh, 2e-8f * W.hi));
        if (fabsf(Gf) <= floor || ++steps >= rc.cap || !(yh < kYMax)) {
            if (!(fabsf(Gf) <= floor) && lane == 0) capped++;
            break;
        }
        if (!(Gf <= 0.0f)) hi = Y; else lo = Y;
        float delta = 0.0f;
        const bool root = rowm_delta(Gf, sch, aQ, yh, delta);
        ff yn = root ? ff_add_f(Y, delta) : Y;
        bool check = cnoise * A * yh <= 2e-8f * W.hi && fabsf(delta) <= 0.0625f * yh;
        if (!root || !(ff_gt(yn, lo) && ff_gt(hi, yn))) {
            yn = isinf(hi.hi) ? ff_make(2.0f * yh, 0.0f) : ff_mul_f(ff_add(lo, hi), 0.5f);
            check = false;
        }
        if (yn.hi == yh && yn.lo == yl) break;               // no representable progress
        yh = yn.hi;
        yl = yn.lo;
        if (check) {
            // activity counts at the new y, writing x^{k+1} behind the check
            const bool wr = spec;
            spec = false;
            const float dsave = dx2;
            int cn = 0;
            for (int c = 0; c < nch; c++) {
                load_chunk(c);
#pragma unroll
                for (int k = 0; k < kSlots; k++) {
                    rtd[k] = td_at(k, yh, yl);
                    cn += rtd[k] < rx[k] ? 1 : 0;
                }
                if (wr) write_chunk(c, false);
            }
            const bool chg = __any_sync(0xffffffffu, cn != cnt);
            if (!chg) {
                written = wr;
                break;
            }
            if (wr) {
                for (int c = 0; c < nch; c++) {
                    load_chunk(c);
#pragma unroll
                    for (int k = 0; k < kSlots; k++) rtd[k] = td_at(k, yh, yl);
                    write_chunk(c, true);
                }
                dx2 = dsave;
            }
        }
        // evaluation at y
        C = A = Q = 0.0f;
        cnt = 0;
        for (int c = 0; c < nch; c++) {
            load_chunk(c);
#pragma unroll
            for (int k = 0; k < kSlots; k++) {
                const float u = ru[k];
                const float td = td_at(k, yh, yl);
                const float cr = fminf(td, rx[k]);
                C = fmaf(u, cr, C);
                A = fmaf(u, fabsf(cr), A);
                if (td < rx[k]) {
                    Q = fmaf(u, u, Q);
                    cnt++;
                }
            }
        }
        C = group_sum<32>(C);
        A = group_sum<32>(A);
        Q = group_sum<32>(Q);
    }
    if (lane == 0) {
        yst[row] = make_float2(yh, yl);
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

}  // namespace pdhcg
