// One PDHCG iteration on the GPU (Alg. 2), as three kernels:
//
//   price_kernel  (m threads)  commit the accepted candidate p^{k+1} and fold it
//                              into p-bar; new candidate
//                              p_j + sigma (2 c^k_j - c^{k-1}_j - 1)   (Eq. update:py)
//   prox_kernel   (persistent) per buyer: the exact row subproblem of Section 2.2,
//                              x_ij = [x^k_ij - tau p_j + tau w_i u_ij / s]_+ with
//                              s = u_i^T x_i (utility factor restored, Eq.
//                              KKT-system-6); folds x^k into x-bar; accumulates
//                              the column sums c_j = sum_i x_ij and ||dx||^2
//   dual_kernel   (m threads)  finishes c^{k+1}, the step-size quantities
//                              dp^T K dx and ||dp||^2, and in its last block
//                              applies the adaptive step rule (Section 5)
//
// Row solver.  phi(s) = s - sum_j u_j [a_j + c_j / s]_+ (a = x - tau p,
// c = tau w u) is increasing (Section 2.2).  Freezing the active set S at the
// current s turns the equation into s^2 - A s - C = 0 (A = sum_S u a,
// C = sum_S u c); its positive root is a lower bound of s* (the frozen sum is a
// minorant that touches at s), and iterating "active set -> root" climbs
// monotonically to s*, ending when the active set no longer changes; the
// result is then exact.  The rounds run in FP32 to find the active set; one
// final float-float round evaluates A, C, s* and the new x with about 48 bits,
// which the cancellation a_j + c_j/s (a_j can be much larger than x_j) needs.
// This replaces the paper's 32-section search (a GPU design for H100) by an
// exact finite procedure; the paper's searches remain in the oracle.
#include "common.cuh"

namespace pdhcg {

// ---------------------------------------------------------------------------
// positive root of s^2 - A s - C = 0 (C >= 0), cancellation free
// ---------------------------------------------------------------------------
__device__ __forceinline__ float root32(float A, float C) {
    float D = fmaf(A, A, 4.0f * C);
    float sq = sqrtf(fmaxf(D, 0.0f));
    return A >= 0.0f ? 0.5f * (A + sq) : (2.0f * C) / (sq - A);
}
__device__ __forceinline__ ff root_ff(ff A, ff C) {
    ff D = ff_add(ff_mul(A, A), ff_mul_f(C, 4.0f));
    ff sq = ff_sqrt(D);
    if (A.hi >= 0.0f) return ff_mul_f(ff_add(A, sq), 0.5f);
    return ff_div(ff_mul_f(C, 2.0f), ff_sub(sq, A));
}
__device__ __forceinline__ double root64(double A, double C) {
    double D = fma(A, A, 4.0 * C);
    double sq = sqrt(fmax(D, 0.0));
    return A >= 0.0 ? 0.5 * (A + sq) : (2.0 * C) / (sq - A);
}

// ---------------------------------------------------------------------------
// column-sum accumulation
// ---------------------------------------------------------------------------
__device__ __forceinline__ void acc_add_fixed(unsigned long long* s, unsigned long long* g, int hot, int j, float x) {
    if (x > 0.0f) {
        unsigned long long v = (unsigned long long)__float2ll_rn(x * kFixScaleF);
        if (j < hot) atomicAdd(&s[j], v);
        else atomicAdd(&g[j], v);
    }
}
__device__ __forceinline__ void acc_add_f64(unsigned long long* s, unsigned long long* g, int hot, int j, double x) {
    if (x > 0.0) {
        if (j < hot) atomicAdd((double*)&s[j], x);
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
};

// ---------------------------------------------------------------------------
// MIXED row solve: G lanes per row, row data either in registers (LONG=false,
// d <= G*kSlots) or streamed in chunks of 32*kSlots (LONG=true, G=32).
// Every lane of the warp calls this together; `valid` marks real rows.
// ---------------------------------------------------------------------------
template <int G, bool LONG>
__device__ void row_mixed(const DevMarket& mk, const float* __restrict__ U, const float* __restrict__ Xin,
                          float* __restrict__ Xout, float* __restrict__ Xb, const float2* __restrict__ pff,
                          unsigned long long* acc_s, unsigned long long* acc_g, double* __restrict__ t_out,
                          const RowCtx& rc, int row, bool valid, float& dx2, int& capped) {
    const int tl = (threadIdx.x & 31) & (G - 1);
    const long long b = valid ? mk.rp[row] : 0;
    const long long e = valid ? mk.rp[row + 1] : 0;
    const ff tau = ff_make(rc.tau_hi, rc.tau_lo);
    const double wi = valid ? mk.w[row] : 1.0;
    const ff tw = ff_mul(tau, ff_from_double(wi));
    const int span = G * kSlots;
    const int nch = LONG ? (int)((e - b + span - 1) / span) : 1;

    float ru[kSlots], rx[kSlots], rah[kSlots], ral[kSlots];
    int rj[kSlots];
    bool rin[kSlots];

    auto load_chunk = [&](int c) {
#pragma unroll
        for (int k = 0; k < kSlots; k++) {
            long long idx = b + (long long)c * span + k * G + tl;
            rin[k] = idx < e;
            if (rin[k]) {
                int j = __ldg(mk.cj + idx);
                float u = __ldg(U + idx);
                float x = Xin[idx];
                float2 p = __ldg(pff + j);
                ff a = ff_sub(ff_make(x, 0.0f), ff_mul(tau, ff_make(p.x, p.y)));
                rj[k] = j; ru[k] = u; rx[k] = x; rah[k] = a.hi; ral[k] = a.lo;
            } else {
                rj[k] = 0; ru[k] = 0.0f; rx[k] = 0.0f; rah[k] = 0.0f; ral[k] = 0.0f;
            }
        }
    };

    // ---- starting point s0 = u^T x^k (Alg. 3's trial value) ----
    float s0 = 0.0f, qall = 0.0f;
    for (int c = 0; c < nch; c++) {
        if (LONG || c == 0) load_chunk(c);
#pragma unroll
        for (int k = 0; k < kSlots; k++) { s0 = fmaf(ru[k], rx[k], s0); qall = fmaf(ru[k], ru[k], qall); }
    }
    s0 = group_sum<G>(s0);
    qall = group_sum<G>(qall);
    if (!(s0 > 0.0f)) s0 = sqrtf(tw.hi * qall);   // all entries active: s^2 ~ C
    if (!(s0 > 0.0f)) s0 = 1.0f;

    // ---- FP32 active-set rounds ----
    float s = s0, s_last = -1.0f;
    bool gdone = !valid;
    int rounds = 0;
    while (__any_sync(0xffffffffu, !gdone)) {
        const float R = tw.hi / s;
        float A = 0.0f, Q = 0.0f;
        for (int c = 0; c < nch; c++) {
            if (LONG) load_chunk(c);
#pragma unroll
            for (int k = 0; k < kSlots; k++) {
                if (rin[k] && fmaf(ru[k], R, rah[k]) > 0.0f) {
                    A = fmaf(ru[k], rah[k], A);
                    Q = fmaf(ru[k], ru[k], Q);
                }
            }
        }
        A = group_sum<G>(A);
        Q = group_sum<G>(Q);
        if (!gdone) {
            float sn = root32(A, tw.hi * Q);
            if (sn == s_last) {
                gdone = true;                    // same root twice: the set is stable
            } else {
                s = (rounds == 0) ? sn : fmaxf(s, sn);
                s_last = sn;
                if (++rounds >= rc.cap) { gdone = true; if (tl == 0 && valid) capped++; }
            }
        }
    }

    // ---- float-float round(s): exact root for the active set, re-checked ----
    float R32 = tw.hi / s;
    ff sst = ff_make(s, 0.0f), Rff = ff_make(R32, 0.0f);
    bool pdone = !valid;
    for (int att = 0; att < 3; att++) {
        ff A = ff_make(0.0f, 0.0f), Q = ff_make(0.0f, 0.0f);
        for (int c = 0; c < nch; c++) {
            if (LONG) load_chunk(c);
#pragma unroll
            for (int k = 0; k < kSlots; k++) {
                bool act = rin[k] && (att == 0 ? fmaf(ru[k], R32, rah[k]) > 0.0f
                                               : ff_pos(ff_add(ff_make(rah[k], ral[k]), ff_mul_f(Rff, ru[k]))));
                if (act) {
                    A = ff_add(A, ff_mul_f(ff_make(rah[k], ral[k]), ru[k]));
                    Q = ff_add(Q, two_prod(ru[k], ru[k]));
                }
            }
        }
        A = group_sum<G>(A);
        Q = group_sum<G>(Q);
        ff sn = root_ff(A, ff_mul(tw, Q));
        ff Rn = ff_div(tw, sn);
        // does the active set at the new root agree with the one used?
        bool changed = false;
        for (int c = 0; c < nch; c++) {
            if (LONG) load_chunk(c);
#pragma unroll
            for (int k = 0; k < kSlots; k++) {
                if (!rin[k]) continue;
                bool was = att == 0 ? fmaf(ru[k], R32, rah[k]) > 0.0f
                                    : ff_pos(ff_add(ff_make(rah[k], ral[k]), ff_mul_f(Rff, ru[k])));
                bool now = ff_pos(ff_add(ff_make(rah[k], ral[k]), ff_mul_f(Rn, ru[k])));
                changed |= (was != now);
            }
        }
        bool any_changed = group_any<G>(changed);
        if (!pdone) { sst = sn; Rff = Rn; }
        if (!any_changed) pdone = true;
        if (!__any_sync(0xffffffffu, !pdone)) break;
    }

    // ---- new iterate, average fold, column sums ----
    const float fw = rc.fold_w;
    for (int c = 0; c < nch; c++) {
        if (LONG) load_chunk(c);
#pragma unroll
        for (int k = 0; k < kSlots; k++) {
            if (!rin[k]) continue;
            long long idx = b + (long long)c * span + k * G + tl;
            ff v = ff_add(ff_make(rah[k], ral[k]), ff_mul_f(Rff, ru[k]));
            float xn = v.hi > 0.0f ? v.hi : 0.0f;
            Xout[idx] = xn;
            float d = xn - rx[k];
            dx2 = fmaf(d, d, dx2);
            if (rc.fold) {
                float xb = (fw == 1.0f) ? rx[k] : fmaf(fw, rx[k] - Xb[idx], Xb[idx]);
                Xb[idx] = xb;
            }
            acc_add_fixed(acc_s, acc_g, mk.hot, rj[k], xn);
        }
    }
    if (valid && tl == 0) t_out[row] = ff_to_double(sst);
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
                rj[k] = j; ru[k] = u; rx[k] = x; ra[k] = x - rc.tau * __ldg(pc + j);
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

// ---------------------------------------------------------------------------
// the persistent row kernel
// ---------------------------------------------------------------------------
template <bool MIXED>
__global__ void __launch_bounds__(kThreads) prox_kernel(DevMarket mk, const void* Xin_fixed, void* Xout_fixed,
                                                         IterBufs bf, Ctl* ctl, int fixed) {
    extern __shared__ unsigned long long acc_s[];
    if (!ctl->active) return;
    RowCtx rc;
    rc.tau = ctl->tau;
    rc.tau_hi = (float)rc.tau;
    rc.tau_lo = (float)(rc.tau - (double)rc.tau_hi);
    rc.fold = !fixed && ctl->fold_pending;
    rc.fold_wd = ctl->fold_wgt;
    rc.fold_w = (float)rc.fold_wd;
    rc.cap = ctl->row_cap;
    const int cur = ctl->cur;
    const void* Xin = fixed ? Xin_fixed : (cur ? bf.X[1] : bf.X[0]);
    void* Xout = fixed ? Xout_fixed : (cur ? bf.X[0] : bf.X[1]);

    for (int j = threadIdx.x; j < mk.hot; j += blockDim.x) acc_s[j] = 0ull;
    __syncthreads();

    const int lane = threadIdx.x & 31;
    const long long gw = (long long)blockIdx.x * kWarps + (threadIdx.x >> 5);
    const long long tw_ = (long long)gridDim.x * kWarps;
    float dxf = 0.0f;
    double dxd = 0.0;
    int capped = 0;

    for (int bi = 0; bi < mk.nb; bi++) {
        const Bucket bk = mk.buckets[bi];
        const int g = bk.g;
        const int rpw = 32 / g;
        const long long units = (bk.count + rpw - 1) / rpw;
        for (long long u = gw; u < units; u += tw_) {
            long long slot = u * rpw + lane / g;
            bool valid = slot < bk.count;
            int row = valid ? mk.row_order[bk.first + slot] : 0;
            if (MIXED) {
                const float* U = (const float*)mk.uv;
                float* Xo = (float*)Xout;
                const float* Xi = (const float*)Xin;
                float* Xb = (float*)bf.Xb;
                if (bk.chunks) row_mixed<32, true>(mk, U, Xi, Xo, Xb, bf.pff, acc_s, bf.acc, bf.t, rc, row, valid, dxf, capped);
                else if (g == 4) row_mixed<4, false>(mk, U, Xi, Xo, Xb, bf.pff, acc_s, bf.acc, bf.t, rc, row, valid, dxf, capped);
                else if (g == 8) row_mixed<8, false>(mk, U, Xi, Xo, Xb, bf.pff, acc_s, bf.acc, bf.t, rc, row, valid, dxf, capped);
                else if (g == 16) row_mixed<16, false>(mk, U, Xi, Xo, Xb, bf.pff, acc_s, bf.acc, bf.t, rc, row, valid, dxf, capped);
                else row_mixed<32, false>(mk, U, Xi, Xo, Xb, bf.pff, acc_s, bf.acc, bf.t, rc, row, valid, dxf, capped);
            } else {
                const double* U = (const double*)mk.uv;
                double* Xo = (double*)Xout;
                const double* Xi = (const double*)Xin;
                double* Xb = (double*)bf.Xb;
                if (bk.chunks) row_fp64<32, true>(mk, U, Xi, Xo, Xb, bf.pc, acc_s, bf.acc, bf.t, rc, row, valid, dxd, capped);
                else if (g == 4) row_fp64<4, false>(mk, U, Xi, Xo, Xb, bf.pc, acc_s, bf.acc, bf.t, rc, row, valid, dxd, capped);
                else if (g == 8) row_fp64<8, false>(mk, U, Xi, Xo, Xb, bf.pc, acc_s, bf.acc, bf.t, rc, row, valid, dxd, capped);
                else if (g == 16) row_fp64<16, false>(mk, U, Xi, Xo, Xb, bf.pc, acc_s, bf.acc, bf.t, rc, row, valid, dxd, capped);
                else row_fp64<32, false>(mk, U, Xi, Xo, Xb, bf.pc, acc_s, bf.acc, bf.t, rc, row, valid, dxd, capped);
            }
        }
    }

    // ---- block epilogue: ||dx||^2 partial, capped rows, flush hot column sums ----
    double v = MIXED ? (double)dxf : dxd;
    v = warp_sum_d(v);
    __shared__ double red[kWarps];
    __shared__ int capred;
    if (threadIdx.x == 0) capred = 0;
    __syncthreads();
    if (lane == 0) red[threadIdx.x >> 5] = v;
    if (capped) atomicAdd(&capred, capped);
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < kWarps; w++) t += red[w];
        bf.part[blockIdx.x] = t;
        if (capred) atomicAdd((unsigned long long*)&ctl->capped, (unsigned long long)capred);
    }
    for (int j = threadIdx.x; j < mk.hot; j += blockDim.x) {
        unsigned long long a = acc_s[j];
        if (a) {
            if (MIXED) atomicAdd(&bf.acc[j], a);
            else atomicAdd((double*)&bf.acc[j], __longlong_as_double((long long)a));
        }
    }
}

// ---------------------------------------------------------------------------
// price kernel: commit + fold p, new candidate (Eq. update:py)
// ---------------------------------------------------------------------------
template <bool MIXED>
__global__ void price_kernel(DevMarket mk, IterBufs bf, Ctl* ctl) {
    if (!ctl->active) return;
    const bool pending = ctl->fold_pending;
    const double wgt = ctl->fold_wgt;
    const double sigma = ctl->sigma;
    const int ick = ctl->ck, ickm1 = ctl->ckm1;
    const double* ck = ick == 0 ? bf.C[0] : (ick == 1 ? bf.C[1] : bf.C[2]);
    const double* ckm1 = ickm1 == 0 ? bf.C[0] : (ickm1 == 1 ? bf.C[1] : bf.C[2]);
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < mk.m; j += gridDim.x * blockDim.x) {
        double p = bf.p[j];
        if (pending) {
            p = bf.pc[j];
            bf.p[j] = p;
            double pb = bf.pbar[j];
            bf.pbar[j] = (wgt == 1.0) ? p : fma(wgt, p - pb, pb);
        }
        double pc = fma(sigma, 2.0 * ck[j] - ckm1[j] - 1.0, p);
        bf.pc[j] = pc;
        if (MIXED) {
            float h = (float)pc;
            bf.pff[j] = make_float2(h, (float)(pc - (double)h));
        }
    }
}

// ---------------------------------------------------------------------------
// dual kernel: column sums of x^{k+1}, step-size quantities, step control
// ---------------------------------------------------------------------------
template <bool MIXED>
__global__ void dual_kernel(DevMarket mk, IterBufs bf, Ctl* ctl, int nprox) {
    if (!ctl->active) return;
    const int icn = ctl->cnew, ick = ctl->ck;
    double* cn = icn == 0 ? bf.C[0] : (icn == 1 ? bf.C[1] : bf.C[2]);
    const double* ck = ick == 0 ? bf.C[0] : (ick == 1 ? bf.C[1] : bf.C[2]);
    double s1 = 0.0, s2 = 0.0;
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < mk.m; j += gridDim.x * blockDim.x) {
        unsigned long long a = bf.acc[j];
        bf.acc[j] = 0ull;
        double c = MIXED ? (double)(long long)a * kFixInv : __longlong_as_double((long long)a);
        cn[j] = c;
        double dp = bf.pc[j] - bf.p[j];
        s1 = fma(dp, c - ck[j], s1);
        s2 = fma(dp, dp, s2);
    }
    s1 = warp_sum_d(s1);
    s2 = warp_sum_d(s2);
    __shared__ double r1[32], r2[32];
    __shared__ bool last;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) { r1[wid] = s1; r2[wid] = s2; }
    __syncthreads();
    if (threadIdx.x == 0) {
        double a1 = 0.0, a2 = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); w++) { a1 += r1[w]; a2 += r2[w]; }
        bf.part2[2 * blockIdx.x] = a1;
        bf.part2[2 * blockIdx.x + 1] = a2;
        __threadfence();
        unsigned int t = atomicAdd(&ctl->ticket, 1u);
        last = (t == gridDim.x - 1);
    }
    __syncthreads();
    if (!last || threadIdx.x != 0) return;
    __threadfence();
    // ---- last block: adaptive step rule (Section 5, PDLP form) ----
    double dx2 = 0.0, inter = 0.0, dp2 = 0.0;
    for (int i = 0; i < nprox; i++) dx2 += ((volatile double*)bf.part)[i];
    for (int i = 0; i < (int)gridDim.x; i++) {
        inter += ((volatile double*)bf.part2)[2 * i];
        dp2 += ((volatile double*)bf.part2)[2 * i + 1];
    }
    inter = fabs(inter);
    ctl->ticket = 0u;
    const double om = ctl->omega, eta = ctl->eta;
    ctl->passes += 1;
    if (!isfinite(dx2) || !isfinite(dp2) || !isfinite(inter)) {
        ctl->nan_flag = 1;
        ctl->active = 0;
        return;
    }
    const double movement = om * dx2 + dp2 / om;
    const double eta_max = inter > 0.0 ? movement / (2.0 * inter) : INFINITY;
    const double k1 = (double)(ctl->iters + 1);
    const double grow = (1.0 + pow(k1, -0.6)) * eta;
    double eta_next = isinf(eta_max) ? grow : fmin((1.0 - pow(k1, -0.3)) * eta_max, grow);
    eta_next = fmin(fmax(eta_next, ctl->eta_min), ctl->eta_max_abs);
    const bool accept = (eta <= eta_max) || (eta <= ctl->eta_min * (1.0 + 1e-12));
    if (accept) {
        ctl->iters += 1;
        ctl->chunk_acc += 1;
        ctl->sum_eta += eta;
        ctl->fold_wgt = eta / ctl->sum_eta;
        ctl->eta_used = eta;
        ctl->fold_pending = 1;
        ctl->accepted = 1;
        ctl->cur = 1 - ctl->cur;
        const int old_ckm1 = ctl->ckm1;
        ctl->ckm1 = ctl->ck;
        ctl->ck = ctl->cnew;
        ctl->cnew = old_ckm1;
        if (ctl->chunk_acc >= ctl->chunk_quota) ctl->active = 0;
    } else {
        ctl->fold_pending = 0;
        ctl->accepted = 0;
    }
    ctl->eta = eta_next;
    ctl->tau = eta_next / om;
    ctl->sigma = eta_next * om;
}

// ---------------------------------------------------------------------------
// flush: commit + fold the last accepted step into the averages (chunk end)
// ---------------------------------------------------------------------------
template <typename V>
__global__ void flush_x_kernel(long long nnz, IterBufs bf, Ctl* ctl) {
    if (!ctl->fold_pending) return;
    const V* x = (const V*)(ctl->cur ? bf.X[1] : bf.X[0]);
    V* xb = (V*)bf.Xb;
    const double wgt = ctl->fold_wgt;
    const V wv = (V)wgt;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < nnz; i += (long long)gridDim.x * blockDim.x) {
        V xv = x[i];
        xb[i] = (wgt == 1.0) ? xv : xb[i] + wv * (xv - xb[i]);
    }
}
__global__ void flush_p_kernel(int m, IterBufs bf, Ctl* ctl) {
    if (!ctl->fold_pending) return;
    const double wgt = ctl->fold_wgt;
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < m; j += gridDim.x * blockDim.x) {
        double p = bf.pc[j];
        bf.p[j] = p;
        double pb = bf.pbar[j];
        bf.pbar[j] = (wgt == 1.0) ? p : fma(wgt, p - pb, pb);
    }
}
__global__ void flush_done_kernel(Ctl* ctl) { ctl->fold_pending = 0; }

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
static size_t prox_smem(const DevMarket& mk) { return (size_t)mk.hot * sizeof(unsigned long long); }

static void set_smem_attr() {
    static bool done = false;
    if (done) return;
    done = true;
    cudaFuncSetAttribute(prox_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    cudaFuncSetAttribute(prox_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
}

static int sm_count() {
    static int sm = 0;
    if (!sm) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sm, cudaDevAttrMultiProcessorCount, dev);
    }
    return sm;
}

// Persistent grid: every SM holds as many blocks as registers and shared
// memory allow (PDHCG_PROX_BLOCKS_PER_SM caps it for tuning).
int prox_blocks(bool mixed, int hot) {
    set_smem_attr();
    int per = 0;
    size_t smem = (size_t)hot * sizeof(unsigned long long);
    if (mixed) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, prox_kernel<true>, kThreads, smem);
    else cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, prox_kernel<false>, kThreads, smem);
    if (per < 1) per = 1;
    const char* env = getenv("PDHCG_PROX_BLOCKS_PER_SM");
    if (env && atoi(env) > 0 && atoi(env) < per) per = atoi(env);
    return sm_count() * per;
}
int max_prox_blocks() { return sm_count() * 8; }

static int vec_blocks(int m) {
    int b = (m + 255) / 256;
    return b < 1 ? 1 : (b > 1024 ? 1024 : b);
}

void launch_price(bool mixed, const DevMarket& mk, const IterBufs& b, Ctl* ctl, cudaStream_t s) {
    if (mixed) price_kernel<true><<<vec_blocks(mk.m), 256, 0, s>>>(mk, b, ctl);
    else price_kernel<false><<<vec_blocks(mk.m), 256, 0, s>>>(mk, b, ctl);
}
void launch_prox(bool mixed, const DevMarket& mk, const IterBufs& b, Ctl* ctl, cudaStream_t s) {
    set_smem_attr();
    if (mixed) prox_kernel<true><<<mk.nprox, kThreads, prox_smem(mk), s>>>(mk, nullptr, nullptr, b, ctl, 0);
    else prox_kernel<false><<<mk.nprox, kThreads, prox_smem(mk), s>>>(mk, nullptr, nullptr, b, ctl, 0);
}
void launch_dual(bool mixed, const DevMarket& mk, const IterBufs& b, Ctl* ctl, cudaStream_t s) {
    int nb = vec_blocks(mk.m);
    if (nb > 256) nb = 256;
    if (mixed) dual_kernel<true><<<nb, 256, 0, s>>>(mk, b, ctl, mk.nprox);
    else dual_kernel<false><<<nb, 256, 0, s>>>(mk, b, ctl, mk.nprox);
}
void launch_flush(bool mixed, const DevMarket& mk, const IterBufs& b, Ctl* ctl, cudaStream_t s) {
    int nbx = (int)((mk.nnz + 255) / 256);
    if (nbx > 4096) nbx = 4096;
    if (nbx < 1) nbx = 1;
    if (mixed) flush_x_kernel<float><<<nbx, 256, 0, s>>>(mk.nnz, b, ctl);
    else flush_x_kernel<double><<<nbx, 256, 0, s>>>(mk.nnz, b, ctl);
    flush_p_kernel<<<vec_blocks(mk.m), 256, 0, s>>>(mk.m, b, ctl);
    flush_done_kernel<<<1, 1, 0, s>>>(ctl);
}

// standalone pass: prices given, no step control, column sums returned
__global__ void p_to_ff_kernel(int m, const double* p, float2* pff, double* pc) {
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < m; j += gridDim.x * blockDim.x) {
        double v = p[j];
        float h = (float)v;
        pff[j] = make_float2(h, (float)(v - (double)h));
        pc[j] = v;
    }
}
__global__ void cols_out_kernel(int m, bool mixed, unsigned long long* acc, double* c_out) {
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < m; j += gridDim.x * blockDim.x) {
        unsigned long long a = acc[j];
        acc[j] = 0ull;
        double c = mixed ? (double)(long long)a * kFixInv : __longlong_as_double((long long)a);
        if (c_out) c_out[j] = c;
    }
}
__global__ void ctl_fixed_kernel(Ctl* ctl, double tau, int cap) {
    ctl->active = 1;
    ctl->tau = tau;
    ctl->fold_pending = 0;
    ctl->cur = 0;
    ctl->row_cap = cap;
    ctl->capped = 0;
}

void launch_prox_fixed(bool mixed, const DevMarket& mk, const void* x_in, void* x_out, const double* p,
                       double tau, unsigned long long* acc, double* t_out, double* c_out,
                       double* part, Ctl* ctl, cudaStream_t s) {
    set_smem_attr();
    IterBufs b = {};
    b.acc = acc;
    b.t = t_out;
    b.part = part;
    // scratch for the converted prices lives after the m accumulators
    b.pff = (float2*)(acc + mk.m);
    b.pc = (double*)(acc + 2 * (size_t)mk.m);
    p_to_ff_kernel<<<vec_blocks(mk.m), 256, 0, s>>>(mk.m, p, b.pff, b.pc);
    ctl_fixed_kernel<<<1, 1, 0, s>>>(ctl, tau, 64);
    if (mixed) prox_kernel<true><<<mk.nprox, kThreads, prox_smem(mk), s>>>(mk, x_in, x_out, b, ctl, 1);
    else prox_kernel<false><<<mk.nprox, kThreads, prox_smem(mk), s>>>(mk, x_in, x_out, b, ctl, 1);
    cols_out_kernel<<<vec_blocks(mk.m), 256, 0, s>>>(mk.m, mixed, acc, c_out);
}

}  // namespace pdhcg
