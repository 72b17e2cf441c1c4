// Batched Fisher markets: B independent markets of uneven size solved by one
// launch of a persistent kernel.
//
// Each block takes the next market from a work queue (markets ordered by
// decreasing nnz, an LPT schedule) and runs the whole of Alg. 2 on it:
//   price phase   goods of the market        (shared memory)
//   row phase     the row subproblems of Section 2.2 (rowsolve.cuh), G lanes per
//                 row with G chosen per market by the autotuner; column sums
//                 accumulate in shared memory (every good of the market is "hot")
//   dual phase    column sums, step-size quantities and, in thread 0, the
//                 adaptive step rule of Section 5
// and every kkt_check_every accepted iterations the relative KKT error of the
// current point and of the average, the adaptive restart, the primal-weight
// update and the termination test, all on the device with per-market state.
// Block barriers replace the kernel boundaries of the single-market path, so
// there is no host round trip and no grid-wide wait.  Every loop is bounded:
// max_iter per market, the row-solve round cap, and the time limit (read from
// the global timer).  Markets may have at most kBatchMaxGoods goods (their
// per-good vectors live in shared memory).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <type_traits>
#include <vector>

#include "common.cuh"
#include "prep.cuh"
#include "rowsolve.cuh"
#include "solver.cuh"

namespace pdhcg {

constexpr int kBatchMaxGoods = 4096;

struct MState {
    double eta, omega, omega0, eta0, eta_min, eta_maxa, sum_eta, fold_wgt;
    double kkt_rs, kkt_prev, sum_w, normK, x0n2;
    double r_p, r_d, r_g, kkt;
    long long iters, passes, iters_rs, capped, chunk_acc;
    int restarts, cur, ck, ckm1, cnew, fold_pending, status, use_avg, maxdeg, g, err;
    int pad;
};

struct BatchArgs {
    int B;
    const long long* row_off;
    const long long* good_off;
    const long long* nnz_off;
    const long long* rp;
    const int* col;
    const void* val;
    int val_f32;
    const double* w;
    void* uv;
    double* rowmax;
    void* X[2];
    void* Xb;
    void* Xr;
    double *p, *pc, *pbar, *prs, *C[3], *cc, *ca;
    double *tc, *ta;
    int* deg;
    MState* st;
    const int* order;
    unsigned int* queue;
    const int* gsel;
    double tol, eta_lo, eta_hi, eta0_scale, beta_suff, beta_nec, beta_art, theta, omega_range;
    long long max_iter;
    int check_every, omega_reset_every, row_cap;
    double time_limit_ns;
    int smem_goods;
};

__device__ __forceinline__ unsigned long long gtimer() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// max of positive doubles held as bit patterns, by compare-and-swap (64-bit
// atomicMax is not available on shared memory); each retry sees a larger value,
// so the loop ends after at most as many rounds as there are contenders.
__device__ __forceinline__ void cas_max_pos(unsigned long long* a, double v) {
    const unsigned long long nv = dbits(v);
    unsigned long long old = *((volatile unsigned long long*)a);
    while (nv > old) {
        const unsigned long long prev = shared_cas_b64(a, old, nv);
        if (prev == old) break;
        old = prev;
    }
}

// block-wide reductions (all threads call; result valid in every thread)
__device__ double block_sum(double v, double* scratch) {
    v = warp_sum_d(v);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) scratch[wid] = v;
    __syncthreads();
    double t = 0.0;
    for (int i = 0; i < (int)(blockDim.x >> 5); i++) t += scratch[i];
    __syncthreads();
    return t;
}
__device__ double block_max(double v, double* scratch) {
    v = warp_max_d(v);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) scratch[wid] = v;
    __syncthreads();
    double t = -INFINITY;
    for (int i = 0; i < (int)(blockDim.x >> 5); i++) t = fmax(t, scratch[i]);
    __syncthreads();
    return t;
}

// ---------------------------------------------------------------------------
// preprocessing: one block per market (validation, degrees, scaling, x^0)
// ---------------------------------------------------------------------------
template <typename V>
__global__ void batch_prep_kernel(BatchArgs a) {
    extern __shared__ int sdeg[];
    __shared__ double scratch[32];
    __shared__ int err;
    const int b = blockIdx.x;
    if (b >= a.B) return;
    const long long r0 = a.row_off[b], r1 = a.row_off[b + 1];
    const long long g0 = a.good_off[b];
    const int m = (int)(a.good_off[b + 1] - g0);
    if (threadIdx.x == 0) err = 0;
    if (m <= 0 || m > kBatchMaxGoods || r1 <= r0) {
        if (threadIdx.x == 0) { a.st[b].status = PDHCG_ERR_INVALID; a.st[b].err = ERR_ROWPTR; }
        return;
    }
    for (int j = threadIdx.x; j < m; j += blockDim.x) sdeg[j] = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    unsigned int e = 0;
    if (threadIdx.x == 0 && (a.rp[r0] != a.nnz_off[b] || a.rp[r1] != a.nnz_off[b + 1])) e |= ERR_ROWPTR;
    double sw = 0.0;
    for (long long i = r0 + wid; i < r1; i += nw) {
        const long long q0 = a.rp[i], q1 = a.rp[i + 1];
        if (lane == 0) {
            double wi = a.w[i];
            if (!(wi > 0.0) || !isfinite(wi)) e |= ERR_BUDGET;
            sw += wi;
        }
        if (q1 <= q0) { e |= ERR_EMPTY_ROW; continue; }
        for (long long q = q0 + lane; q < q1; q += 32) {
            const int j = a.col[q];
            if (j < 0 || j >= m) { e |= ERR_COL_RANGE; continue; }
            if (q > q0 && a.col[q - 1] >= j) e |= ERR_COL_ORDER;
            const double u = a.val_f32 ? (double)((const float*)a.val)[q] : ((const double*)a.val)[q];
            if (!(u > 0.0) || !isfinite(u)) e |= ERR_UTIL;
            shared_add_s32(&sdeg[j], 1);
        }
    }
    if (e) shared_or_b32((unsigned int*)&err, e);
    __syncthreads();
    double inv = 0.0, mx = 0.0;
    for (int j = threadIdx.x; j < m; j += blockDim.x) {
        const int d = sdeg[j];
        a.deg[g0 + j] = d;
        if (d == 0) shared_or_b32((unsigned int*)&err, ERR_EMPTY_COL);
        else inv += 1.0 / (double)d;
        mx = fmax(mx, (double)d);
    }
    const double x0n2 = block_sum(inv, scratch);
    const double maxdeg = block_max(mx, scratch);
    const double sumw = block_sum(sw, scratch);
    if (err) {
        if (threadIdx.x == 0) { a.st[b].status = PDHCG_ERR_INVALID; a.st[b].err = err; }
        return;
    }
    V* uv = (V*)a.uv;
    V* x0 = (V*)a.X[0];
    int rowdeg_max = 0;
    for (long long i = r0 + wid; i < r1; i += nw) {
        const long long q0 = a.rp[i], q1 = a.rp[i + 1];
        rowdeg_max = max(rowdeg_max, (int)(q1 - q0));
        double rmx = 0.0;
        for (long long q = q0 + lane; q < q1; q += 32)
            rmx = fmax(rmx, a.val_f32 ? (double)((const float*)a.val)[q] : ((const double*)a.val)[q]);
        rmx = row_scale<V>(warp_max_d(rmx));
        if (lane == 0) a.rowmax[i] = rmx;
        for (long long q = q0 + lane; q < q1; q += 32) {
            const double u = a.val_f32 ? (double)((const float*)a.val)[q] : ((const double*)a.val)[q];
            uv[q] = (V)(u / rmx);
            x0[q] = (V)(1.0 / (double)sdeg[a.col[q]]);
        }
    }
    const double rdm = block_max((double)rowdeg_max, scratch);
    if (threadIdx.x == 0) {
        MState& S = a.st[b];
        S.status = PDHCG_ERR_NOT_CONVERGED;
        S.err = 0;
        S.sum_w = sumw;
        S.normK = sqrt(maxdeg);
        S.x0n2 = x0n2;
        S.maxdeg = (int)rdm;
    }
}

// ---------------------------------------------------------------------------
// KKT of one market (Section 5), computed by the whole block
// ---------------------------------------------------------------------------
template <bool MIXED>
__device__ void kkt_market(const BatchArgs& a, long long r0, long long r1, long long g0, int m, const void* Xv,
                           const double* p, unsigned long long* acc, unsigned long long* Mx, double* cout,
                           double* tout, double* scratch, double out[4]) {
    for (int j = threadIdx.x; j < m; j += blockDim.x) { acc[j] = 0ull; Mx[j] = 0ull; }
    __syncthreads();
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    double mxx = 0.0, mg = 0.0, mxg = 0.0, my = 0.0;
    for (long long i = r0 + wid; i < r1; i += nw) {
        const long long q0 = a.rp[i], q1 = a.rp[i + 1];
        double t = 0.0, um = 0.0;
        for (long long q = q0 + lane; q < q1; q += 32) {
            double u = MIXED ? (double)((const float*)a.uv)[q] : ((const double*)a.uv)[q];
            double x = MIXED ? (double)((const float*)Xv)[q] : ((const double*)Xv)[q];
            t = fma(u, x, t);
            um = fmax(um, u);
        }
        t = warp_sum_d(t);
        um = warp_max_d(um);
        const double y = a.w[i] / t;
        if (lane == 0) tout[i] = t;
        my = fmax(my, y * um);         // y of the max-scaled row
        for (long long q = q0 + lane; q < q1; q += 32) {
            const int j = a.col[q];
            double u = MIXED ? (double)((const float*)a.uv)[q] : ((const double*)a.uv)[q];
            double x = MIXED ? (double)((const float*)Xv)[q] : ((const double*)Xv)[q];
            const double uy = u * y;
            const double g = fmax(p[j] - uy, 0.0);
            mxx = fmax(mxx, x);
            mg = fmax(mg, g);
            mxg = fmax(mxg, x * g);
            cas_max_pos(&Mx[j], uy);
            if (x > 0.0) {
                if (MIXED) shared_add_u64(&acc[j], (unsigned long long)__double2ll_rn(x * kFixScale));
                else shared_add_f64(&acc[j], x);
            }
        }
    }
    mxx = block_max(mxx, scratch);
    mg = block_max(mg, scratch);
    mxg = block_max(mxg, scratch);
    my = block_max(my, scratch);
    double np = 0.0, mc = 0.0, nd = 0.0, dd = -INFINITY;
    for (int j = threadIdx.x; j < m; j += blockDim.x) {
        unsigned long long v = acc[j];
        const double c = MIXED ? (double)(long long)v * kFixInv : __longlong_as_double((long long)v);
        acc[j] = 0ull;
        cout[j] = c;
        const double Mj = __longlong_as_double((long long)Mx[j]);
        np = fmax(np, fabs(c - 1.0));
        mc = fmax(mc, c);
        const double d = p[j] - Mj;
        nd = fmax(nd, fmax(-d, 0.0));
        dd = fmax(dd, d);
    }
    np = block_max(np, scratch);
    mc = block_max(mc, scratch);
    nd = block_max(nd, scratch);
    dd = block_max(dd, scratch);
    out[0] = np / (1.0 + fmax(mc, 1.0));
    out[1] = nd / (1.0 + fmax(my, dd));
    out[2] = mxg / (1.0 + fmax(mxx, mg));
    out[3] = fmax(out[0], fmax(out[1], out[2]));
    if (!(out[3] == out[3])) out[3] = INFINITY;
}

// squared distance of a block-strided range, with copy r <- a
template <typename V>
__device__ double dist_copy_block(const V* a, V* r, long long n0, long long n1, double* scratch) {
    double s = 0.0;
    for (long long i = n0 + threadIdx.x; i < n1; i += blockDim.x) {
        const double d = (double)a[i] - (double)r[i];
        s = fma(d, d, s);
        r[i] = a[i];
    }
    return block_sum(s, scratch);
}

template <bool MIXED, int G, bool LONG>
__device__ void row_phase(const BatchArgs& a, const DevMarket& dm, long long r0, long long r1, const void* Xin,
                          void* Xout, const RowCtx& rc, const float2* pff, const double* pcs,
                          unsigned long long* acc, double& dx2, int& capped) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    constexpr int rpw = 32 / G;
    const long long rows = r1 - r0;
    const long long units = (rows + rpw - 1) / rpw;
    float dxf = 0.0f;
    double dxd = 0.0;
    int evals = 0;
    for (long long u = wid; u < units; u += nw) {
        const long long slot = u * rpw + lane / G;
        const bool valid = slot < rows;
        const int row = valid ? (int)(r0 + slot) : (int)r0;
        if (MIXED)
            row_mixed<G, LONG>(dm, (const float*)a.uv, (const float*)Xin, (float*)Xout, (float*)a.Xb, pff, acc, acc,
                               a.tc, rc, row, valid, dxf, capped, evals);
        else
            row_fp64<G, LONG>(dm, (const double*)a.uv, (const double*)Xin, (double*)Xout, (double*)a.Xb, pcs, acc,
                              acc, a.tc, rc, row, valid, dxd, capped);
    }
    dx2 += MIXED ? (double)dxf : dxd;
}

template <bool MIXED>
__global__ void __launch_bounds__(kThreads, 2) batch_solve_kernel(BatchArgs a) {
    extern __shared__ unsigned long long smem[];
    const int M = a.smem_goods;
    unsigned long long* acc = smem;
    unsigned long long* Mx = smem + M;
    float2* pff = (float2*)(smem + 2 * M);
    double* pcs = (double*)(smem + 2 * M);
    __shared__ double scratch[32];
    __shared__ MState S;
    __shared__ int sh_b;
    __shared__ int go_on, do_restart;
    typedef typename std::conditional<MIXED, float, double>::type V;
    const unsigned long long t_start = gtimer();

    while (true) {
        if (threadIdx.x == 0) sh_b = (int)atomicAdd(a.queue, 1u);
        __syncthreads();
        if (sh_b >= a.B) break;
        const int b = a.order[sh_b];
        if (threadIdx.x == 0) S = a.st[b];
        __syncthreads();
        if (S.status == PDHCG_ERR_INVALID) { __syncthreads(); continue; }
        const long long r0 = a.row_off[b], r1 = a.row_off[b + 1];
        const long long g0 = a.good_off[b];
        const int m = (int)(a.good_off[b + 1] - g0);
        const long long z0 = a.nnz_off[b], z1 = a.nnz_off[b + 1];
        double* P = a.p + g0;
        double* PC = a.pc + g0;
        double* PB = a.pbar + g0;
        double* PR = a.prs + g0;
        double* C0 = a.C[0] + g0;
        double* C1 = a.C[1] + g0;
        double* C2 = a.C[2] + g0;
        V* X0 = (V*)a.X[0];
        V* X1 = (V*)a.X[1];
        V* XB = (V*)a.Xb;
        V* XR = (V*)a.Xr;
        DevMarket dm = {};
        dm.n = (int)(r1 - r0);
        dm.m = m;
        dm.rp = a.rp;
        dm.cj = a.col;
        dm.uv = a.uv;
        dm.w = a.w;
        dm.hot = m;
        const int g = a.gsel[b];
        // ---- initial point (x_ij = 1/deg_j written by the prep kernel) ----
        const double p_init = S.sum_w / m;
        for (int j = threadIdx.x; j < m; j += blockDim.x) { P[j] = p_init; PB[j] = p_init; PR[j] = p_init; }
        for (long long q = z0 + threadIdx.x; q < z1; q += blockDim.x) XR[q] = X0[q];
        __syncthreads();
        double kout[4];
        kkt_market<MIXED>(a, r0, r1, g0, m, X0, P, acc, Mx, a.cc + g0, a.tc, scratch, kout);
        for (int j = threadIdx.x; j < m; j += blockDim.x) { C0[j] = a.cc[g0 + j]; C1[j] = a.cc[g0 + j]; }
        if (threadIdx.x == 0) {
            S.eta0 = a.eta0_scale / S.normK;
            S.omega0 = sqrt((double)m) * p_init / sqrt(S.x0n2);
            S.omega = S.omega0;
            S.eta = S.eta0;
            S.eta_min = a.eta_lo * S.eta0;
            S.eta_maxa = a.eta_hi * S.eta0;
            S.sum_eta = 0.0;
            S.fold_wgt = 1.0;
            S.fold_pending = 0;
            S.cur = 0; S.ck = 0; S.ckm1 = 1; S.cnew = 2;
            S.iters = S.passes = S.iters_rs = S.capped = 0;
            S.restarts = 0;
            S.kkt_rs = kout[3];
            S.kkt_prev = INFINITY;
            S.kkt = kout[3]; S.r_p = kout[0]; S.r_d = kout[1]; S.r_g = kout[2];
            S.use_avg = 0;
            S.g = g;
            go_on = kout[3] > a.tol;
            if (!go_on) S.status = PDHCG_OK;
        }
        for (int j = threadIdx.x; j < m; j += blockDim.x) acc[j] = 0ull;
        __syncthreads();
        while (go_on) {
            if (threadIdx.x == 0) S.chunk_acc = 0;
            __syncthreads();
            for (int q = 0; q < a.check_every + 8 && S.chunk_acc < a.check_every; q++) {
                // ---- price phase ----
                const double* ck = S.ck == 0 ? C0 : (S.ck == 1 ? C1 : C2);
                const double* ckm1 = S.ckm1 == 0 ? C0 : (S.ckm1 == 1 ? C1 : C2);
                for (int j = threadIdx.x; j < m; j += blockDim.x) {
                    double p = P[j];
                    if (S.fold_pending) {
                        p = PC[j];
                        P[j] = p;
                        PB[j] = (S.fold_wgt == 1.0) ? p : fma(S.fold_wgt, p - PB[j], PB[j]);
                    }
                    const double pc = fma(S.eta * S.omega, 2.0 * ck[j] - ckm1[j] - 1.0, p);   // sigma = eta * omega
                    PC[j] = pc;
                    if (MIXED) {
                        float h = (float)pc;
                        pff[j] = make_float2(h, (float)(pc - (double)h));
                    } else {
                        pcs[j] = pc;
                    }
                }
                __syncthreads();
                // ---- row phase ----
                RowCtx rc;
                rc.tau = S.eta / S.omega;
                rc.tau_hi = (float)rc.tau;
                rc.tau_lo = (float)(rc.tau - (double)rc.tau_hi);
                rc.fold = S.fold_pending;
                rc.fold_wd = S.fold_wgt;
                rc.fold_w = (float)rc.fold_wd;
                rc.cap = a.row_cap;
                rc.seed = mix32((unsigned)S.passes * 2u + 1u);
                const void* Xin = S.cur ? (const void*)X1 : (const void*)X0;
                void* Xout = S.cur ? (void*)X0 : (void*)X1;
                double dx2 = 0.0;
                int capped = 0;
                switch (g) {
                    case 4: row_phase<MIXED, 4, false>(a, dm, r0, r1, Xin, Xout, rc, pff, pcs, acc, dx2, capped); break;
                    case 8: row_phase<MIXED, 8, false>(a, dm, r0, r1, Xin, Xout, rc, pff, pcs, acc, dx2, capped); break;
                    case 16: row_phase<MIXED, 16, false>(a, dm, r0, r1, Xin, Xout, rc, pff, pcs, acc, dx2, capped); break;
                    case 32: row_phase<MIXED, 32, false>(a, dm, r0, r1, Xin, Xout, rc, pff, pcs, acc, dx2, capped); break;
                    default: row_phase<MIXED, 32, true>(a, dm, r0, r1, Xin, Xout, rc, pff, pcs, acc, dx2, capped); break;
                }
                dx2 = block_sum(dx2, scratch);
                const double capsum = block_sum((double)capped, scratch);
                // ---- dual phase ----
                double* cn = S.cnew == 0 ? C0 : (S.cnew == 1 ? C1 : C2);
                double s1 = 0.0, s2 = 0.0;
                for (int j = threadIdx.x; j < m; j += blockDim.x) {
                    unsigned long long v = acc[j];
                    acc[j] = 0ull;
                    const double c = MIXED ? (double)(long long)v * kFixInv : __longlong_as_double((long long)v);
                    cn[j] = c;
                    const double dp = PC[j] - P[j];
                    s1 = fma(dp, c - ck[j], s1);
                    s2 = fma(dp, dp, s2);
                }
                s1 = block_sum(s1, scratch);
                s2 = block_sum(s2, scratch);
                if (threadIdx.x == 0) {
                    S.capped += (long long)capsum;
                    S.passes += 1;
                    const double inter = fabs(s1);
                    const double om = S.omega, eta = S.eta;
                    if (!isfinite(dx2) || !isfinite(s2) || !isfinite(inter)) {
                        S.status = PDHCG_ERR_NUMERIC;
                        S.chunk_acc = a.check_every;   // leave the pass loop
                    } else {
                        const double movement = om * dx2 + s2 / om;
                        const double eta_max = inter > 0.0 ? movement / (2.0 * inter) : INFINITY;
                        const double k1 = (double)(S.iters + 1);
                        const double grow = (1.0 + pow(k1, -0.6)) * eta;
                        double en = isinf(eta_max) ? grow : fmin((1.0 - pow(k1, -0.3)) * eta_max, grow);
                        en = fmin(fmax(en, S.eta_min), S.eta_maxa);
                        const bool accept = (eta <= eta_max) || (eta <= S.eta_min * (1.0 + 1e-12));
                        if (accept) {
                            S.iters += 1;
                            S.chunk_acc += 1;
                            S.sum_eta += eta;
                            S.fold_wgt = eta / S.sum_eta;
                            S.fold_pending = 1;
                            S.cur = 1 - S.cur;
                            const int o = S.ckm1;
                            S.ckm1 = S.ck;
                            S.ck = S.cnew;
                            S.cnew = o;
                        } else {
                            S.fold_pending = 0;
                        }
                        S.eta = en;
                    }
                }
                __syncthreads();
            }
            if (S.status == PDHCG_ERR_NUMERIC) break;
            // ---- flush the last accepted step into the averages ----
            if (S.fold_pending) {
                const double wgt = S.fold_wgt;
                for (int j = threadIdx.x; j < m; j += blockDim.x) {
                    const double p = PC[j];
                    P[j] = p;
                    PB[j] = (wgt == 1.0) ? p : fma(wgt, p - PB[j], PB[j]);
                }
                const V* xc = S.cur ? X1 : X0;
                const V wv = (V)wgt;
                for (long long q = z0 + threadIdx.x; q < z1; q += blockDim.x)
                    XB[q] = (wgt == 1.0) ? xc[q] : XB[q] + wv * (xc[q] - XB[q]);
            }
            __syncthreads();
            if (threadIdx.x == 0) S.fold_pending = 0;
            __syncthreads();
            // ---- KKT of the current point and of the average ----
            double k0[4], k1[4];
            kkt_market<MIXED>(a, r0, r1, g0, m, S.cur ? (const void*)X1 : (const void*)X0, P, acc, Mx, a.cc + g0,
                              a.tc, scratch, k0);
            kkt_market<MIXED>(a, r0, r1, g0, m, XB, PB, acc, Mx, a.ca + g0, a.ta, scratch, k1);
            if (threadIdx.x == 0) {
                const bool avg = k1[3] < k0[3];
                const double* kb = avg ? k1 : k0;
                S.use_avg = avg;
                S.r_p = kb[0]; S.r_d = kb[1]; S.r_g = kb[2]; S.kkt = kb[3];
                do_restart = 0;
                go_on = 1;
                if (kb[3] <= a.tol) { S.status = PDHCG_OK; go_on = 0; }
                else if (S.iters >= a.max_iter || S.passes >= 4 * a.max_iter + 10000) {
                    S.status = PDHCG_ERR_NOT_CONVERGED;
                    go_on = 0;
                }
                else if ((double)(gtimer() - t_start) > a.time_limit_ns) { S.status = PDHCG_ERR_TIMEOUT; go_on = 0; }
                else {
                    const double kcand = kb[3];
                    const long long inner = S.iters - S.iters_rs;
                    bool rs = (kcand <= a.beta_suff * S.kkt_rs) ||
                              (kcand <= a.beta_nec * S.kkt_rs && kcand > S.kkt_prev) ||
                              ((double)inner >= a.beta_art * (double)S.iters);
                    do_restart = rs;
                    if (!rs) S.kkt_prev = kcand;
                }
            }
            __syncthreads();
            if (do_restart) {
                V* xc = S.cur ? X1 : X0;
                const bool avg = S.use_avg;
                if (avg) {
                    for (long long q = z0 + threadIdx.x; q < z1; q += blockDim.x) xc[q] = XB[q];
                    for (int j = threadIdx.x; j < m; j += blockDim.x) P[j] = PB[j];
                    for (long long i = r0 + threadIdx.x; i < r1; i += blockDim.x) a.tc[i] = a.ta[i];
                }
                double* ck = S.ck == 0 ? C0 : (S.ck == 1 ? C1 : C2);
                double* ckm1 = S.ckm1 == 0 ? C0 : (S.ckm1 == 1 ? C1 : C2);
                const double* csrc = avg ? a.ca + g0 : a.cc + g0;
                for (int j = threadIdx.x; j < m; j += blockDim.x) { ck[j] = csrc[j]; ckm1[j] = csrc[j]; }
                __syncthreads();
                const double dx2 = dist_copy_block<V>(xc, XR, z0, z1, scratch);
                const double dp2 = dist_copy_block<double>(P, PR, 0, m, scratch);
                if (threadIdx.x == 0) {
                    S.restarts += 1;
                    const double dx = sqrt(dx2), dp = sqrt(dp2);
                    if (dx > 1e-300 && dp > 1e-300)
                        S.omega = exp(a.theta * log(dp / dx) + (1.0 - a.theta) * log(S.omega));
                    if (a.omega_reset_every > 0 && S.restarts % a.omega_reset_every == 0) {
                        if (!(S.omega >= S.omega0 / a.omega_range && S.omega <= S.omega0 * a.omega_range))
                            S.omega = S.omega0;
                    }
                    S.sum_eta = 0.0;
                    S.fold_wgt = 1.0;
                    S.kkt_rs = S.kkt;
                    S.kkt_prev = INFINITY;
                    S.iters_rs = S.iters;
                    S.use_avg = 0;
                }
                __syncthreads();
            }
        }
        __syncthreads();
        if (threadIdx.x == 0) a.st[b] = S;
        __syncthreads();
    }
}

// final candidate of every market: prices and utilities in caller units, and
// the equilibrium kept for the derivative (x, p, scaled t, global good ids)
template <typename V>
__global__ void batch_out_kernel(BatchArgs a, double* p_out, double* u_out, V* xf, double* pf, double* tf, int* cjg,
                                 double* wcopy) {
    const int b = blockIdx.x;
    if (b >= a.B) return;
    const MState& S = a.st[b];
    const long long r0 = a.row_off[b], r1 = a.row_off[b + 1], g0 = a.good_off[b];
    const long long z0 = a.nnz_off[b], z1 = a.nnz_off[b + 1];
    const int m = (int)(a.good_off[b + 1] - g0);
    const bool avg = S.use_avg;
    const V* xs = avg ? (const V*)a.Xb : (S.cur ? (const V*)a.X[1] : (const V*)a.X[0]);
    for (int j = threadIdx.x; j < m; j += blockDim.x) {
        const double p = avg ? a.pbar[g0 + j] : a.p[g0 + j];
        p_out[g0 + j] = p;
        pf[g0 + j] = p;
    }
    for (long long i = r0 + threadIdx.x; i < r1; i += blockDim.x) {
        const double t = avg ? a.ta[i] : a.tc[i];
        tf[i] = t;
        wcopy[i] = a.w[i];
        if (u_out) u_out[i] = t * a.rowmax[i];
    }
    for (long long q = z0 + threadIdx.x; q < z1; q += blockDim.x) {
        xf[q] = xs[q];
        cjg[q] = (int)g0 + a.col[q];
    }
}

}  // namespace pdhcg

using namespace pdhcg;


namespace {

// default lanes per row for a market whose longest row has `maxdeg` entries
int default_group(int maxdeg) {
    if (maxdeg <= 4 * kSlots) return 4;
    if (maxdeg <= 8 * kSlots) return 8;
    if (maxdeg <= 16 * kSlots) return 16;
    if (maxdeg <= 32 * kSlots) return 32;
    return 0;   // long rows: 32 lanes, streamed in chunks
}
int degree_class(int maxdeg) {
    int g = default_group(maxdeg);
    return g == 4 ? 0 : g == 8 ? 1 : g == 16 ? 2 : g == 32 ? 3 : 4;
}

size_t solve_smem(int mmax) { return (size_t)mmax * 3 * sizeof(unsigned long long); }

void launch_solve(bool mixed, const BatchArgs& a, int grid, size_t smem, cudaStream_t s) {
    if (mixed) batch_solve_kernel<true><<<grid, kThreads, smem, s>>>(a);
    else batch_solve_kernel<false><<<grid, kThreads, smem, s>>>(a);
}
void launch_prep(bool mixed, const BatchArgs& a, int mmax, cudaStream_t s) {
    size_t sm = (size_t)mmax * sizeof(int);
    if (mixed) batch_prep_kernel<float><<<a.B, 256, sm, s>>>(a);
    else batch_prep_kernel<double><<<a.B, 256, sm, s>>>(a);
}

}  // namespace

pdhcg_status pdhcg_fisher_solve_batched(pdhcg_handle h, int32_t B, const int64_t* row_off, const int64_t* good_off,
                                        const int64_t* nnz_off, const int64_t* row_ptr, const int32_t* col,
                                        const void* val, pdhcg_valtype val_type, const double* w,
                                        const pdhcg_params* prm, double* p_out, double* util_out,
                                        pdhcg_info* info_out) {
    if (!h || B <= 0 || !row_off || !good_off || !nnz_off || !row_ptr || !col || !val || !w || !prm || !p_out)
        return PDHCG_ERR_INVALID;
    if (!(prm->tol > 0) || prm->max_iter <= 0 || prm->kkt_check_every <= 0 || prm->row_solve_max_iter <= 0)
        return PDHCG_ERR_INVALID;
    {
        const int bl = prm->batch_lanes;
        if (bl != 0 && bl != 4 && bl != 8 && bl != 16 && bl != 32 && bl != 64) return PDHCG_ERR_INVALID;
    }
    enter(h);
    h->state.valid = false;
    cudaStream_t s = h->stream;
    const bool mixed = prm->prec == PDHCG_MIXED;
    const bool f32 = val_type == PDHCG_VAL_F32;
    const size_t vb = mixed ? 4 : 8;
    // offsets on the host (for sizes and the schedule) and on the device
    std::vector<long long> ro(B + 1), go(B + 1), zo(B + 1);
    const bool dev_off = is_device_ptr(row_off);
    if (dev_off) {
        CK(cudaMemcpyAsync(ro.data(), row_off, (B + 1) * 8, cudaMemcpyDeviceToHost, s));
        CK(cudaMemcpyAsync(go.data(), good_off, (B + 1) * 8, cudaMemcpyDeviceToHost, s));
        CK(cudaMemcpyAsync(zo.data(), nnz_off, (B + 1) * 8, cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
    } else {
        memcpy(ro.data(), row_off, (B + 1) * 8);
        memcpy(go.data(), good_off, (B + 1) * 8);
        memcpy(zo.data(), nnz_off, (B + 1) * 8);
    }
    if (ro[0] != 0 || go[0] != 0 || zo[0] != 0) return PDHCG_ERR_INVALID;
    int mmax = 0;
    for (int b = 0; b < B; b++) {
        const long long mb = go[b + 1] - go[b];
        if (ro[b + 1] <= ro[b] || mb <= 0 || mb > kBatchMaxGoods || zo[b + 1] < zo[b]) return PDHCG_ERR_INVALID;
        mmax = std::max<int>(mmax, (int)mb);
    }
    const long long N = ro[B], Mt = go[B], NNZ = zo[B];
    cudaError_t err = cudaSuccess;
    DevBuf* bt = h->bt;
    const long long* d_ro = (const long long*)stage_in(bt[14], row_off, (B + 1) * 8, s, &err);
    const long long* d_go = (const long long*)stage_in(bt[15], good_off, (B + 1) * 8, s, &err);
    const long long* d_zo = (const long long*)stage_in(bt[16], nnz_off, (B + 1) * 8, s, &err);
    const long long* d_rp = (const long long*)stage_in(h->in_rp, row_ptr, (N + 1) * 8, s, &err);
    const int* d_col = (const int*)stage_in(h->in_col, col, NNZ * 4, s, &err);
    const void* d_val = stage_in(h->in_val, val, NNZ * (f32 ? 4 : 8), s, &err);
    const double* d_w = (const double*)stage_in(h->in_w, w, N * 8, s, &err);
    CK(err);
    CK(ensure(bt[0], NNZ * vb));
    CK(ensure(bt[1], NNZ * vb));
    CK(ensure(bt[2], NNZ * vb));
    CK(ensure(bt[3], NNZ * vb));
    CK(ensure(bt[4], NNZ * vb));
    CK(ensure(bt[5], 3 * N * sizeof(double)));
    CK(ensure(bt[8], 9 * Mt * sizeof(double)));
    CK(ensure(bt[9], Mt * sizeof(int)));
    CK(ensure(bt[10], B * sizeof(MState)));
    CK(ensure(bt[11], B * sizeof(int)));
    CK(ensure(bt[12], B * sizeof(int)));
    CK(ensure(bt[13], 16));
    CK(ensure(bt[17], B * sizeof(int)));
    BatchArgs a = {};
    a.B = B;
    a.row_off = d_ro;
    a.good_off = d_go;
    a.nnz_off = d_zo;
    a.rp = d_rp;
    a.col = d_col;
    a.val = d_val;
    a.val_f32 = f32 ? 1 : 0;
    a.w = d_w;
    a.uv = bt[0].p;
    a.X[0] = bt[1].p;
    a.X[1] = bt[2].p;
    a.Xb = bt[3].p;
    a.Xr = bt[4].p;
    a.rowmax = (double*)bt[5].p;
    a.tc = a.rowmax + N;
    a.ta = a.rowmax + 2 * N;
    double* gv = (double*)bt[8].p;
    a.p = gv;
    a.pc = gv + Mt;
    a.pbar = gv + 2 * Mt;
    a.prs = gv + 3 * Mt;
    a.C[0] = gv + 4 * Mt;
    a.C[1] = gv + 5 * Mt;
    a.C[2] = gv + 6 * Mt;
    a.cc = gv + 7 * Mt;
    a.ca = gv + 8 * Mt;
    a.deg = (int*)bt[9].p;
    a.st = (MState*)bt[10].p;
    a.order = (const int*)bt[11].p;
    a.gsel = (const int*)bt[12].p;
    a.queue = (unsigned int*)bt[13].p;
    a.tol = prm->tol;
    a.eta_lo = prm->eta_lo;
    a.eta_hi = prm->eta_hi;
    a.eta0_scale = prm->eta0_scale;
    a.beta_suff = prm->beta_suff;
    a.beta_nec = prm->beta_nec;
    a.beta_art = prm->beta_art;
    a.theta = prm->theta;
    a.omega_range = prm->omega_range;
    a.max_iter = prm->max_iter;
    a.check_every = prm->kkt_check_every;
    a.omega_reset_every = prm->omega_reset_every;
    a.row_cap = prm->row_solve_max_iter;
    a.time_limit_ns = prm->time_limit_s * 1e9;
    a.smem_goods = mmax;
    const size_t smem = solve_smem(mmax);
    static bool attr = false;
    if (!attr) {
        attr = true;
        cudaFuncSetAttribute(batch_solve_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
        cudaFuncSetAttribute(batch_solve_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    }
    int per = 0, sm = 0, dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sm, cudaDevAttrMultiProcessorCount, dev);
    if (mixed) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, batch_solve_kernel<true>, kThreads, smem);
    else cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, batch_solve_kernel<false>, kThreads, smem);
    if (per < 1) per = 1;
    const int grid = std::min<long long>((long long)sm * per, B);
    // ---- preprocessing and per-market validation ----
    launch_prep(mixed, a, mmax, s);
    CK(cudaGetLastError());
    std::vector<MState> st(B);
    CK(cudaMemcpyAsync(st.data(), a.st, B * sizeof(MState), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    for (int b = 0; b < B; b++)
        if (st[b].status == PDHCG_ERR_INVALID) {
            h->last_err = st[b].err;
            return PDHCG_ERR_INVALID;
        }
    // ---- schedule: largest markets first ----
    std::vector<int> order(B);
    for (int b = 0; b < B; b++) order[b] = b;
    std::stable_sort(order.begin(), order.end(),
                     [&](int x, int y) { return zo[x + 1] - zo[x] > zo[y + 1] - zo[y]; });
    CK(cudaMemcpyAsync((void*)a.order, order.data(), B * sizeof(int), cudaMemcpyHostToDevice, s));
    // ---- autotuner: lanes per row for each degree class ----
    std::vector<int> cls(B);
    std::vector<std::vector<int>> members(5);
    for (int b = 0; b < B; b++) {
        cls[b] = degree_class(st[b].maxdeg);
        members[cls[b]].push_back(b);
    }
    int* table = mixed ? h->bt_table_mixed : h->bt_table_fp64;
    int forced[5] = {-1, -1, -1, -1, -1};
    if (prm->batch_lanes) {
        // a caller's width for every class whose rows fit it (classes are
        // ordered by the width their longest rows need; 0 = chunked)
        const int cand[5] = {4, 8, 16, 32, 0};
        for (int c = 0; c < 5; c++) {
            if (prm->batch_lanes == 64 || c == 4) forced[c] = 0;
            else forced[c] = std::max(prm->batch_lanes, cand[c]);
        }
        table = forced;
    }
    const int cand_g[5] = {4, 8, 16, 32, 0};
    bool tuned = false;
    for (int c = 0; c < 5; c++) {
        if (members[c].empty() || table[c] >= 0) continue;
        // up to 4 markets of the class, from the middle of its size range
        std::vector<int> smp = members[c];
        std::stable_sort(smp.begin(), smp.end(), [&](int x, int y) { return zo[x + 1] - zo[x] > zo[y + 1] - zo[y]; });
        const size_t k0 = smp.size() / 2 > 2 ? smp.size() / 2 - 2 : 0;
        std::vector<int> sample(smp.begin() + k0, smp.begin() + std::min(smp.size(), k0 + 4));
        float best_ms = 1e30f;
        int best_g = cand_g[c];
        for (int q = c; q < 5; q++) {
            const int gq = cand_g[q];
            std::vector<int> gs(B, gq);
            CK(cudaMemcpyAsync((void*)a.gsel, gs.data(), B * sizeof(int), cudaMemcpyHostToDevice, s));
            BatchArgs t = a;
            t.B = (int)sample.size();
            t.order = (const int*)h->bt[17].p;
            t.max_iter = prm->kkt_check_every;
            t.tol = 0.0;
            CK(cudaMemcpyAsync((void*)t.order, sample.data(), sample.size() * sizeof(int), cudaMemcpyHostToDevice, s));
            cudaEvent_t e0, e1;
            cudaEventCreate(&e0);
            cudaEventCreate(&e1);
            float ms = 0.0f;
            cudaError_t te = cudaSuccess;
            for (int rep = 0; rep < 2 && te == cudaSuccess; rep++) {      // first run warms up
                te = cudaMemsetAsync(a.queue, 0, 16, s);
                if (te != cudaSuccess) break;
                cudaEventRecord(e0, s);
                launch_solve(mixed, t, std::min<int>(grid, t.B), smem, s);
                cudaEventRecord(e1, s);
                te = cudaEventSynchronize(e1);
                if (te == cudaSuccess) cudaEventElapsedTime(&ms, e0, e1);
            }
            cudaEventDestroy(e0);
            cudaEventDestroy(e1);
            CK(te);
            CK(cudaGetLastError());
            if (ms < best_ms) { best_ms = ms; best_g = gq; }
            if (prm->verbose) fprintf(stderr, "[pdhcg-batch] tune class %d g %d: %.3f ms\n", c, gq, ms);
        }
        table[c] = best_g;
        tuned = true;
    }
    std::vector<int> gsel(B);
    for (int b = 0; b < B; b++) gsel[b] = table[cls[b]] >= 0 ? table[cls[b]] : default_group(st[b].maxdeg);
    CK(cudaMemcpyAsync((void*)a.gsel, gsel.data(), B * sizeof(int), cudaMemcpyHostToDevice, s));
    if (tuned) {           // tuning runs moved the iterates: start again from the prepared point
        launch_prep(mixed, a, mmax, s);
        CK(cudaGetLastError());
    }
    // ---- the persistent launch (one kernel: nothing for a graph to batch) ----
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    cudaEventRecord(e0, s);
    cudaError_t ce = cudaMemsetAsync(a.queue, 0, 16, s);
    if (ce == cudaSuccess) {
        launch_solve(mixed, a, grid, smem, s);
        ce = cudaGetLastError();
    }
    cudaEventRecord(e1, s);
    if (ce == cudaSuccess) ce = cudaStreamSynchronize(s);
    float solve_ms = 0.0f;
    cudaEventElapsedTime(&solve_ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    CK(ce);
    CK(cudaGetLastError());
    // ---- outputs ----
    double* pd = (double*)out_loc(h->o_p, p_out, Mt * 8, &err);
    double* ud = (double*)out_loc(h->o_u, util_out, N * 8, &err);
    CK(err);
    CK(ensure(bt[18], NNZ * vb));
    CK(ensure(bt[19], NNZ * sizeof(int)));
    CK(ensure(bt[20], N * sizeof(double)));
    CK(ensure(bt[21], (N + 1) * sizeof(long long)));
    CK(ensure(bt[22], Mt * sizeof(double)));
    CK(ensure(bt[23], N * sizeof(double)));
    CK(cudaMemcpyAsync(bt[21].p, d_rp, (N + 1) * sizeof(long long), cudaMemcpyDeviceToDevice, s));
    if (mixed)
        batch_out_kernel<float><<<B, 256, 0, s>>>(a, pd, ud, (float*)bt[18].p, (double*)bt[22].p, (double*)bt[23].p,
                                                  (int*)bt[19].p, (double*)bt[20].p);
    else
        batch_out_kernel<double><<<B, 256, 0, s>>>(a, pd, ud, (double*)bt[18].p, (double*)bt[22].p,
                                                   (double*)bt[23].p, (int*)bt[19].p, (double*)bt[20].p);
    CK(copy_out(p_out, pd, Mt * 8, s));
    CK(copy_out(util_out, ud, N * 8, s));
    CK(cudaMemcpyAsync(st.data(), a.st, B * sizeof(MState), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    pdhcg_status all = PDHCG_OK;
    for (int b = 0; b < B; b++) {
        const MState& S = st[b];
        if (S.status != PDHCG_OK && all == PDHCG_OK) all = (pdhcg_status)S.status;
        if (info_out) {
            pdhcg_info& I = info_out[b];
            memset(&I, 0, sizeof(I));
            I.iters = S.iters;
            I.passes = S.passes;
            I.restarts = S.restarts;
            I.kkt = S.kkt;
            I.r_primal = S.r_p;
            I.r_dual = S.r_d;
            I.r_gap = S.r_g;
            I.solve_ms = solve_ms;
            I.bytes_moved = (double)S.passes * (double)(zo[b + 1] - zo[b]) * (mixed ? 24.0 : 44.0);
            I.row_solve_capped = (int32_t)std::min<long long>(S.capped, 2147483647LL);
            I.status = (pdhcg_status)S.status;
            I.kernel_launches = 1;
        }
    }
    h->state.valid = (all == PDHCG_OK);
    h->state.kind = 2;
    h->batch_B = B;
    h->bt_N = (int)N;
    h->bt_M = (int)Mt;
    h->bt_NNZ = NNZ;
    h->bt_mixed = mixed;
    h->tight_kappa = prm->tight_kappa;
    h->bt_kkt_max = 0.0;
    for (int b = 0; b < B; b++) h->bt_kkt_max = std::max(h->bt_kkt_max, st[b].kkt);
    return all;
}
