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
// The row solver itself (rowsolve.cuh) replaces the paper's 32-section search
// (a GPU design for H100) by an exact finite procedure; the paper's searches
// remain in the oracle.
#include "common.cuh"
#include "rowsolve.cuh"
#include "rowsolve_mixed.cuh"

namespace pdhcg {

// ---------------------------------------------------------------------------
// the persistent row kernel
// ---------------------------------------------------------------------------
// One bucket of register-resident rows (MIXED): each warp takes chunks of
// units from the bucket's counter; while one unit is solved the next unit's
// (good id, utility, x^k) are already being loaded (software prefetch).
template <int G>
__device__ void bucket_mixed(const DevMarket& mk, const Bucket& bk, unsigned long long* counter, const void* Xin,
                             void* Xout, const IterBufs& bf, const float2* sp, unsigned long long* acc_s,
                             const RowCtxM& rc, float& dxf, int& capped, int& evals) {
    constexpr int rpw = 32 / G;
    const int lane = threadIdx.x & 31;
    const long long units = (bk.count + rpw - 1) / rpw;
    const float* U = (const float*)mk.uv;
    const float* Xi = (const float*)Xin;
    while (true) {
        unsigned long long base = 0;
        if (lane == 0) base = atomicAdd(counter, 16ull);
        base = __shfl_sync(0xffffffffu, base, 0);
        if ((long long)base >= units) break;
        const long long uend = min((long long)base + 16, units);
        long long slot = (long long)base * rpw + lane / G;
        bool vn = slot < bk.count;
        int rn = vn ? (int)(bk.first + slot) : 0;
        RowRegsM nx;
        rowm_load<G>(mk, U, Xi, rn, vn, nx);
        for (long long u = (long long)base; u < uend; u++) {
            RowRegsM cr = nx;
            const int rc_row = rn;
            const bool vc = vn;
            if (u + 1 < uend) {
                slot = (u + 1) * rpw + lane / G;
                vn = slot < bk.count;
                rn = vn ? (int)(bk.first + slot) : 0;
                rowm_load<G>(mk, U, Xi, rn, vn, nx);
            }
            rowm_core<G>(mk, (float*)Xout, bf.pff, sp, acc_s, bf.acc, bf.yst, rc, rc_row, vc, dxf, capped, evals,
                         cr);
        }
    }
}

template <bool MIXED>
__global__ void __launch_bounds__(kProxThreads, 1) prox_kernel(DevMarket mk, const void* Xin_fixed, void* Xout_fixed,
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
    rc.seed = mix32((unsigned)ctl->passes * 2u + 1u);
    rc.sections = ctl->sections;
    rc.sec_tol = ctl->sec_tol;
    RowCtxM rm;       // MIXED: x-bar is folded by fold_pair_kernel, not here
    rm.tau = rc.tau_hi;
    rm.cap = rc.cap;
    rm.seed = rc.seed;
    const int cur = ctl->cur;
    const void* Xin = fixed ? Xin_fixed : (cur ? bf.X[1] : bf.X[0]);
    void* Xout = fixed ? Xout_fixed : (cur ? bf.X[0] : bf.X[1]);
    // shared memory: column sums of the hot goods, then (MIXED) their prices
    float2* sp = (float2*)(acc_s + mk.hot);
    for (int j = threadIdx.x; j < mk.hot; j += blockDim.x) {
        acc_s[j] = 0ull;
        if (MIXED) sp[j] = bf.pff[j];
    }
    __syncthreads();

    const int lane = threadIdx.x & 31;
    float dxf = 0.0f;
    double dxd = 0.0;
    int capped = 0, evals = 0;

    for (int bi = 0; bi < mk.nb; bi++) {
        const Bucket bk = mk.buckets[bi];
        const int g = bk.g;
        if (MIXED && !bk.chunks) {
            switch (g) {
                case 4: bucket_mixed<4>(mk, bk, &ctl->work[bi], Xin, Xout, bf, sp, acc_s, rm, dxf, capped, evals); break;
                case 8: bucket_mixed<8>(mk, bk, &ctl->work[bi], Xin, Xout, bf, sp, acc_s, rm, dxf, capped, evals); break;
                case 16: bucket_mixed<16>(mk, bk, &ctl->work[bi], Xin, Xout, bf, sp, acc_s, rm, dxf, capped, evals); break;
                default: bucket_mixed<32>(mk, bk, &ctl->work[bi], Xin, Xout, bf, sp, acc_s, rm, dxf, capped, evals); break;
            }
            continue;
        }
        const int rpw = 32 / g;
        const long long units = (bk.count + rpw - 1) / rpw;
        const long long grab = bk.chunks ? 1 : 16;       // units taken per atomic
        while (true) {
            unsigned long long base = 0;
            if (lane == 0) base = atomicAdd(&ctl->work[bi], (unsigned long long)grab);
            base = __shfl_sync(0xffffffffu, base, 0);
            if ((long long)base >= units) break;
            const long long uend = min((long long)base + grab, units);
            for (long long u = (long long)base; u < uend; u++) {
                long long slot = u * rpw + lane / g;
                bool valid = slot < bk.count;
                int row = valid ? (int)(bk.first + slot) : 0;
                if (MIXED) {
                    if (valid)
                        rowm_long(mk, (const float*)mk.uv, (const float*)Xin, (float*)Xout, bf.pff, sp, acc_s,
                                  bf.acc, bf.yst, rm, row, dxf, capped, evals);
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
    }

    // ---- block epilogue: ||dx||^2 partial, capped rows, flush hot column sums ----
    double v = MIXED ? (double)dxf : dxd;
    v = warp_sum_d(v);
    __shared__ double red[kProxWarps];
    __shared__ int capred, evred;
    if (threadIdx.x == 0) capred = evred = 0;
    __syncthreads();
    if (lane == 0) red[threadIdx.x >> 5] = v;
    if (capped) atomicAdd(&capred, capped);
    if (evals) atomicAdd(&evred, evals);
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < kProxWarps; w++) t += red[w];
        bf.part[blockIdx.x] = t;
        if (capred) atomicAdd((unsigned long long*)&ctl->capped, (unsigned long long)capred);
        if (evred) atomicAdd((unsigned long long*)&ctl->evals, (unsigned long long)evred);
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
    if (blockIdx.x == 0 && threadIdx.x < kMaxBuckets) ctl->work[threadIdx.x] = 0ull;
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
    // MIXED x-bar: a pair waiting at the start of this pass has been folded by
    // the fold kernel that ran after the previous pass
    int xf = ctl->xf_n == 2 ? 0 : ctl->xf_n;
    ctl->xf_folded = 0;
    if (accept) {
        ctl->iters += 1;
        ctl->chunk_acc += 1;
        ctl->sum_eta += eta;
        ctl->fold_wgt = eta / ctl->sum_eta;
        if (xf == 0) ctl->xf_w1 = ctl->fold_wgt;
        else ctl->xf_w2 = ctl->fold_wgt;
        xf++;
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
    ctl->xf_n = xf;
    ctl->eta = eta_next;
    ctl->tau = eta_next / om;
    ctl->sigma = eta_next * om;
}

// ---------------------------------------------------------------------------
// flush: commit + fold the last accepted step into the averages (chunk end)
// ---------------------------------------------------------------------------
template <typename V>
__global__ void flush_x_kernel(long long nnz, IterBufs bf, Ctl* ctl) {
    const V* x = (const V*)(ctl->cur ? bf.X[1] : bf.X[0]);
    V* xb = (V*)bf.Xb;
    if constexpr (sizeof(V) == sizeof(float)) {
        // MIXED: fold a single waiting accepted iterate (a pair has already
        // been folded by fold_pair_kernel)
        const int nf = ctl->xf_n;
        if (nf != 1) return;
        const V* xo = (const V*)(ctl->cur ? bf.X[0] : bf.X[1]);      // the older one of a pair
        const double w1 = ctl->xf_w1, w2 = ctl->xf_w2;
        const float fw1 = (float)w1, fw2 = (float)w2, c1 = (float)((1.0 - w2) * w1);
        const unsigned seed = mix32((unsigned)ctl->passes * 2u + 2u);
        for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < nnz; i += (long long)gridDim.x * blockDim.x) {
            const float r = rand01_hi(sr_bits(i, seed));
            const float b = x[i];
            float v;
            if (nf == 1) v = (w1 == 1.0) ? b : sr_add_rd(xb[i], fw1 * (b - xb[i]), r);
            else {
                const float a = xo[i];
                v = (w1 == 1.0) ? sr_add_rd(a, fw2 * (b - a), r) : sr_add_rd(xb[i], fmaf(c1, a - xb[i], fw2 * (b - xb[i])), r);
            }
            xb[i] = v;
        }
    } else {
        if (!ctl->fold_pending) return;
        const double wgt = ctl->fold_wgt;
        for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < nnz; i += (long long)gridDim.x * blockDim.x) {
            const V xv = x[i];
            xb[i] = (wgt == 1.0) ? xv : xb[i] + (V)wgt * (xv - xb[i]);
        }
    }
}
// MIXED x-bar, two accepted iterates at a time (Alg. 2 average, weights
// eta_k / sum eta, reading R5).  Runs after every dual kernel and acts when two
// accepted iterates are waiting: the older (weight w1) in X[1 - cur], the newer
// (weight w2) in X[cur], both untouched until the next row pass writes
// X[1 - cur].  Folding x_a then x_b,
//     x-bar <- (1 - w2)(1 - w1) x-bar + (1 - w2) w1 x_a + w2 x_b
//            = x-bar + c1 (x_a - x-bar) + w2 (x_b - x-bar),   c1 = (1 - w2) w1,
// and w1 = 1 (the first iterate after a restart) gives x_a + w2 (x_b - x_a).
// A streaming pass (16 B per entry for two iterations) instead of a fold
// inside the row kernel, where its loads and registers slowed the row solve.
__global__ void __launch_bounds__(256) fold_pair_kernel(long long nnz, IterBufs bf, Ctl* ctl) {
    // the kernel runs after every dual kernel of the chunk graph, also after the
    // idle ones at the end of a chunk: each pair is folded exactly once
    if (ctl->xf_n != 2 || ctl->xf_folded) return;
    const int cur = ctl->cur;
    const float* __restrict__ xa = (const float*)(cur ? bf.X[0] : bf.X[1]);
    const float* __restrict__ xn = (const float*)(cur ? bf.X[1] : bf.X[0]);
    float* __restrict__ xb = (float*)bf.Xb;
    const double w1 = ctl->xf_w1, w2 = ctl->xf_w2;
    const bool first = w1 == 1.0;
    const float fw2 = (float)w2, c1 = (float)((1.0 - w2) * w1);
    const unsigned seed = mix32((unsigned)ctl->passes * 2u + 2u);
    const long long n4 = nnz >> 2;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < n4; q += stride) {
        const float4 a = __ldcs((const float4*)xa + q);
        const float4 b = __ldcs((const float4*)xn + q);
        const float4 v = first ? make_float4(0.f, 0.f, 0.f, 0.f) : __ldcs((const float4*)xb + q);
        const unsigned h = row_hash(q, seed);
        float4 o;
        o.x = first ? sr_add_rd(a.x, fw2 * (b.x - a.x), rand01_lo(entry_hash(h, 0)))
                    : sr_add_rd(v.x, fmaf(c1, a.x - v.x, fw2 * (b.x - v.x)), rand01_lo(entry_hash(h, 0)));
        o.y = first ? sr_add_rd(a.y, fw2 * (b.y - a.y), rand01_lo(entry_hash(h, 1)))
                    : sr_add_rd(v.y, fmaf(c1, a.y - v.y, fw2 * (b.y - v.y)), rand01_lo(entry_hash(h, 1)));
        o.z = first ? sr_add_rd(a.z, fw2 * (b.z - a.z), rand01_lo(entry_hash(h, 2)))
                    : sr_add_rd(v.z, fmaf(c1, a.z - v.z, fw2 * (b.z - v.z)), rand01_lo(entry_hash(h, 2)));
        o.w = first ? sr_add_rd(a.w, fw2 * (b.w - a.w), rand01_lo(entry_hash(h, 3)))
                    : sr_add_rd(v.w, fmaf(c1, a.w - v.w, fw2 * (b.w - v.w)), rand01_lo(entry_hash(h, 3)));
        __stcs((float4*)xb + q, o);
    }
    // the ragged tail (nnz not a multiple of 4)
    for (long long i = 4 * n4 + blockIdx.x * (long long)blockDim.x + threadIdx.x; i < nnz; i += stride) {
        const float a = xa[i], b = xn[i];
        const float r = rand01_lo(entry_hash(row_hash(i >> 2, seed), (unsigned)(i & 3)));
        xb[i] = first ? sr_add_rd(a, fw2 * (b - a), r) : sr_add_rd(xb[i], fmaf(c1, a - xb[i], fw2 * (b - xb[i])), r);
    }
    // last block done: mark the pair folded (every block has read the flag by now)
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        if (atomicAdd(&ctl->xf_ticket, 1u) == gridDim.x - 1) {
            ctl->xf_ticket = 0u;
            ctl->xf_folded = 1;
        }
    }
}

__global__ void flush_p_kernel(int m, IterBufs bf, Ctl* ctl) {
    const bool pending = ctl->fold_pending;
    const double wgt = ctl->fold_wgt;
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < m; j += gridDim.x * blockDim.x) {
        double p = bf.p[j], pb = bf.pbar[j];
        if (pending) {
            p = bf.pc[j];
            bf.p[j] = p;
            pb = (wgt == 1.0) ? p : fma(wgt, p - pb, pb);
            bf.pbar[j] = pb;
        }
        if (bf.pff_p) {
            float h = (float)p;
            bf.pff_p[j] = make_float2(h, (float)(p - (double)h));
            h = (float)pb;
            bf.pff_pb[j] = make_float2(h, (float)(pb - (double)h));
        }
    }
}
__global__ void flush_done_kernel(Ctl* ctl) {
    ctl->fold_pending = 0;
    ctl->xf_n = 0;
    ctl->xf_folded = 0;
}

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
// shared memory of the row kernel: hot column sums (8 B) and, MIXED, hot prices (8 B)
static size_t prox_smem_bytes(bool mixed, int hot) { return (size_t)hot * (mixed ? 16 : 8); }
static size_t prox_smem(const DevMarket& mk) { return prox_smem_bytes(mk.uv != nullptr && mk.mixed, mk.hot); }

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
    size_t smem = prox_smem_bytes(mixed, hot);
    if (mixed) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, prox_kernel<true>, kProxThreads, smem);
    else cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, prox_kernel<false>, kProxThreads, smem);
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
    if (mixed) prox_kernel<true><<<mk.nprox, kProxThreads, prox_smem(mk), s>>>(mk, nullptr, nullptr, b, ctl, 0);
    else prox_kernel<false><<<mk.nprox, kProxThreads, prox_smem(mk), s>>>(mk, nullptr, nullptr, b, ctl, 0);
}
void launch_dual(bool mixed, const DevMarket& mk, const IterBufs& b, Ctl* ctl, cudaStream_t s) {
    int nb = vec_blocks(mk.m);
    if (nb > 256) nb = 256;
    if (mixed) dual_kernel<true><<<nb, 256, 0, s>>>(mk, b, ctl, mk.nprox);
    else dual_kernel<false><<<nb, 256, 0, s>>>(mk, b, ctl, mk.nprox);
}
void launch_fold(bool mixed, const DevMarket& mk, const IterBufs& b, Ctl* ctl, cudaStream_t s) {
    if (!mixed) return;          // FP64 folds x-bar inside the row kernel, one iterate per pass
    fold_pair_kernel<<<sm_count() * 8, 256, 0, s>>>(mk.nnz, b, ctl);
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
__global__ void to_ff_kernel(int m, const double* p, float2* pff) {
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < m; j += gridDim.x * blockDim.x) {
        const double v = p[j];
        const float h = (float)v;
        pff[j] = make_float2(h, (float)(v - (double)h));
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
    for (int i = 0; i < kMaxBuckets; i++) ctl->work[i] = 0ull;
    ctl->active = 1;
    ctl->tau = tau;
    ctl->fold_pending = 0;
    ctl->xf_n = 0;
    ctl->sections = 0;
    ctl->cur = 0;
    ctl->row_cap = cap;
    ctl->capped = 0;
    ctl->evals = 0;
}

void launch_to_ff(int m, const double* p, float2* pff, cudaStream_t s) {
    to_ff_kernel<<<vec_blocks(m), 256, 0, s>>>(m, p, pff);
}

// MIXED fixed pass: the y state starts at 1 (any y > 0 is a valid start) and
// is converted to s = w / y afterwards, in place
__global__ void yfill_kernel(int n, float2* y) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) y[i] = make_float2(1.0f, 0.0f);
}
__global__ void y_to_s_kernel(int n, const double* __restrict__ w, double* t) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const float2 v = ((const float2*)t)[i];
        t[i] = w[i] / ((double)v.x + (double)v.y);
    }
}

void launch_prox_fixed(bool mixed, const DevMarket& mk, const void* x_in, void* x_out, const double* p,
                       double tau, unsigned long long* acc, double* t_out, double* c_out,
                       double* part, Ctl* ctl, cudaStream_t s) {
    set_smem_attr();
    IterBufs b = {};
    b.acc = acc;
    b.t = t_out;
    b.yst = (float2*)t_out;     // MIXED: y state in the same buffer (8 bytes per row)
    b.part = part;
    // scratch for the converted prices lives after the m accumulators
    b.pff = (float2*)(acc + mk.m);
    b.pc = (double*)(acc + 2 * (size_t)mk.m);
    p_to_ff_kernel<<<vec_blocks(mk.m), 256, 0, s>>>(mk.m, p, b.pff, b.pc);
    ctl_fixed_kernel<<<1, 1, 0, s>>>(ctl, tau, 64);
    if (mixed) {
        yfill_kernel<<<vec_blocks(mk.n), 256, 0, s>>>(mk.n, b.yst);
        prox_kernel<true><<<mk.nprox, kProxThreads, prox_smem(mk), s>>>(mk, x_in, x_out, b, ctl, 1);
        y_to_s_kernel<<<vec_blocks(mk.n), 256, 0, s>>>(mk.n, mk.w, t_out);
    } else {
        prox_kernel<false><<<mk.nprox, kProxThreads, prox_smem(mk), s>>>(mk, x_in, x_out, b, ctl, 1);
    }
    cols_out_kernel<<<vec_blocks(mk.m), 256, 0, s>>>(mk.m, mixed, acc, c_out);
}

}  // namespace pdhcg
