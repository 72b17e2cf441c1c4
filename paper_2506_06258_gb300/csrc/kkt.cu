// Relative KKT error of Section 5 ("Criteria") for a point (x, p) of the
// row-scaled market, with t_i = u_i^T x_i and y = w/t (so the terms
// ||w/t - y|| and |t - u^T x| vanish):
//
//   r_primal = max_j |c_j - 1| / (1 + max(max_j c_j, 1)),   c_j = sum_i x_ij
//   r_dual   = max_j (p_j - M_j)_- / (1 + max(max_i y_i, max_j (p_j - M_j))),
//              M_j = max_i u_ij y_i
//   r_gap    = max_ij x_ij (p_j - u_ij y_i)_+ / (1 + max(max x, max_ij (p_j - u_ij y_i)_+))
//
// (maxima over the support of U).  Two kernels: a row pass (one warp per row:
// t_i, y_i, the per-entry gap terms, the column maxima M_j and the column sums)
// and a goods pass whose last block (last-block-done ticket, no spin) combines
// every partial into KktOut.  Products and maxima are in FP64 for FP64 markets;
// the MIXED row pass forms t and y in float-float and its maxima in FP32.
#include "common.cuh"

namespace pdhcg {

template <bool MIXED>
__global__ void __launch_bounds__(kThreads) kkt_rows_kernel(DevMarket mk, const void* Xv, const double* __restrict__ p,
                                                            KktBufs kb) {
    extern __shared__ unsigned long long acc_s[];
    if (kb.sel) Xv = (*kb.sel) ? kb.xsel[1] : kb.xsel[0];
    for (int j = threadIdx.x; j < mk.hot; j += blockDim.x) acc_s[j] = 0ull;
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const long long gw = (long long)blockIdx.x * kWarps + (threadIdx.x >> 5);
    const long long nw = (long long)gridDim.x * kWarps;
    double mx = 0.0, mg = 0.0, mxg = 0.0, my = 0.0;
    for (long long i = gw; i < mk.n; i += nw) {
        const long long b = mk.rp[i], e = mk.rp[i + 1];
        double t = 0.0, um = 0.0;
        for (long long q = b + lane; q < e; q += 32) {
            double u = MIXED ? (double)((const float*)mk.uv)[q] : ((const double*)mk.uv)[q];
            double x = MIXED ? (double)((const float*)Xv)[q] : ((const double*)Xv)[q];
            t = fma(u, x, t);
            um = fmax(um, u);
        }
        t = warp_sum_d(t);
        um = warp_max_d(um);
        const double y = mk.w[i] / t;
        if (lane == 0 && kb.t_out) kb.t_out[i] = t;
        my = fmax(my, y * um);         // y of the max-scaled row
        for (long long q = b + lane; q < e; q += 32) {
            const int j = mk.cj[q];
            double u = MIXED ? (double)((const float*)mk.uv)[q] : ((const double*)mk.uv)[q];
            double x = MIXED ? (double)((const float*)Xv)[q] : ((const double*)Xv)[q];
            const double uy = u * y;
            const double g = fmax(p[j] - uy, 0.0);
            mx = fmax(mx, x);
            mg = fmax(mg, g);
            mxg = fmax(mxg, x * g);
            // column maximum of u_ij y_i: read first, update only when larger
            unsigned long long cur = ((volatile unsigned long long*)kb.M)[j];
            if (dbits(uy) > cur) atomicMax(&kb.M[j], dbits(uy));
            if (x > 0.0) {
                if (MIXED) {
                    unsigned long long v = (unsigned long long)__double2ll_rn(x * kFixScale);
                    if (j < mk.hot) shared_add_u64(&acc_s[j], v);
                    else atomicAdd(&kb.acc[j], v);
                } else {
                    if (j < mk.hot) shared_add_f64(&acc_s[j], x);
                    else atomicAdd((double*)&kb.acc[j], x);
                }
            }
        }
    }
    mx = warp_max_d(mx);
    mg = warp_max_d(mg);
    mxg = warp_max_d(mxg);
    my = warp_max_d(my);
    __shared__ KktPart red[kWarps];
    if (lane == 0) red[threadIdx.x >> 5] = KktPart{mx, mg, mxg, my};
    __syncthreads();
    if (threadIdx.x == 0) {
        KktPart r = red[0];
        for (int w = 1; w < kWarps; w++) {
            r.max_x = fmax(r.max_x, red[w].max_x);
            r.max_g = fmax(r.max_g, red[w].max_g);
            r.max_xg = fmax(r.max_xg, red[w].max_xg);
            r.max_y = fmax(r.max_y, red[w].max_y);
        }
        kb.part[blockIdx.x] = r;
    }
    for (int j = threadIdx.x; j < mk.hot; j += blockDim.x) {
        unsigned long long a = acc_s[j];
        if (a) {
            if (MIXED) atomicAdd(&kb.acc[j], a);
            else atomicAdd((double*)&kb.acc[j], __longlong_as_double((long long)a));
        }
    }
}

// MIXED: the same quantities without per-entry FP64.  With y = w / t carried in
// float-float and p as float-float, d_ij = p_j - u_ij y_i is evaluated by the
// cancellation-free FMA form used by the row solver, so the gap terms are
// accurate relative to themselves.  Because p_j - M_j = min_i d_ij, the dual
// residual needs max_ij (-d_ij) (a plain maximum) and, for its denominator, the
// per-good minimum of d (kept as order-preserving integer keys of floats).
__device__ __forceinline__ int fkey(float f) {
    const int b = __float_as_int(f);
    return b >= 0 ? b : b ^ 0x7fffffff;
}
__device__ __forceinline__ float fkey_inv(int k) { return __int_as_float(k >= 0 ? k : k ^ 0x7fffffff); }

__global__ void __launch_bounds__(kThreads) kkt_rows_mixed_kernel(DevMarket mk, const float* Xv, KktBufs kb) {
    extern __shared__ unsigned long long acc_s[];
    int* dmin_s = (int*)(acc_s + mk.hot);
    int* dmin_g = (int*)kb.M;
    if (kb.sel) Xv = (const float*)((*kb.sel) ? kb.xsel[1] : kb.xsel[0]);
    for (int j = threadIdx.x; j < mk.hot; j += blockDim.x) { acc_s[j] = 0ull; dmin_s[j] = 0x7fffffff; }
    __syncthreads();
    const float* U = (const float*)mk.uv;
    const int lane = threadIdx.x & 31;
    const long long gw = (long long)blockIdx.x * kWarps + (threadIdx.x >> 5);
    const long long nw = (long long)gridDim.x * kWarps;
    float mx = 0.0f, mg = 0.0f, mxg = 0.0f, mnd = 0.0f, my = 0.0f;
    // one entry of the second pass: gap terms, column minimum of p_j - u_ij y_i, column sum
    auto entry = [&](int j, float u, float x, float2 p, ff y) {
        const float d = fmaf(-u, y.lo, fmaf(-u, y.hi, p.x) + p.y);   // p_j - u_ij y_i
        const float g = fmaxf(d, 0.0f);
        mx = fmaxf(mx, x);
        mg = fmaxf(mg, g);
        mxg = fmaxf(mxg, x * g);
        mnd = fmaxf(mnd, -d);
        const int key = fkey(d);
        if (j < mk.hot) {
            if (key < dmin_s[j]) shared_min_s32(&dmin_s[j], key);
            if (x > 0.0f) shared_add_u64(&acc_s[j], (unsigned long long)__float2ll_rn(x * kFixScaleF));
        } else {
            if (key < ((volatile int*)dmin_g)[j]) atomicMin(&dmin_g[j], key);
            if (x > 0.0f) atomicAdd(&kb.acc[j], (unsigned long long)__float2ll_rn(x * kFixScaleF));
        }
    };
    for (long long i = gw; i < mk.n; i += nw) {
        const long long b = mk.rp[i], e = mk.rp[i + 1];
        // rows of at most 32 * kSlots entries are read once into registers
        // (lane l holds entries l, l + 32, ...), longer ones are streamed twice;
        // either way a lane visits its entries in increasing order
        const bool reg = e - b <= 32 * kSlots;
        float ru[kSlots], rx[kSlots];
        int rj[kSlots];
        // t = u_i^T x_i in float-float: TwoProduct terms, their high parts
        // summed by TwoSum, every low part added in FP32
        float th = 0.0f, tl = 0.0f;
        float um = 0.0f;
        if (reg) {
#pragma unroll
            for (int k = 0; k < kSlots; k++) {
                const long long q = b + lane + 32 * k;
                const bool in = q < e;
                rj[k] = in ? mk.cj[q] : -1;
                ru[k] = in ? U[q] : 0.0f;
                rx[k] = in ? Xv[q] : 0.0f;
            }
#pragma unroll
            for (int k = 0; k < kSlots; k++) {
                if (rj[k] < 0) continue;
                const ff pr = two_prod(ru[k], rx[k]);
                const ff sm = two_sum(th, pr.hi);
                th = sm.hi;
                tl += sm.lo + pr.lo;
                um = fmaxf(um, ru[k]);
            }
        } else {
            for (long long q = b + lane; q < e; q += 32) {
                const float u = U[q];
                const ff pr = two_prod(u, Xv[q]);
                const ff sm = two_sum(th, pr.hi);
                th = sm.hi;
                tl += sm.lo + pr.lo;
                um = fmaxf(um, u);
            }
        }
        const ff t = group_sum<32>(ff_make(th, tl));
        for (int o = 16; o > 0; o >>= 1) um = fmaxf(um, __shfl_xor_sync(0xffffffffu, um, o));
        // budgets as float-float (no FP64 per row: FP64 is a slow pipe here)
        const ff wi = mk.wff ? ff_make(mk.wff[i].x, mk.wff[i].y) : ff_from_double(mk.w[i]);
        const ff y = ff_div(wi, t);
        if (lane == 0 && kb.t_out) kb.t_out[i] = ff_to_double(t);
        my = fmaxf(my, (y.hi + y.lo) * um);   // y of the max-scaled row
        if (reg) {
            float2 pp[kSlots];
#pragma unroll
            for (int k = 0; k < kSlots; k++) pp[k] = kb.pff[rj[k] >= 0 ? rj[k] : 0];   // gathers issued together
#pragma unroll
            for (int k = 0; k < kSlots; k++)
                if (rj[k] >= 0) entry(rj[k], ru[k], rx[k], pp[k], y);
        } else {
            for (long long q = b + lane; q < e; q += 32) {
                const int j = mk.cj[q];
                entry(j, U[q], Xv[q], kb.pff[j], y);
            }
        }
    }
    for (int o = 16; o > 0; o >>= 1) {
        mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
        mg = fmaxf(mg, __shfl_xor_sync(0xffffffffu, mg, o));
        mxg = fmaxf(mxg, __shfl_xor_sync(0xffffffffu, mxg, o));
        mnd = fmaxf(mnd, __shfl_xor_sync(0xffffffffu, mnd, o));
    }
    for (int o = 16; o > 0; o >>= 1) my = fmaxf(my, __shfl_xor_sync(0xffffffffu, my, o));
    __shared__ KktPart red[kWarps];
    __shared__ float red2[kWarps];
    if (lane == 0) { red[threadIdx.x >> 5] = KktPart{mx, mg, mxg, my}; red2[threadIdx.x >> 5] = mnd; }
    __syncthreads();
    if (threadIdx.x == 0) {
        KktPart r = red[0];
        float nd = red2[0];
        for (int w = 1; w < kWarps; w++) {
            r.max_x = fmax(r.max_x, red[w].max_x);
            r.max_g = fmax(r.max_g, red[w].max_g);
            r.max_xg = fmax(r.max_xg, red[w].max_xg);
            r.max_y = fmax(r.max_y, red[w].max_y);
            nd = fmaxf(nd, red2[w]);
        }
        kb.part[blockIdx.x] = r;
        kb.nd_part[blockIdx.x] = nd;
    }
    for (int j = threadIdx.x; j < mk.hot; j += blockDim.x) {
        const unsigned long long a = acc_s[j];
        if (a) atomicAdd(&kb.acc[j], a);
        const int dk = dmin_s[j];
        if (dk != 0x7fffffff) atomicMin(&dmin_g[j], dk);
    }
}

__global__ void kkt_goods_mixed_kernel(int m, KktBufs kb, int nrow_blocks) {
    int* dmin_g = (int*)kb.M;
    double np = 0.0, mc = 0.0, dd = -INFINITY;
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < m; j += gridDim.x * blockDim.x) {
        const unsigned long long a = kb.acc[j];
        kb.acc[j] = 0ull;
        const double c = (double)(long long)a * kFixInv;
        if (kb.c_out) kb.c_out[j] = c;
        np = fmax(np, fabs(c - 1.0));
        mc = fmax(mc, c);
        dd = fmax(dd, (double)fkey_inv(dmin_g[j]));     // p_j - M_j
        dmin_g[j] = 0x7fffffff;
    }
    np = warp_max_d(np);
    mc = warp_max_d(mc);
    dd = warp_max_d(dd);
    __shared__ double r[32][3];
    __shared__ bool last;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) { r[wid][0] = np; r[wid][1] = mc; r[wid][2] = dd; }
    __syncthreads();
    if (threadIdx.x == 0) {
        double a0 = 0.0, a1 = 0.0, a3 = -INFINITY;
        for (int w = 0; w < (int)(blockDim.x >> 5); w++) { a0 = fmax(a0, r[w][0]); a1 = fmax(a1, r[w][1]); a3 = fmax(a3, r[w][2]); }
        kb.gpart[4 * blockIdx.x + 0] = a0;
        kb.gpart[4 * blockIdx.x + 1] = a1;
        kb.gpart[4 * blockIdx.x + 2] = 0.0;
        kb.gpart[4 * blockIdx.x + 3] = a3;
        __threadfence();
        unsigned int t = atomicAdd(&kb.ctl->ticket2, 1u);
        last = (t == gridDim.x - 1);
    }
    __syncthreads();
    if (!last || threadIdx.x != 0) return;
    __threadfence();
    volatile double* gp = kb.gpart;
    double np_ = 0.0, mc_ = 0.0, dd_ = -INFINITY;
    for (int b = 0; b < (int)gridDim.x; b++) {
        np_ = fmax(np_, gp[4 * b]); mc_ = fmax(mc_, gp[4 * b + 1]); dd_ = fmax(dd_, gp[4 * b + 3]);
    }
    volatile KktPart* rp = kb.part;
    volatile float* ndp = kb.nd_part;
    double mx = 0.0, mg = 0.0, mxg = 0.0, my = 0.0, nd = 0.0;
    for (int b = 0; b < nrow_blocks; b++) {
        mx = fmax(mx, rp[b].max_x); mg = fmax(mg, rp[b].max_g);
        mxg = fmax(mxg, rp[b].max_xg); my = fmax(my, rp[b].max_y);
        nd = fmax(nd, (double)ndp[b]);
    }
    KktOut o;
    o.r_primal = np_ / (1.0 + fmax(mc_, 1.0));
    o.r_dual = nd / (1.0 + fmax(my, dd_));
    o.r_gap = mxg / (1.0 + fmax(mx, mg));
    o.kkt = fmax(o.r_primal, fmax(o.r_dual, o.r_gap));
    if (!(o.kkt == o.kkt)) o.kkt = INFINITY;
    *kb.out = o;
    kb.ctl->ticket2 = 0u;
}

template <bool MIXED>
__global__ void kkt_goods_kernel(int m, const double* __restrict__ p, KktBufs kb, int nrow_blocks) {
    double np = 0.0, mc = 0.0, nd = 0.0, dd = -INFINITY;
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < m; j += gridDim.x * blockDim.x) {
        unsigned long long a = kb.acc[j];
        kb.acc[j] = 0ull;
        const double c = MIXED ? (double)(long long)a * kFixInv : __longlong_as_double((long long)a);
        if (kb.c_out) kb.c_out[j] = c;
        const double Mj = __longlong_as_double((long long)kb.M[j]);
        kb.M[j] = 0ull;
        np = fmax(np, fabs(c - 1.0));
        mc = fmax(mc, c);
        const double d = p[j] - Mj;
        nd = fmax(nd, fmax(-d, 0.0));
        dd = fmax(dd, d);
    }
    np = warp_max_d(np);
    mc = warp_max_d(mc);
    nd = warp_max_d(nd);
    dd = warp_max_d(dd);
    __shared__ double r[32][4];
    __shared__ bool last;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) { r[wid][0] = np; r[wid][1] = mc; r[wid][2] = nd; r[wid][3] = dd; }
    __syncthreads();
    if (threadIdx.x == 0) {
        double a0 = 0.0, a1 = 0.0, a2 = 0.0, a3 = -INFINITY;
        for (int w = 0; w < (int)(blockDim.x >> 5); w++) {
            a0 = fmax(a0, r[w][0]); a1 = fmax(a1, r[w][1]); a2 = fmax(a2, r[w][2]); a3 = fmax(a3, r[w][3]);
        }
        kb.gpart[4 * blockIdx.x + 0] = a0;
        kb.gpart[4 * blockIdx.x + 1] = a1;
        kb.gpart[4 * blockIdx.x + 2] = a2;
        kb.gpart[4 * blockIdx.x + 3] = a3;
        __threadfence();
        unsigned int t = atomicAdd(&kb.ctl->ticket2, 1u);
        last = (t == gridDim.x - 1);
    }
    __syncthreads();
    if (!last || threadIdx.x != 0) return;
    __threadfence();
    volatile double* gp = kb.gpart;
    double np_ = 0.0, mc_ = 0.0, nd_ = 0.0, dd_ = -INFINITY;
    for (int b = 0; b < (int)gridDim.x; b++) {
        np_ = fmax(np_, gp[4 * b]); mc_ = fmax(mc_, gp[4 * b + 1]);
        nd_ = fmax(nd_, gp[4 * b + 2]); dd_ = fmax(dd_, gp[4 * b + 3]);
    }
    volatile KktPart* rp = kb.part;
    double mx = 0.0, mg = 0.0, mxg = 0.0, my = 0.0;
    for (int b = 0; b < nrow_blocks; b++) {
        mx = fmax(mx, rp[b].max_x); mg = fmax(mg, rp[b].max_g);
        mxg = fmax(mxg, rp[b].max_xg); my = fmax(my, rp[b].max_y);
    }
    KktOut o;
    o.r_primal = np_ / (1.0 + fmax(mc_, 1.0));
    o.r_dual = nd_ / (1.0 + fmax(my, dd_));
    o.r_gap = mxg / (1.0 + fmax(mx, mg));
    o.kkt = fmax(o.r_primal, fmax(o.r_dual, o.r_gap));
    if (!(o.kkt == o.kkt)) o.kkt = INFINITY;
    *kb.out = o;
    kb.ctl->ticket2 = 0u;
}

static int g_kkt_blocks = 0;
int kkt_blocks() {
    if (!g_kkt_blocks) {
        int dev = 0, sm = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sm, cudaDevAttrMultiProcessorCount, dev);
        g_kkt_blocks = sm * 3;
    }
    return g_kkt_blocks;
}
static const int kGoodsBlocks = 64;

void launch_kkt(bool mixed, const DevMarket& mk, const void* x, const double* p, const KktBufs& kb, cudaStream_t s) {
    static bool attr = false;
    if (!attr) {
        attr = true;
        cudaFuncSetAttribute(kkt_rows_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
        cudaFuncSetAttribute(kkt_rows_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
        cudaFuncSetAttribute(kkt_rows_mixed_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    }
    size_t smem = (size_t)mk.hot * sizeof(unsigned long long);
    if (mixed) {
        kkt_rows_mixed_kernel<<<kkt_blocks(), kThreads, smem + (size_t)mk.hot * sizeof(int), s>>>(
            mk, (const float*)x, kb);
        kkt_goods_mixed_kernel<<<kGoodsBlocks, 256, 0, s>>>(mk.m, kb, kkt_blocks());
    } else {
        kkt_rows_kernel<false><<<kkt_blocks(), kThreads, smem, s>>>(mk, x, p, kb);
        kkt_goods_kernel<false><<<kGoodsBlocks, 256, 0, s>>>(mk.m, p, kb, kkt_blocks());
    }
}

}  // namespace pdhcg
