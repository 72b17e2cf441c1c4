// pdhcg_kkt_noalloc: the relative KKT error of Section 5 for a caller's point,
// computed without allocating any memory.
//
// Why it exists: some callers cannot allocate device memory at the moment they
// need the residual -- code running inside a memory pool or allocator callback,
// a process whose device memory is fully reserved by another framework, or a
// real-time loop that forbids allocation after start-up.  pdhcg_kkt works through
// a handle whose workspace grows with cudaMalloc; this entry point instead keeps
// all of its scratch in one file-scope device array of fixed size, so a call
// performs no cudaMalloc, cudaFree or allocating library routine.
//
// Scratch (kNaMaxGoods goods at most):
//   column sums      FP64   [kNaMaxGoods]
//   column maxima    double bits of max_i u_ij y_i  [kNaMaxGoods]
//   block partials   KKT maxima of each row block, then of each goods block
//   control          last-block ticket, error flag, result
// Every call clears the parts that must start at zero, so each call starts from
// a clean state; the array is shared by all calls, so calls that overlap on the
// GPU (two streams, or two host threads) race and must be serialised by the
// caller.  The device address of the array is looked up once per device with
// cudaGetSymbolAddress on the first call made with that device current; that
// first call should come before any stream capture.
#include <cstring>
#include <mutex>

#include "common.cuh"

namespace {

constexpr int kNaMaxGoods = 262144;      // 2 x 2 MiB of per-good scratch
constexpr int kNaRowBlocks = 456;
constexpr int kNaGoodBlocks = 64;
constexpr int kNaThreads = 256;

struct NaCtl {
    unsigned int ticket;
    unsigned int error;
    double out[4];
};

struct NaScratch {
    double colsum[kNaMaxGoods];
    unsigned long long colmax[kNaMaxGoods];
    double rowpart[kNaRowBlocks][4];
    double goodpart[kNaGoodBlocks][4];
    NaCtl ctl;
};

static __device__ __align__(256) NaScratch g_na_scratch;

__global__ void na_clear_kernel(NaScratch* S, int m) {
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < m; j += gridDim.x * blockDim.x) {
        S->colsum[j] = 0.0;
        S->colmax[j] = 0ull;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        S->ctl.ticket = 0u;
        S->ctl.error = 0u;
        // NaN until the goods pass writes the result: a pass that never ran
        // cannot be mistaken for a converged point
        for (int k = 0; k < 4; k++) S->ctl.out[k] = __longlong_as_double(0x7ff8000000000000ll);
    }
}

// one warp per buyer: row scaling (Section 5), t_i = u_i^T x_i, y_i = w_i / t_i,
// and the per-entry terms; indices are bounds-checked (a bad index sets the error
// flag and is skipped, so a malformed market cannot write outside the scratch)
__global__ void __launch_bounds__(kNaThreads) na_rows_kernel(int n, int m, long long nnz, const long long* rp,
                                                            const int* col, const void* val, int f32,
                                                            const double* w, const double* x, const double* p,
                                                            NaScratch* S) {
    const int lane = threadIdx.x & 31;
    const long long gw = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
    const long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
    double mx = 0.0, mg = 0.0, mxg = 0.0, my = 0.0;
    for (long long i = gw; i < n; i += nw) {
        long long b = rp[i], e = rp[i + 1];
        if (b < 0 || e > nnz || e <= b) {
            if (lane == 0) atomicOr(&S->ctl.error, 1u);
            continue;
        }
        double rmax = 0.0;
        for (long long q = b + lane; q < e; q += 32)
            rmax = fmax(rmax, f32 ? (double)((const float*)val)[q] : ((const double*)val)[q]);
        rmax = pdhcg::warp_max_d(rmax);
        double t = 0.0;
        for (long long q = b + lane; q < e; q += 32) {
            const double u = (f32 ? (double)((const float*)val)[q] : ((const double*)val)[q]) / rmax;
            t = fma(u, x[q], t);
        }
        t = pdhcg::warp_sum_d(t);
        const double y = w[i] / t;
        my = fmax(my, y);
        for (long long q = b + lane; q < e; q += 32) {
            const int j = col[q];
            if (j < 0 || j >= m) {
                atomicOr(&S->ctl.error, 2u);
                continue;
            }
            const double u = (f32 ? (double)((const float*)val)[q] : ((const double*)val)[q]) / rmax;
            const double xq = x[q];
            const double uy = u * y;
            const double g = fmax(p[j] - uy, 0.0);
            mx = fmax(mx, xq);
            mg = fmax(mg, g);
            mxg = fmax(mxg, xq * g);
            const unsigned long long bits = (unsigned long long)__double_as_longlong(uy);
            if (uy > 0.0 && bits > ((volatile unsigned long long*)S->colmax)[j]) atomicMax(&S->colmax[j], bits);
            if (xq > 0.0) atomicAdd(&S->colsum[j], xq);
        }
    }
    mx = pdhcg::warp_max_d(mx);
    mg = pdhcg::warp_max_d(mg);
    mxg = pdhcg::warp_max_d(mxg);
    my = pdhcg::warp_max_d(my);
    __shared__ double red[kNaThreads / 32][4];
    if (lane == 0) {
        red[threadIdx.x >> 5][0] = mx;
        red[threadIdx.x >> 5][1] = mg;
        red[threadIdx.x >> 5][2] = mxg;
        red[threadIdx.x >> 5][3] = my;
    }
    __syncthreads();
    if (threadIdx.x < 4) {
        double v = 0.0;
        for (int k = 0; k < kNaThreads / 32; k++) v = fmax(v, red[k][threadIdx.x]);
        S->rowpart[blockIdx.x][threadIdx.x] = v;
    }
}

__global__ void __launch_bounds__(kNaThreads) na_goods_kernel(int m, const double* p, NaScratch* S) {
    double np = 0.0, mc = 0.0, nd = 0.0, dd = -INFINITY;
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < m; j += gridDim.x * blockDim.x) {
        const double c = S->colsum[j];
        const double Mj = __longlong_as_double((long long)S->colmax[j]);
        np = fmax(np, fabs(c - 1.0));
        mc = fmax(mc, c);
        const double d = p[j] - Mj;
        nd = fmax(nd, fmax(-d, 0.0));
        dd = fmax(dd, d);
    }
    np = pdhcg::warp_max_d(np);
    mc = pdhcg::warp_max_d(mc);
    nd = pdhcg::warp_max_d(nd);
    dd = pdhcg::warp_max_d(dd);
    __shared__ double red[kNaThreads / 32][4];
    __shared__ bool last;
    const int lane = threadIdx.x & 31;
    if (lane == 0) {
        red[threadIdx.x >> 5][0] = np;
        red[threadIdx.x >> 5][1] = mc;
        red[threadIdx.x >> 5][2] = nd;
        red[threadIdx.x >> 5][3] = dd;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double a0 = 0.0, a1 = 0.0, a2 = 0.0, a3 = -INFINITY;
        for (int k = 0; k < kNaThreads / 32; k++) {
            a0 = fmax(a0, red[k][0]);
            a1 = fmax(a1, red[k][1]);
            a2 = fmax(a2, red[k][2]);
            a3 = fmax(a3, red[k][3]);
        }
        S->goodpart[blockIdx.x][0] = a0;
        S->goodpart[blockIdx.x][1] = a1;
        S->goodpart[blockIdx.x][2] = a2;
        S->goodpart[blockIdx.x][3] = a3;
        __threadfence();
        last = atomicAdd(&S->ctl.ticket, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!last || threadIdx.x != 0) return;
    __threadfence();
    volatile double* gp = &S->goodpart[0][0];
    volatile double* rp = &S->rowpart[0][0];
    double np_ = 0.0, mc_ = 0.0, nd_ = 0.0, dd_ = -INFINITY;
    for (int b = 0; b < (int)gridDim.x; b++) {
        np_ = fmax(np_, gp[4 * b]);
        mc_ = fmax(mc_, gp[4 * b + 1]);
        nd_ = fmax(nd_, gp[4 * b + 2]);
        dd_ = fmax(dd_, gp[4 * b + 3]);
    }
    double mx = 0.0, mg = 0.0, mxg = 0.0, my = 0.0;
    for (int b = 0; b < kNaRowBlocks; b++) {
        mx = fmax(mx, rp[4 * b]);
        mg = fmax(mg, rp[4 * b + 1]);
        mxg = fmax(mxg, rp[4 * b + 2]);
        my = fmax(my, rp[4 * b + 3]);
    }
    double o0 = np_ / (1.0 + fmax(mc_, 1.0));
    double o1 = nd_ / (1.0 + fmax(my, dd_));
    double o2 = mxg / (1.0 + fmax(mx, mg));
    double o3 = fmax(o0, fmax(o1, o2));
    if (!(o3 == o3)) o3 = INFINITY;
    S->ctl.out[0] = o0;
    S->ctl.out[1] = o1;
    S->ctl.out[2] = o2;
    S->ctl.out[3] = o3;
}

// device address of the scratch array, looked up once per device
std::mutex g_na_mutex;
NaScratch* g_na_ptr[64] = {};

NaScratch* na_scratch_for_current_device(cudaError_t* err) {
    int dev = 0;
    *err = cudaGetDevice(&dev);
    if (*err != cudaSuccess || dev < 0 || dev >= 64) return nullptr;
    std::lock_guard<std::mutex> lock(g_na_mutex);
    if (!g_na_ptr[dev]) {
        void* ptr = nullptr;
        *err = cudaGetSymbolAddress(&ptr, g_na_scratch);
        if (*err != cudaSuccess) return nullptr;
        g_na_ptr[dev] = (NaScratch*)ptr;
    }
    return g_na_ptr[dev];
}

bool is_device(const void* p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

}  // namespace

pdhcg_status pdhcg_kkt_noalloc(const pdhcg_market* mk, const double* x, const double* p, double* out,
                               void* stream) {
    if (!mk || !x || !p || !out || !mk->row_ptr || !mk->col || !mk->val || !mk->w) return PDHCG_ERR_INVALID;
    if (mk->n <= 0 || mk->m <= 0 || mk->nnz <= 0 || mk->m > kNaMaxGoods) return PDHCG_ERR_INVALID;
    if (!is_device(mk->row_ptr) || !is_device(mk->col) || !is_device(mk->val) || !is_device(mk->w) ||
        !is_device(x) || !is_device(p))
        return PDHCG_ERR_INVALID;
    cudaError_t err = cudaSuccess;
    NaScratch* S = na_scratch_for_current_device(&err);
    if (!S) return PDHCG_ERR_CUDA;
    cudaStream_t s = (cudaStream_t)stream;
    // every call ends with a blocking copy and a stream synchronisation, which a
    // capturing stream does not allow
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &cap) != cudaSuccess) {
        cudaGetLastError();
        return PDHCG_ERR_CUDA;
    }
    if (cap != cudaStreamCaptureStatusNone) return PDHCG_ERR_INVALID;
    const int m = mk->m, n = mk->n;
    na_clear_kernel<<<(m + 255) / 256 < 1024 ? (m + 255) / 256 : 1024, 256, 0, s>>>(S, m);
    na_rows_kernel<<<kNaRowBlocks, kNaThreads, 0, s>>>(n, m, mk->nnz, (const long long*)mk->row_ptr, mk->col,
                                                       mk->val, mk->val_type == PDHCG_VAL_F32 ? 1 : 0, mk->w, x,
                                                       p, S);
    na_goods_kernel<<<kNaGoodBlocks, kNaThreads, 0, s>>>(m, p, S);
    err = cudaGetLastError();
    if (err != cudaSuccess) return PDHCG_ERR_CUDA;
    NaCtl ctl;
    err = cudaMemcpyAsync(&ctl, &S->ctl, sizeof(NaCtl), cudaMemcpyDeviceToHost, s);
    if (err == cudaSuccess) err = cudaStreamSynchronize(s);
    if (err != cudaSuccess) return PDHCG_ERR_CUDA;
    if (ctl.error) return PDHCG_ERR_INVALID;
    if (ctl.out[3] != ctl.out[3]) return PDHCG_ERR_CUDA;     // the goods pass did not run
    if (is_device(out)) {
        err = cudaMemcpyAsync(out, S->ctl.out, 4 * sizeof(double), cudaMemcpyDeviceToDevice, s);
        if (err == cudaSuccess) err = cudaStreamSynchronize(s);
        if (err != cudaSuccess) return PDHCG_ERR_CUDA;
    } else {
        memcpy(out, ctl.out, 4 * sizeof(double));
    }
    return PDHCG_OK;
}
