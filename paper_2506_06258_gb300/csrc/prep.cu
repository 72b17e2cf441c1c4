// Preprocessing and helper kernels:
//   - validation of the CSR market (Assumption 1: no empty row or column;
//     u > 0 finite; w > 0 finite; strictly increasing columns within a row),
//   - row scaling u_ij / max_j u_ij (Section 5, "Preprocessing"),
//   - column degrees and relabelling of goods by decreasing degree,
//   - the initial point x_ij = 1/deg_j (which clears the market),
//   - restart helpers (copies, squared distances) and output gathers.
#include "common.cuh"
#include "prep.cuh"

namespace pdhcg {

__global__ void validate_kernel(int n, int m, long long nnz, const long long* __restrict__ rp,
                                const int* __restrict__ col, const void* val, int val_f32,
                                const double* __restrict__ w, unsigned int* err) {
    const int lane = threadIdx.x & 31;
    const long long gw = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
    const long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
    unsigned int e = 0;
    if (gw == 0 && lane == 0 && (rp[0] != 0 || rp[n] != nnz)) e |= ERR_ROWPTR;
    for (long long i = gw; i < n; i += nw) {
        const long long b = rp[i], en = rp[i + 1];
        if (lane == 0) {
            const double wi = w[i];
            if (!(wi > 0.0) || !isfinite(wi)) e |= ERR_BUDGET;
        }
        if (en < b || b < 0 || en > nnz) { e |= ERR_ROWPTR; continue; }
        if (en == b) { e |= ERR_EMPTY_ROW; continue; }
        for (long long q = b + lane; q < en; q += 32) {
            const int j = col[q];
            if (j < 0 || j >= m) e |= ERR_COL_RANGE;
            if (q > b && col[q - 1] >= j) e |= ERR_COL_ORDER;
            const double u = val_f32 ? (double)((const float*)val)[q] : ((const double*)val)[q];
            if (!(u > 0.0) || !isfinite(u)) e |= ERR_UTIL;
        }
    }
    if (e) atomicOr(err, e);
}

__global__ void col_degree_kernel(long long nnz, const int* __restrict__ col, int m, int* deg) {
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < nnz; q += (long long)gridDim.x * blockDim.x) {
        const int j = col[q];
        if (j >= 0 && j < m) atomicAdd(&deg[j], 1);
    }
}

// row scale (row_scale), scaled utilities, relabelled goods, initial x; caller
// row i is written as internal row inv[i], whose entries start at irp[inv[i]]
template <typename V>
__global__ void scale_kernel(int n, const long long* __restrict__ rp, const int* __restrict__ col, const void* val,
                             int val_f32, const int* __restrict__ rank, const int* __restrict__ deg,
                             const int* __restrict__ inv, const long long* __restrict__ irp,
                             double* __restrict__ rowmax, V* __restrict__ uv, int* __restrict__ cj,
                             V* __restrict__ x0, int init_x) {
    const int lane = threadIdx.x & 31;
    const long long gw = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
    const long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
    for (long long i = gw; i < n; i += nw) {
        const long long b = rp[i], e = rp[i + 1];
        const int r = inv[i];
        const long long ib = irp[r] - b;       // internal index = caller index + ib
        double mx = 0.0;
        for (long long q = b + lane; q < e; q += 32) {
            const double u = val_f32 ? (double)((const float*)val)[q] : ((const double*)val)[q];
            mx = fmax(mx, u);
        }
        mx = row_scale<V>(warp_max_d(mx));
        if (lane == 0) rowmax[r] = mx;
        for (long long q = b + lane; q < e; q += 32) {
            const double u = val_f32 ? (double)((const float*)val)[q] : ((const double*)val)[q];
            uv[q + ib] = (V)(u / mx);
            const int j = col[q];
            cj[q + ib] = rank[j];
            if (init_x) x0[q + ib] = (V)(1.0 / (double)deg[j]);
        }
    }
}

// internal row r <-> caller row perm[r]: dst[perm[r]] = src[r] (times mul[r])
__global__ void rows_to_caller_kernel(int n, const int* __restrict__ perm, const double* __restrict__ src,
                                      const double* __restrict__ mul, double* __restrict__ dst) {
    for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < n; r += gridDim.x * blockDim.x)
        dst[perm[r]] = mul ? src[r] * mul[r] : src[r];
}
__global__ void rows_to_internal_kernel(int n, const int* __restrict__ perm, const double* __restrict__ src,
                                        double* __restrict__ dst) {
    for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < n; r += gridDim.x * blockDim.x) dst[r] = src[perm[r]];
}
// per-entry arrays: internal row r holds entries [irp[r], irp[r+1]), the same
// entries as caller row perm[r] from crp[perm[r]] on, in the same order
template <typename V>
__global__ void entries_kernel(int n, const int* __restrict__ perm, const long long* __restrict__ crp,
                               const long long* __restrict__ irp, const V* __restrict__ src, V* __restrict__ dst,
                               int to_caller) {
    const int lane = threadIdx.x & 31;
    const long long gw = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
    const long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
    for (long long r = gw; r < n; r += nw) {
        const long long ib = irp[r], d = irp[r + 1] - ib;
        const long long cb = crp[perm[r]];
        for (long long k = lane; k < d; k += 32) {
            if (to_caller) dst[cb + k] = src[ib + k];
            else dst[ib + k] = src[cb + k];
        }
    }
}

__global__ void fill_kernel(double* a, long long n, double v) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) a[i] = v;
}

// internal (relabelled) <-> caller good order
__global__ void gather_goods_kernel(int m, const int* __restrict__ rank, const double* __restrict__ src_int,
                                    double* __restrict__ dst_orig) {
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < m; j += gridDim.x * blockDim.x) dst_orig[j] = src_int[rank[j]];
}
__global__ void scatter_goods_kernel(int m, const int* __restrict__ rank, const double* __restrict__ src_orig,
                                     double* __restrict__ dst_int) {
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < m; j += gridDim.x * blockDim.x) dst_int[rank[j]] = src_orig[j];
}
template <typename Vs, typename Vd>
__global__ void convert_kernel(long long n, const Vs* __restrict__ s, Vd* __restrict__ d) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) d[i] = (Vd)s[i];
}

// squared distance ||a - r||^2 accumulated in FP64 per block, then r <- a
template <typename V>
__global__ void dist_copy_kernel(long long n, const V* __restrict__ a, V* __restrict__ r, double* part) {
    double s = 0.0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const double d = (double)a[i] - (double)r[i];
        s = fma(d, d, s);
        r[i] = a[i];
    }
    s = warp_sum_d(s);
    __shared__ double red[32];
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); w++) t += red[w];
        part[blockIdx.x] = t;
    }
}

static int grid_for(long long n, int per = 256, int cap = 4096) {
    long long b = (n + per - 1) / per;
    if (b < 1) b = 1;
    if (b > cap) b = cap;
    return (int)b;
}

void k_validate(int n, int m, long long nnz, const long long* rp, const int* col, const void* val, int f32,
                const double* w, unsigned int* err, cudaStream_t s) {
    validate_kernel<<<grid_for((long long)n * 32, 256, 8192), 256, 0, s>>>(n, m, nnz, rp, col, val, f32, w, err);
}
void k_col_degree(long long nnz, const int* col, int m, int* deg, cudaStream_t s) {
    col_degree_kernel<<<grid_for(nnz), 256, 0, s>>>(nnz, col, m, deg);
}
void k_scale(bool mixed, int n, const long long* rp, const int* col, const void* val, int f32, const int* rank,
             const int* deg, const int* inv, const long long* irp, double* rowmax, void* uv, int* cj, void* x0,
             int init_x, cudaStream_t s) {
    int g = grid_for((long long)n * 32, 256, 8192);
    if (mixed)
        scale_kernel<float><<<g, 256, 0, s>>>(n, rp, col, val, f32, rank, deg, inv, irp, rowmax, (float*)uv, cj,
                                              (float*)x0, init_x);
    else
        scale_kernel<double><<<g, 256, 0, s>>>(n, rp, col, val, f32, rank, deg, inv, irp, rowmax, (double*)uv, cj,
                                               (double*)x0, init_x);
}
void k_rows_to_caller(int n, const int* perm, const double* src, const double* mul, double* dst, cudaStream_t s) {
    rows_to_caller_kernel<<<grid_for(n), 256, 0, s>>>(n, perm, src, mul, dst);
}
void k_rows_to_internal(int n, const int* perm, const double* src, double* dst, cudaStream_t s) {
    rows_to_internal_kernel<<<grid_for(n), 256, 0, s>>>(n, perm, src, dst);
}
void k_entries(int n, const int* perm, const long long* crp, const long long* irp, const void* src, void* dst,
               int bytes, bool to_caller, cudaStream_t s) {
    int g = grid_for((long long)n * 32, 256, 8192);
    if (bytes == 4)
        entries_kernel<float><<<g, 256, 0, s>>>(n, perm, crp, irp, (const float*)src, (float*)dst, to_caller ? 1 : 0);
    else
        entries_kernel<double><<<g, 256, 0, s>>>(n, perm, crp, irp, (const double*)src, (double*)dst, to_caller ? 1 : 0);
}
__global__ void w_to_ff_kernel(int n, const double* __restrict__ w, float2* __restrict__ wff) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const double v = w[i];
        const float h = (float)v;
        wff[i] = make_float2(h, (float)(v - (double)h));
    }
}
__global__ void t_to_y_kernel(int n, const double* __restrict__ w, const double* t, float2* y) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const double tv = t[i];
        const double v = (tv > 0.0 && tv < 1e300) ? w[i] / tv : 1.0;
        const float h = (float)v;
        y[i] = make_float2(h, (float)(v - (double)h));
    }
}
__global__ void y_to_t_kernel(int n, const double* __restrict__ w, const float2* y, double* t) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const float2 v = y[i];
        t[i] = w[i] / ((double)v.x + (double)v.y);
    }
}
__global__ void fill_ff_kernel(int n, float2* a, float v) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) a[i] = make_float2(v, 0.0f);
}
void k_w_to_ff(int n, const double* w, float2* wff, cudaStream_t s) {
    w_to_ff_kernel<<<grid_for(n), 256, 0, s>>>(n, w, wff);
}
void k_t_to_y(int n, const double* w, const double* t, float2* y, cudaStream_t s) {
    t_to_y_kernel<<<grid_for(n), 256, 0, s>>>(n, w, t, y);
}
void k_y_to_t(int n, const double* w, const float2* y, double* t, cudaStream_t s) {
    y_to_t_kernel<<<grid_for(n), 256, 0, s>>>(n, w, y, t);
}
void k_fill_ff(int n, float2* a, float v, cudaStream_t s) { fill_ff_kernel<<<grid_for(n), 256, 0, s>>>(n, a, v); }
void k_fill(double* a, long long n, double v, cudaStream_t s) { fill_kernel<<<grid_for(n), 256, 0, s>>>(a, n, v); }
void k_gather_goods(int m, const int* rank, const double* src_int, double* dst, cudaStream_t s) {
    gather_goods_kernel<<<grid_for(m), 256, 0, s>>>(m, rank, src_int, dst);
}
void k_scatter_goods(int m, const int* rank, const double* src, double* dst_int, cudaStream_t s) {
    scatter_goods_kernel<<<grid_for(m), 256, 0, s>>>(m, rank, src, dst_int);
}
// FP32 rows are scaled by a power of two (row_scale); t of the max-scaled row
// is t / max_j u_ij of the stored row.
__global__ void max_scaled_t_kernel(int n, const long long* __restrict__ rp, const float* __restrict__ uv,
                                    const double* __restrict__ t, double* __restrict__ out) {
    const int lane = threadIdx.x & 31;
    const long long gw = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
    const long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
    for (long long i = gw; i < n; i += nw) {
        float um = 0.0f;
        for (long long q = rp[i] + lane; q < rp[i + 1]; q += 32) um = fmaxf(um, uv[q]);
        for (int o = 16; o > 0; o >>= 1) um = fmaxf(um, __shfl_xor_sync(0xffffffffu, um, o));
        if (lane == 0) out[i] = t[i] / (double)um;
    }
}

void k_max_scaled_t(int n, const long long* rp, const float* uv, const double* t, double* out, cudaStream_t s) {
    max_scaled_t_kernel<<<grid_for((long long)n * 32), 256, 0, s>>>(n, rp, uv, t, out);
}

void k_convert(long long n, const void* src, bool src_f32, void* dst, bool dst_f32, cudaStream_t s) {
    int g = grid_for(n);
    if (src_f32 && dst_f32) cudaMemcpyAsync(dst, src, n * 4, cudaMemcpyDeviceToDevice, s);
    else if (!src_f32 && !dst_f32) cudaMemcpyAsync(dst, src, n * 8, cudaMemcpyDeviceToDevice, s);
    else if (src_f32) convert_kernel<float, double><<<g, 256, 0, s>>>(n, (const float*)src, (double*)dst);
    else convert_kernel<double, float><<<g, 256, 0, s>>>(n, (const double*)src, (float*)dst);
}
int dist_blocks() { return 1024; }
void k_dist_copy(bool f32, long long n, const void* a, void* r, double* part, cudaStream_t s) {
    if (f32) dist_copy_kernel<float><<<dist_blocks(), 256, 0, s>>>(n, (const float*)a, (float*)r, part);
    else dist_copy_kernel<double><<<dist_blocks(), 256, 0, s>>>(n, (const double*)a, (double*)r, part);
}

}  // namespace pdhcg
