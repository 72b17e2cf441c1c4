// Launchers of the preprocessing and helper kernels (prep.cu).
#pragma once
#include <cuda_runtime.h>

namespace pdhcg {

enum : unsigned int {
    ERR_ROWPTR = 1u, ERR_EMPTY_ROW = 2u, ERR_COL_RANGE = 4u, ERR_COL_ORDER = 8u,
    ERR_UTIL = 16u, ERR_BUDGET = 32u, ERR_EMPTY_COL = 64u
};

void k_validate(int n, int m, long long nnz, const long long* rp, const int* col, const void* val, int f32,
                const double* w, unsigned int* err, cudaStream_t s);
void k_col_degree(long long nnz, const int* col, int m, int* deg, cudaStream_t s);
void k_scale(bool mixed, int n, const long long* rp, const int* col, const void* val, int f32, const int* rank,
             const int* deg, double* rowmax, void* uv, int* cj, void* x0, int init_x, cudaStream_t s);
void k_fill(double* a, long long n, double v, cudaStream_t s);
void k_gather_goods(int m, const int* rank, const double* src_int, double* dst, cudaStream_t s);
void k_scatter_goods(int m, const int* rank, const double* src, double* dst_int, cudaStream_t s);
void k_util_out(int n, const double* t, const double* rowmax, double* out, cudaStream_t s);
void k_max_scaled_t(int n, const long long* rp, const float* uv, const double* t, double* out, cudaStream_t s);
void k_convert(long long n, const void* src, bool src_f32, void* dst, bool dst_f32, cudaStream_t s);
int dist_blocks();
void k_dist_copy(bool f32, long long n, const void* a, void* r, double* part, cudaStream_t s);

}  // namespace pdhcg
