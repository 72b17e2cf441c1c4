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
             const int* deg, const int* inv, const long long* irp, double* rowmax, void* uv, int* cj, void* x0,
             int init_x, cudaStream_t s);
// The preprocessed market stores its rows bucket by bucket: internal row r is
// caller row perm[r].  Conversions between the two orders, per row (doubles;
// with mul, dst[perm[r]] = src[r] * mul[r]) and per entry (4- or 8-byte values).
void k_rows_to_caller(int n, const int* perm, const double* src, const double* mul, double* dst, cudaStream_t s);
void k_rows_to_internal(int n, const int* perm, const double* src, double* dst, cudaStream_t s);
void k_entries(int n, const int* perm, const long long* crp, const long long* irp, const void* src, void* dst,
               int bytes, bool to_caller, cudaStream_t s);
void k_fill(double* a, long long n, double v, cudaStream_t s);
void k_gather_goods(int m, const int* rank, const double* src_int, double* dst, cudaStream_t s);
void k_scatter_goods(int m, const int* rank, const double* src, double* dst_int, cudaStream_t s);
void k_max_scaled_t(int n, const long long* rp, const float* uv, const double* t, double* out, cudaStream_t s);
void k_convert(long long n, const void* src, bool src_f32, void* dst, bool dst_f32, cudaStream_t s);
// MIXED row state: budgets as float-float, and y = w / t (the warm start of
// the row kernel, float-float) from utilities t; y_to_t converts in place back
// to t = w / y in FP64 (the two arrays may alias: same index, same 8 bytes).
void k_w_to_ff(int n, const double* w, float2* wff, cudaStream_t s);
void k_t_to_y(int n, const double* w, const double* t, float2* y, cudaStream_t s);
void k_y_to_t(int n, const double* w, const float2* y, double* t, cudaStream_t s);
void k_fill_ff(int n, float2* a, float v, cudaStream_t s);
int dist_blocks();
void k_dist_copy(bool f32, long long n, const void* a, void* r, double* part, cudaStream_t s);

}  // namespace pdhcg
