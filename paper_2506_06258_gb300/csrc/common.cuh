// Internal declarations shared by the libpdhcg translation units.
//
// Data layout in HBM (one market, n buyers, m goods, nnz utilities):
//   rp[n+1]  int64   row pointers (copy of the caller's)
//   cj[nnz]  int32   good id of each entry, RELABELLED by decreasing column
//                    degree (rank 0 = most popular good) so that the hot goods
//                    are ids [0, H) and their column sums live in shared memory
//   uv[nnz]  V       row-scaled utilities u_ij / max_j u_ij (Section 5)
//   X0,X1    V       x^k and x^{k+1} (ping-pong, roles in Ctl::cur)
//   Xb       V       running average x-bar (Alg. 2)
//   Xr       V       x at the last restart (primal-weight update)
// with V = float (MIXED) or double (FP64).  Per-good vectors are double and sit
// in L2 (m * 8 B each).  Column sums are accumulated exactly as 64-bit fixed
// point (MIXED) or as FP64 atomics (FP64).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>
#include <stdio.h>
#include "../../include/pdhcg.h"

namespace pdhcg {

// ---------------------------------------------------------------------------
// constants
// ---------------------------------------------------------------------------
constexpr double kFixScale = 1099511627776.0;          // 2^40
constexpr double kFixInv = 1.0 / 1099511627776.0;
constexpr float kFixScaleF = 1099511627776.0f;
constexpr int kWarps = 8;                               // warps per block of the row kernels
constexpr int kThreads = kWarps * 32;
// the persistent row kernel: one block of 24 warps per SM (80 registers a
// thread, one shared copy of the hot goods per SM)
constexpr int kProxWarps = 24;
constexpr int kProxThreads = kProxWarps * 32;
constexpr int kMaxBuckets = 8;
constexpr int kSlots = 4;                               // entries per lane held in registers
constexpr int kPadEntries = 16;                         // slack after the nnz arrays

// ---------------------------------------------------------------------------
// iteration control block (device resident; one per solve)
// ---------------------------------------------------------------------------
struct Ctl {
    // step control (Section 5: tau = eta/omega, sigma = eta*omega)
    double eta, omega, eta0, eta_min, eta_max_abs;
    double tau, sigma;
    double sum_eta;        // sum of step sizes since the last restart (average weights)
    double fold_wgt;       // weight with which x^k is folded into the average
    double eta_used;       // step size of the last accepted pass
    int fold_pending;      // the last pass was accepted: fold x^k, commit p
    int accepted;          // last pass accepted
    int cur;               // X buffer holding x^k
    int ck, ckm1, cnew;    // roles of the three column-sum buffers
    int active;            // 0: kernels return immediately (quota reached / stopped)
    int nan_flag;
    long long iters;       // accepted iterations in total
    long long passes;      // row passes in total
    long long chunk_acc;   // accepted iterations in the current chunk
    long long chunk_quota; // accepted iterations wanted per chunk
    long long capped;      // rows whose solve hit the round cap
    long long evals;       // row-equation evaluations (MIXED row solves)
    unsigned int ticket;   // last-block-done counter of the dual kernel
    unsigned int ticket2;  // last-block-done counter of the KKT goods kernel
    int row_cap;           // active-set rounds per row solve
    int pad;
    // MIXED x-bar folds in pairs: accepted iterates waiting to be folded (0, 1
    // or 2; with 2 the older one is in X[1 - cur], the newer in X[cur]) and
    // their weights eta_k / sum eta
    double xf_w1, xf_w2;
    int xf_n;
    int xf_folded;         // the waiting pair has been folded (set by the fold kernel's last block)
    int sections;          // FP64 row solve: 0 exact root, K >= 2 K-section search (Section 2.2)
    double sec_tol;        // relative bracket width that ends the K-section search
    unsigned int xf_ticket;   // last-block-done counter of the fold kernel
    int pad2;
    unsigned long long work[kMaxBuckets];   // dynamic work counters of the row kernel
};

// Results of one KKT evaluation (written by the KKT goods kernel's last block).
struct KktOut {
    double r_primal, r_dual, r_gap, kkt;
};

// Per-block partial maxima / sums of the KKT row kernel.
struct KktPart {
    double max_x, max_g, max_xg, max_y;
};

struct Bucket {
    int g;          // lanes per row (4, 8, 16, 32)
    int chunks;     // 0 = row fits in registers (g * kSlots), else multi-chunk
    long long first, count;   // internal rows [first, first + count)
};

// ---------------------------------------------------------------------------
// float-float ("double-single") arithmetic: an unevaluated sum hi + lo of two
// floats with |lo| <= ulp(hi)/2, giving about 48 significant bits.  Built from
// the error-free transformations TwoSum (Knuth) and TwoProduct via FMA
// (Dekker's product, exact with a fused multiply-add).
// ---------------------------------------------------------------------------
struct ff { float hi, lo; };

__device__ __forceinline__ ff ff_make(float h, float l) { ff r; r.hi = h; r.lo = l; return r; }
__device__ __forceinline__ ff ff_from_double(double d) {
    float h = (float)d;
    return ff_make(h, (float)(d - (double)h));
}
__device__ __forceinline__ double ff_to_double(ff a) { return (double)a.hi + (double)a.lo; }

// s + e = a + b exactly
__device__ __forceinline__ ff two_sum(float a, float b) {
    float s = __fadd_rn(a, b);
    float bb = __fsub_rn(s, a);
    float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return ff_make(s, e);
}
// requires |a| >= |b| (or a == 0)
__device__ __forceinline__ ff quick_two_sum(float a, float b) {
    float s = __fadd_rn(a, b);
    float e = __fsub_rn(b, __fsub_rn(s, a));
    return ff_make(s, e);
}
// p + e = a * b exactly
__device__ __forceinline__ ff two_prod(float a, float b) {
    float p = __fmul_rn(a, b);
    float e = __fmaf_rn(a, b, -p);
    return ff_make(p, e);
}
__device__ __forceinline__ ff ff_add(ff a, ff b) {
    ff s = two_sum(a.hi, b.hi);
    float e = __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo));
    return quick_two_sum(s.hi, e);
}
__device__ __forceinline__ ff ff_neg(ff a) { return ff_make(-a.hi, -a.lo); }
__device__ __forceinline__ ff ff_sub(ff a, ff b) { return ff_add(a, ff_neg(b)); }
__device__ __forceinline__ ff ff_add_f(ff a, float b) {
    ff s = two_sum(a.hi, b);
    return quick_two_sum(s.hi, __fadd_rn(s.lo, a.lo));
}
__device__ __forceinline__ ff ff_mul(ff a, ff b) {
    ff p = two_prod(a.hi, b.hi);
    float e = __fmaf_rn(a.hi, b.lo, p.lo);
    e = __fmaf_rn(a.lo, b.hi, e);
    return quick_two_sum(p.hi, e);
}
__device__ __forceinline__ ff ff_mul_f(ff a, float b) {
    ff p = two_prod(a.hi, b);
    float e = __fmaf_rn(a.lo, b, p.lo);
    return quick_two_sum(p.hi, e);
}
// a / b with one correction step
__device__ __forceinline__ ff ff_div(ff a, ff b) {
    float q1 = __fdiv_rn(a.hi, b.hi);
    ff r = ff_sub(a, ff_mul_f(b, q1));
    float q2 = __fdiv_rn(r.hi, b.hi);
    return quick_two_sum(q1, q2);
}
// ---------------------------------------------------------------------------
// stochastic rounding of FP32 iterates
// ---------------------------------------------------------------------------
// Near convergence a PDHCG increment tau (u_ij y_i - p_j) can fall below half
// an ulp of a large x_ij; round-to-nearest then drops it every iteration and
// the iteration stalls short of the tolerance.  Rounding to one of the two
// neighbouring floats with probability proportional to proximity keeps every
// stored value unbiased, so small increments accumulate in expectation.  The
// random bits come from a counter-based mixer of (entry, pass), so runs are
// deterministic.
__device__ __forceinline__ unsigned mix32(unsigned x) {   // multiply-xorshift mixer
    x ^= x >> 16;
    x *= 0x9E3779B1u;                                      // 32-bit golden-ratio constant
    x ^= x >> 15;
    x *= 0x85EBCA77u;
    x ^= x >> 13;
    return x;
}
__device__ __forceinline__ unsigned sr_bits(long long idx, unsigned seed) {
    return mix32((unsigned)idx ^ mix32((unsigned)(idx >> 32) + seed));
}
// a + b rounded stochastically with 16 random bits r
__device__ __forceinline__ float sr_add(float a, float b, unsigned r) {
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));   // a + b = s + e
    if (e == 0.0f || s == 0.0f) return s;
    const int sb = __float_as_int(s);
    const float nb = __int_as_float(((e > 0.0f) == (s > 0.0f)) ? sb + 1 : sb - 1);   // neighbour towards e
    return (float)(r & 0xffffu) * (1.0f / 65536.0f) * fabsf(nb - s) < fabsf(e) ? nb : s;
}


// Cheaper generator for the row kernel: one full mix per (row, pass) and a
// short xorshift-multiply per entry of the row (position k within the row),
// in the manner of a Weyl sequence fed through a one-multiply finaliser.
__device__ __forceinline__ unsigned row_hash(long long row, unsigned seed) {
    return mix32((unsigned)row * 0x9E3779B1u ^ seed);
}
__device__ __forceinline__ unsigned entry_hash(unsigned rh, unsigned k) {
    unsigned h = rh + k * 0x9E3779B9u;      // Weyl step by the golden-ratio constant
    h ^= h >> 15;
    h *= 0x2C1B3C6Du;
    h ^= h >> 12;
    return h;
}
// uniform in [0, 1) from 23 random bits (the mantissa of a float in [1, 2))
__device__ __forceinline__ float rand01_lo(unsigned bits) {
    return __int_as_float(0x3f800000u | (bits & 0x7fffffu)) - 1.0f;
}
__device__ __forceinline__ float rand01_hi(unsigned bits) {
    return __int_as_float(0x3f800000u | (bits >> 9)) - 1.0f;
}
// a + b (a, b such that the exact sum is >= 0) rounded stochastically with a
// uniform r in [0, 1): s + e = a + b exactly (TwoSum); with h the spacing of
// the floats next to s on the side of e, s + (e + r h) rounded DOWN is the
// upper neighbour of the exact sum with probability equal to its distance from
// the lower one over h, so the stored value is unbiased.  (At a power of two
// the spacing below s is half the spacing above; taking h on e's side keeps
// the probabilities exact there too.)
__device__ __forceinline__ float sr_add_rd(float a, float b, float r) {
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    const int sb = __float_as_int(s);
    const float nb = __int_as_float(e >= 0.0f ? sb + 1 : sb - 1);
    const float h = fabsf(nb - s);
    return __fadd_rd(s, __fmaf_rn(r, h, e));
}
// a > b for normalised float-float values
__device__ __forceinline__ bool ff_gt(ff a, ff b) { return a.hi > b.hi || (a.hi == b.hi && a.lo > b.lo); }

// ---------------------------------------------------------------------------
// shared-memory atomics with the state space spelled out (a generic-address
// atomic that resolves to shared memory is not supported for every operation)
// ---------------------------------------------------------------------------
__device__ __forceinline__ unsigned smem_addr(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void shared_add_u64(unsigned long long* p, unsigned long long v) {
    asm volatile("red.shared.add.u64 [%0], %1;" ::"r"(smem_addr(p)), "l"(v) : "memory");
}
__device__ __forceinline__ void shared_add_f64(void* p, double v) {
    asm volatile("red.shared.add.f64 [%0], %1;" ::"r"(smem_addr(p)), "d"(v) : "memory");
}
__device__ __forceinline__ void shared_add_s32(int* p, int v) {
    asm volatile("red.shared.add.s32 [%0], %1;" ::"r"(smem_addr(p)), "r"(v) : "memory");
}
__device__ __forceinline__ void shared_or_b32(unsigned* p, unsigned v) {
    asm volatile("red.shared.or.b32 [%0], %1;" ::"r"(smem_addr(p)), "r"(v) : "memory");
}
__device__ __forceinline__ void shared_min_s32(int* p, int v) {
    asm volatile("red.shared.min.s32 [%0], %1;" ::"r"(smem_addr(p)), "r"(v) : "memory");
}
__device__ __forceinline__ unsigned long long shared_cas_b64(unsigned long long* p, unsigned long long cmp,
                                                            unsigned long long val) {
    unsigned long long old;
    asm volatile("atom.shared.cas.b64 %0, [%1], %2, %3;" : "=l"(old) : "r"(smem_addr(p)), "l"(cmp), "l"(val) : "memory");
    return old;
}

// ---------------------------------------------------------------------------
// misc device helpers
// ---------------------------------------------------------------------------
__device__ __forceinline__ unsigned long long dbits(double d) { return (unsigned long long)__double_as_longlong(d); }


template <int G>
__device__ __forceinline__ float group_sum(float v) {
#pragma unroll
    for (int o = G / 2; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
template <int G>
__device__ __forceinline__ double group_sum(double v) {
#pragma unroll
    for (int o = G / 2; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
template <int G>
__device__ __forceinline__ ff group_sum(ff v) {
#pragma unroll
    for (int o = G / 2; o > 0; o >>= 1) {
        ff w = ff_make(__shfl_xor_sync(0xffffffffu, v.hi, o), __shfl_xor_sync(0xffffffffu, v.lo, o));
        v = ff_add(v, w);
    }
    return v;
}
template <int G>
__device__ __forceinline__ bool group_any(bool b) {
    unsigned bal = __ballot_sync(0xffffffffu, b);
    int lane = threadIdx.x & 31;
    unsigned gm = (G == 32) ? 0xffffffffu : (((1u << G) - 1u) << (lane & ~(G - 1)));
    return (bal & gm) != 0u;
}

__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
__device__ __forceinline__ double warp_max_d(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

// Row scale of the Section 5 preprocessing.  FP64 divides a row by its
// maximum.  FP32 divides by the largest power of two not above the maximum, so
// that FP32 utilities are scaled exactly (the scaled maximum lies in [1, 2));
// the KKT evaluation multiplies y by the scaled row maximum to report the
// residuals of the max-scaled market.
template <typename V>
__device__ __forceinline__ double row_scale(double mx) {
    if (sizeof(V) == sizeof(double)) return mx;
    int e;
    frexp(mx, &e);              // mx = f 2^e, f in [0.5, 1)
    return ldexp(1.0, e - 1);
}

// ---------------------------------------------------------------------------
// kernel launchers (defined in prox.cu, kkt.cu, prep.cu)
// ---------------------------------------------------------------------------
// The preprocessed market (single-market solver): rows stored bucket by bucket
// (internal row r is caller row perm[r]; the row kernel solves one bucket after
// another, so it streams the arrays in order), goods relabelled by degree.
struct DevMarket {
    int n, m;
    long long nnz;
    const long long* rp;   // internal row pointer
    const int* cj;
    const void* uv;        // float or double
    const double* w;
    const float2* wff;     // MIXED: budgets as float-float (internal row order)
    Bucket buckets[kMaxBuckets];
    int nb;
    int hot;               // goods [0, hot) accumulate in shared memory
    int nprox;             // persistent grid of the row kernel (blocks)
    int mixed;             // value type of uv: 1 float, 0 double
};

struct IterBufs {
    void* X[2];
    void* Xb;
    double* p;         // p^k (committed)
    double* pc;        // candidate p^{k+1}
    float2* pff;       // candidate as float-float (MIXED)
    double* pbar;
    double* C[3];      // column sums c^{k-1}, c^k, c_new (roles in Ctl)
    unsigned long long* acc;   // fixed-point accumulators (MIXED) or double bits (FP64)
    double* t;         // FP64: s* of the last pass (per row)
    float2* yst;       // MIXED: y = w / s* of the last pass as float-float (per row)
    double* part;      // per-block partials of the row kernel
    double* part2;     // per-block partials of the dual kernel (2 per block)
    float2* pff_p;     // committed p and p-bar as float-float (for the MIXED KKT)
    float2* pff_pb;
};

int prox_blocks(bool mixed, int hot);  // persistent grid of the row kernel (occupancy based)
int max_prox_blocks();                  // upper bound over all configurations
void launch_price(bool mixed, const DevMarket& mk, const IterBufs& b, Ctl* ctl, cudaStream_t s);
void launch_prox(bool mixed, const DevMarket& mk, const IterBufs& b, Ctl* ctl, cudaStream_t s);
void launch_dual(bool mixed, const DevMarket& mk, const IterBufs& b, Ctl* ctl, cudaStream_t s);
void launch_to_ff(int m, const double* p, float2* pff, cudaStream_t s);
void launch_flush(bool mixed, const DevMarket& mk, const IterBufs& b, Ctl* ctl, cudaStream_t s);
// MIXED: fold two waiting accepted iterates into x-bar (no-op otherwise)
void launch_fold(bool mixed, const DevMarket& mk, const IterBufs& b, Ctl* ctl, cudaStream_t s);
// one standalone prox pass with fixed tau and prices (no step control)
void launch_prox_fixed(bool mixed, const DevMarket& mk, const void* x_in, void* x_out, const double* p,
                       double tau, unsigned long long* acc, double* t_out, double* c_out,
                       double* part, Ctl* ctl, cudaStream_t s);

struct KktBufs {
    unsigned long long* acc;   // column-sum accumulator (MIXED fixed point / FP64 bits)
    unsigned long long* M;     // column maxima of u_ij y_i (double bits)
    double* c_out;             // column sums of x (may be null)
    double* t_out;             // row utilities of x (may be null)
    KktPart* part;             // per block
    double* gpart;             // per block of the goods kernel (4 each)
    KktOut* out;
    Ctl* ctl;                  // ticket2
    const void* xsel[2];       // when sel != null the point is xsel[*sel]
    const int* sel;
    const float2* pff;         // MIXED: the prices as float-float
    float* nd_part;            // MIXED: per-block max_ij (u_ij y_i - p_j)
};
int kkt_blocks();
void launch_kkt(bool mixed, const DevMarket& mk, const void* x, const double* p, const KktBufs& kb,
                cudaStream_t s);

}  // namespace pdhcg
