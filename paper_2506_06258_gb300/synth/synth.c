/*
 * Seeded synthetic market generator.
 *
 * This file produces INPUTS only (sparse utility matrices U in CSR form and
 * budget vectors w).  It contains none of the equilibrium method's arithmetic,
 * so both the CUDA solver and the FP64 oracle may consume its output.
 *
 * Randomness: Philox4x32-10, the counter-based generator of Salmon, Moraes,
 * Dror and Shaw, "Parallel random numbers: as easy as 1, 2, 3" (SC'11),
 * implemented here from its published definition.  Every random draw is a pure
 * function of (seed, stream, index, draw number), so the output does not depend
 * on the number of OpenMP threads.
 *
 * Instance families (shapes of the paper's synthetic workloads, Section 5.1):
 *   - bernoulli: each (i,j) kept independently with probability q;
 *   - fixed degree: every buyer has exactly d distinct uniform goods;
 *   - skewed: buyer degrees ~ Zipf(s) clipped to [dmin,dmax] and rescaled to a
 *     target nnz; goods drawn by popularity proportional to rank^-alpha;
 *   - exchange: agent i holds its own good i plus d distinct others.
 * Utility laws: 0 = Uniform(lo,hi), 1 = LogNormal(0,1).
 * Assumption 1 of the paper (no empty row or column) is enforced by a repair
 * step that the Python wrapper applies (an empty row receives one uniform good,
 * an empty column one uniform buyer).
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>

/* ---------------- Philox4x32-10 ---------------- */
#define PH_M0 0xD2511F53u
#define PH_M1 0xCD9E8D57u
#define PH_W0 0x9E3779B9u
#define PH_W1 0xBB67AE85u

void synth_philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2], uint32_t out[4]) {
    uint32_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
    uint32_t k0 = key_in[0], k1 = key_in[1];
    for (int r = 0; r < 10; r++) {
        if (r > 0) { k0 += PH_W0; k1 += PH_W1; }
        uint64_t p0 = (uint64_t)PH_M0 * c0;
        uint64_t p1 = (uint64_t)PH_M1 * c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        c0 = n0; c1 = lo1; c2 = n2; c3 = lo0;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* A stream = fixed (key, ctr[1..2]) with a running draw counter in ctr[3]. */
typedef struct {
    uint32_t key[2];
    uint32_t c0, c1, c2;   /* identify the stream */
    uint32_t draw;         /* block counter */
    uint32_t buf[4];
    int pos;
} rstream;

static void rs_init(rstream* s, uint64_t seed, uint32_t stream, uint64_t index) {
    s->key[0] = (uint32_t)seed; s->key[1] = (uint32_t)(seed >> 32);
    s->c0 = (uint32_t)index; s->c1 = (uint32_t)(index >> 32); s->c2 = stream;
    s->draw = 0; s->pos = 4;
}
static uint32_t rs_u32(rstream* s) {
    if (s->pos == 4) {
        uint32_t ctr[4] = {s->c0, s->c1, s->c2, s->draw++};
        synth_philox4x32_10(ctr, s->key, s->buf);
        s->pos = 0;
    }
    return s->buf[s->pos++];
}
/* Uniform double in the open interval (0,1) with 53 random bits. */
static double rs_unif(rstream* s) {
    uint64_t a = rs_u32(s) >> 5, b = rs_u32(s) >> 6;   /* 27 + 26 bits */
    return ((double)((a << 26) | b) + 0.5) * (1.0 / 9007199254740992.0);
}
/* Uniform integer in [0, n) (n < 2^32) by rejection (no modulo bias). */
static uint32_t rs_below(rstream* s, uint32_t n) {
    uint32_t lim = (uint32_t)(((uint64_t)1 << 32) - (((uint64_t)1 << 32) % n));
    for (;;) {
        uint32_t r = rs_u32(s);
        if (lim == 0 || r < lim) return r % n;
    }
}
static double rs_normal(rstream* s) {   /* Box-Muller, cosine branch */
    double u1 = rs_unif(s), u2 = rs_unif(s);
    return sqrt(-2.0 * log(u1)) * cos(6.283185307179586 * u2);
}
static double rs_util(rstream* s, int law, double lo, double hi) {
    if (law == 1) return exp(rs_normal(s));
    return lo + (hi - lo) * rs_unif(s);
}

/* stream ids */
enum { ST_DEG = 1, ST_COLS = 2, ST_VAL = 3, ST_W = 4, ST_PERM = 5, ST_REPAIR = 6, ST_MKT = 7, ST_AUX = 8 };

static int cmp_i32(const void* a, const void* b) {
    int32_t x = *(const int32_t*)a, y = *(const int32_t*)b;
    return (x > y) - (x < y);
}

/* ---------------- budgets ---------------- */
void synth_budgets(uint64_t seed, int64_t n, double lo, double hi, double* w) {
    #pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; i++) {
        rstream s; rs_init(&s, seed, ST_W, (uint64_t)i);
        w[i] = lo + (hi - lo) * rs_unif(&s);
    }
}

/* ---------------- Bernoulli family ----------------
 * Row degrees: Binomial(m, q) by inversion of the exact CDF (table computed
 * once); the row's goods are then a uniform d-subset (Floyd's algorithm).  This
 * is the same law as keeping each (i,j) independently with probability q. */
static double* binom_cdf(int m, double q) {
    double* cdf = (double*)malloc(sizeof(double) * (m + 1));
    /* log pmf via lgamma for stability */
    double acc = 0.0;
    for (int k = 0; k <= m; k++) {
        double lp = lgamma(m + 1.0) - lgamma(k + 1.0) - lgamma(m - k + 1.0)
                  + (k > 0 ? k * log(q) : 0.0) + (m - k > 0 ? (m - k) * log1p(-q) : 0.0);
        acc += exp(lp);
        cdf[k] = acc;
    }
    for (int k = 0; k <= m; k++) cdf[k] /= acc;
    return cdf;
}
static int sample_cdf(const double* cdf, int len, double u) {  /* smallest k with cdf[k] >= u */
    int lo = 0, hi = len - 1;
    while (lo < hi) { int mid = (lo + hi) / 2; if (cdf[mid] >= u) hi = mid; else lo = mid + 1; }
    return lo;
}
void synth_bernoulli_degrees(uint64_t seed, int64_t n, int32_t m, double q, int32_t* deg) {
    double* cdf = binom_cdf(m, q);
    #pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; i++) {
        rstream s; rs_init(&s, seed, ST_DEG, (uint64_t)i);
        deg[i] = sample_cdf(cdf, m + 1, rs_unif(&s));
    }
    free(cdf);
}

/* Fill a uniform d-subset of [0,m) for every row (Floyd), sorted, plus values. */
static void fill_uniform_rows(uint64_t seed, int64_t n, int32_t m, const int64_t* row_ptr,
                              int32_t* col, double* val, float* valf, int law, double lo, double hi,
                              int32_t self_offset /* -1: none; else row i must contain good (i) */) {
    #pragma omp parallel
    {
        uint8_t* mark = (uint8_t*)calloc((size_t)m, 1);
        #pragma omp for schedule(dynamic, 1024)
        for (int64_t i = 0; i < n; i++) {
            rstream s; rs_init(&s, seed, ST_COLS, (uint64_t)i);
            int64_t b = row_ptr[i], e = row_ptr[i + 1];
            int32_t d = (int32_t)(e - b);
            int32_t k = 0;
            /* With an own good, the other d-1 goods are a uniform subset of the
             * m-1 goods different from i: Floyd over [0, m-1), then skip i. */
            int32_t own = (self_offset >= 0 && d > 0) ? (int32_t)i : -1;
            if (own >= 0) col[b + k++] = own;
            int32_t need = d - k;
            int32_t universe = own >= 0 ? m - 1 : m;
            for (int32_t t = universe - need; t < universe; t++) {
                int32_t r = (int32_t)rs_below(&s, (uint32_t)(t + 1));
                int32_t pick = mark[r] ? t : r;
                mark[pick] = 1;
                col[b + k++] = (own >= 0 && pick >= own) ? pick + 1 : pick;
            }
            /* clear Floyd marks (indices in the pre-skip universe) */
            for (int32_t q = (own >= 0 ? 1 : 0); q < d; q++) {
                int32_t g = col[b + q];
                mark[(own >= 0 && g > own) ? g - 1 : g] = 0;
            }
            qsort(col + b, (size_t)d, sizeof(int32_t), cmp_i32);
            rstream sv; rs_init(&sv, seed, ST_VAL, (uint64_t)i);
            for (int64_t p = b; p < e; p++) {
                double u = rs_util(&sv, law, lo, hi);
                if (val) val[p] = u;
                if (valf) valf[p] = (float)u;
            }
        }
        free(mark);
    }
}

void synth_fill_uniform(uint64_t seed, int64_t n, int32_t m, const int64_t* row_ptr,
                        int32_t* col, double* val, float* valf, int law, double lo, double hi,
                        int32_t with_self) {
    fill_uniform_rows(seed, n, m, row_ptr, col, val, valf, law, lo, hi, with_self ? 0 : -1);
}

/* ---------------- skewed family ---------------- */
/* Base Zipf(s) draw on [dmin, dmax] by inversion of the normalised table. */
void synth_zipf_base(uint64_t seed, int64_t n, double s_exp, int32_t dmin, int32_t dmax, int32_t* z) {
    int len = dmax - dmin + 1;
    double* cdf = (double*)malloc(sizeof(double) * len);
    double acc = 0.0;
    for (int k = 0; k < len; k++) { acc += pow((double)(dmin + k), -s_exp); cdf[k] = acc; }
    for (int k = 0; k < len; k++) cdf[k] /= acc;
    #pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; i++) {
        rstream s; rs_init(&s, seed, ST_DEG, (uint64_t)i);
        z[i] = dmin + sample_cdf(cdf, len, rs_unif(&s));
    }
    free(cdf);
}
/* d_i = clip(round(f * z_i), dmin, dmax); returns the total. */
int64_t synth_scale_degrees(int64_t n, const int32_t* z, double f, int32_t dmin, int32_t dmax, int32_t* d) {
    int64_t tot = 0;
    #pragma omp parallel for reduction(+:tot) schedule(static)
    for (int64_t i = 0; i < n; i++) {
        double v = floor(f * (double)z[i] + 0.5);
        if (v < dmin) v = dmin;
        if (v > dmax) v = dmax;
        int32_t di = (int32_t)v;
        if (d) d[i] = di;
        tot += di;
    }
    return tot;
}
/* Popularity table: good with rank r (0-based) has weight (r+1)^-alpha; rank ->
 * good id through a seeded Fisher-Yates permutation.  cdf has m entries. */
void synth_popularity(uint64_t seed, int32_t m, double alpha, double* cdf, int32_t* rank_to_good) {
    double acc = 0.0;
    for (int32_t r = 0; r < m; r++) { acc += pow((double)(r + 1), -alpha); cdf[r] = acc; }
    for (int32_t r = 0; r < m; r++) cdf[r] /= acc;
    for (int32_t r = 0; r < m; r++) rank_to_good[r] = r;
    rstream s; rs_init(&s, seed, ST_PERM, 0);
    for (int32_t r = m - 1; r > 0; r--) {
        int32_t k = (int32_t)rs_below(&s, (uint32_t)(r + 1));
        int32_t t = rank_to_good[r]; rank_to_good[r] = rank_to_good[k]; rank_to_good[k] = t;
    }
}
/* Fill rows with distinct goods drawn by popularity (rejection of repeats). */
void synth_fill_popular(uint64_t seed, int64_t n, int32_t m, const int64_t* row_ptr,
                        const double* cdf, const int32_t* rank_to_good,
                        int32_t* col, double* val, float* valf, int law, double lo, double hi) {
    #pragma omp parallel
    {
        uint8_t* mark = (uint8_t*)calloc((size_t)m, 1);
        #pragma omp for schedule(dynamic, 256)
        for (int64_t i = 0; i < n; i++) {
            rstream s; rs_init(&s, seed, ST_COLS, (uint64_t)i);
            int64_t b = row_ptr[i], e = row_ptr[i + 1];
            int64_t k = b;
            while (k < e) {
                int32_t g = rank_to_good[sample_cdf(cdf, m, rs_unif(&s))];
                if (mark[g]) continue;
                mark[g] = 1; col[k++] = g;
            }
            qsort(col + b, (size_t)(e - b), sizeof(int32_t), cmp_i32);
            for (int64_t p = b; p < e; p++) mark[col[p]] = 0;
            rstream sv; rs_init(&sv, seed, ST_VAL, (uint64_t)i);
            for (int64_t p = b; p < e; p++) {
                double u = rs_util(&sv, law, lo, hi);
                if (val) val[p] = u;
                if (valf) valf[p] = (float)u;
            }
        }
        free(mark);
    }
}

/* ---------------- Assumption-1 repair helpers ---------------- */
void synth_col_degrees(int64_t nnz, int32_t m, const int32_t* col, int64_t* cdeg) {
    memset(cdeg, 0, sizeof(int64_t) * (size_t)m);
    for (int64_t p = 0; p < nnz; p++) cdeg[col[p]]++;
}
/* Deterministic uniform choices used by the repair step. */
uint32_t synth_repair_draw(uint64_t seed, uint64_t index, uint32_t bound) {
    rstream s; rs_init(&s, seed, ST_REPAIR, index);
    return rs_below(&s, bound);
}
double synth_repair_util(uint64_t seed, uint64_t index, int law, double lo, double hi) {
    rstream s; rs_init(&s, seed, ST_AUX, index);
    return rs_util(&s, law, lo, hi);
}

/* ---------------- generic helpers for Python ---------------- */
void synth_uniform_array(uint64_t seed, uint32_t stream, int64_t n, double lo, double hi, double* out) {
    #pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; i++) {
        rstream s; rs_init(&s, seed, 100u + stream, (uint64_t)i);
        out[i] = lo + (hi - lo) * rs_unif(&s);
    }
}
void synth_normal_array(uint64_t seed, uint32_t stream, int64_t n, double* out) {
    #pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; i++) {
        rstream s; rs_init(&s, seed, 200u + stream, (uint64_t)i);
        out[i] = rs_normal(&s);
    }
}
void synth_int_array(uint64_t seed, uint32_t stream, int64_t n, int64_t lo, int64_t hi, int64_t* out) {
    #pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; i++) {
        rstream s; rs_init(&s, seed, 300u + stream, (uint64_t)i);
        out[i] = lo + (int64_t)rs_below(&s, (uint32_t)(hi - lo + 1));
    }
}
