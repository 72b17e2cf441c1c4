// Row kernel of the MIXED form over CSR tiles: steps a2-a4 of one PDHCG pass
// (the row subproblems of Section 2.2 with the column sums of Eq. update:py
// and the running average of Alg. 2 fused).
//
// Buyers are cut, in CSR order, into tiles of whole rows holding at most
// kTileCap entries and kTileRows rows.  A persistent block takes every
// gridDim.x-th tile.  A tile's utilities, x^k, x-bar and good ids, with its
// row offsets, budgets and the utilities t of the previous pass, arrive by
// bulk asynchronous copies (cp.async.bulk, completion on an mbarrier) in one
// of two shared-memory stages, so the next tile streams in while the current
// one is solved.  Each thread owns kTileE consecutive entries.  Row sums are
// per-thread runs combined by a segmented warp scan and shared-memory atomics.
//
// Row equation (the arithmetic of row_mixed_core): F(y) = s0 - C(y) - w/y with
// s0 = u^T x^k and w/y in float-float and C(y) = sum u min(tau d, x) in FP32.
// Every row starts from y_0 = w / t_prev, so the first sweep computes s0 and
// the evaluation at y_0 together.  A frozen-active-set quadratic step then
// gives y_1; when no entry of the row changes activity between y_0 and y_1
// the frozen model is exact and y_1 is the root, which a sweep without
// reductions verifies.  Only rows whose active set moved are evaluated again.
// Rows longer than a tile go to the warp-chunked path after the tiles.
#include <cstdlib>

#include "common.cuh"
#include "rowsolve.cuh"

namespace pdhcg {

namespace {

// ---- shared-memory stage layout (bytes) ----
constexpr int kTileRowBuf = kTileRows + 4;                  // staged row_ptr / w entries
constexpr int kOffU = 0;
constexpr int kOffX = kOffU + kTileCap * 4;
constexpr int kOffXb = kOffX + kTileCap * 4;
constexpr int kOffJ = kOffXb + kTileCap * 4;
constexpr int kOffRp = kOffJ + kTileCap * 4;
constexpr int kOffW = kOffRp + kTileRowBuf * 8;
constexpr int kOffT = kOffW + kTileRowBuf * 8;
constexpr int kStageBytes = kOffT + kTileRowBuf * 8;
static_assert(kStageBytes % 16 == 0, "stage size must keep 16-byte alignment");
static_assert(kTileCap == kThreads * kTileE, "tile capacity");

struct TileHdr {
    long long ea, eb, A;   // entries [ea, eb); stage holds entries from A = ea rounded down to 4
    int ra, rb;            // rows [ra, rb)
};

// per-row state of the tile being solved
enum : int { kRowEval = 0, kRowCheck = 1, kRowDone = 2 };
struct TileRows {
    double s0[kTileRows];
    double Cf[kTileRows];           // C at the final y (utility t = s0 - Cf)
    float yh[kTileRows], yl[kTileRows];            // current y
    float ymh[kTileRows], yml[kTileRows];          // point of the frozen model (state kRowCheck)
    float loh[kTileRows], lol[kTileRows], hih[kTileRows], hil[kTileRows];
    float C[kTileRows], A[kTileRows], Q[kTileRows];
    float Cm[kTileRows], Qm[kTileRows];            // C and Q of the frozen model
    int st[kTileRows], chg[kTileRows], steps[kTileRows], nev[kTileRows];
    int off[kTileRows + 1];         // entry offsets of the rows, relative to A
};

// ---- bulk copies and mbarriers ----
__device__ __forceinline__ void mbar_init(unsigned long long* bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_init_fence() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(unsigned long long* bar, unsigned bytes) {
    unsigned long long state;
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 %0, [%1], %2;"
                 : "=l"(state) : "r"(smem_addr(bar)), "r"(bytes) : "memory");
    asm volatile("" ::"l"(state));
}
__device__ __forceinline__ bool mbar_try_wait(unsigned long long* bar, unsigned parity) {
    unsigned ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok) : "r"(smem_addr(bar)), "r"(parity) : "memory");
    return ok != 0;
}
// bounded wait: false after ~2^24 polls (seconds), never spins forever
__device__ __forceinline__ bool mbar_wait(unsigned long long* bar, unsigned parity) {
    for (int it = 0; it < (1 << 24); it++)
        if (mbar_try_wait(bar, parity)) return true;
    return false;
}
__device__ __forceinline__ void proxy_fence() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
// global -> shared bulk copy; dst, src 16-byte aligned, bytes a multiple of 16
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, unsigned bytes, unsigned long long* bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                 ::"r"(smem_addr(dst)), "l"(src), "r"(bytes), "r"(smem_addr(bar)) : "memory");
}
__device__ __forceinline__ void shared_add_f32(float* p, float v) {
    asm volatile("red.shared.add.f32 [%0], %1;" ::"r"(smem_addr(p)), "f"(v) : "memory");
}

// thread 0: start the copies of tile t into a stage
__device__ void tile_issue(const DevMarket& mk, const float* Xin, const float* Xb, const double* tprev, bool fold,
                           int2 rr, longlong2 ee, unsigned char* st, unsigned long long* bar, TileHdr* hd) {
    const long long A = ee.x & ~3LL;
    const unsigned vb = (unsigned)(((ee.y - A) + 3) & ~3LL) * 4u;        // <= kTileCap * 4
    const int ra2 = rr.x & ~1;
    const unsigned nrp = (unsigned)((rr.y + 1 - ra2 + 1) & ~1);          // rp[ra2, ra2 + nrp)
    const unsigned nw = (unsigned)((rr.y - ra2 + 1) & ~1);               // w[ra2, ra2 + nw)
    hd->ea = ee.x;
    hd->eb = ee.y;
    hd->A = A;
    hd->ra = rr.x;
    hd->rb = rr.y;
    const unsigned bytes = vb * (fold ? 4u : 3u) + (nrp + 2 * nw) * 8u;
    proxy_fence();
    mbar_expect_tx(bar, bytes);
    bulk_g2s(st + kOffU, (const float*)mk.uv + A, vb, bar);
    bulk_g2s(st + kOffX, Xin + A, vb, bar);
    if (fold) bulk_g2s(st + kOffXb, Xb + A, vb, bar);
    bulk_g2s(st + kOffJ, mk.cj + A, vb, bar);
    bulk_g2s(st + kOffRp, mk.rp + ra2, nrp * 8u, bar);
    bulk_g2s(st + kOffW, mk.w + ra2, nw * 8u, bar);
    bulk_g2s(st + kOffT, tprev + ra2, nw * 8u, bar);
}

// Segmented suffix sums over the lanes of a warp: lanes with equal keys form
// contiguous runs (keys are row ids in entry order); afterwards the first lane
// of each run holds the run's total.  Returns true on that lane.
__device__ __forceinline__ bool seg_head(int key) {
    const int lane = threadIdx.x & 31;
    const int prev = __shfl_up_sync(0xffffffffu, key, 1);
    return lane == 0 || prev != key;
}
__device__ __forceinline__ void seg_sum3(int key, float& a, float& b, float& c) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int k2 = __shfl_down_sync(0xffffffffu, key, o);
        const float a2 = __shfl_down_sync(0xffffffffu, a, o);
        const float b2 = __shfl_down_sync(0xffffffffu, b, o);
        const float c2 = __shfl_down_sync(0xffffffffu, c, o);
        if (lane + o < 32 && k2 == key) { a += a2; b += b2; c += c2; }
    }
}
__device__ __forceinline__ void seg_sum_ff(int key, ff& v) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int k2 = __shfl_down_sync(0xffffffffu, key, o);
        const ff v2 = ff_make(__shfl_down_sync(0xffffffffu, v.hi, o), __shfl_down_sync(0xffffffffu, v.lo, o));
        if (lane + o < 32 && k2 == key) v = ff_add(v, v2);
    }
}

}  // namespace

// hot column sums, then the two stages (16-byte aligned for the bulk copies and vector reads)
__host__ __device__ static inline size_t stage_offset(int hot) { return ((size_t)hot * 8 + 15) & ~(size_t)15; }
size_t tile_smem_bytes(int hot) { return stage_offset(hot) + 2 * (size_t)kStageBytes; }

__global__ void __launch_bounds__(kThreads, 2) tile_kernel(DevMarket mk, const void* Xin_fixed, void* Xout_fixed,
                                                         IterBufs bf, Ctl* ctl, int fixed) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ TileRows R;
    __shared__ __align__(8) unsigned long long bar[2];
    __shared__ TileHdr hdr[2];
    if (!ctl->active) return;
    const int tid = threadIdx.x;
    RowCtx rc;
    rc.tau = ctl->tau;
    rc.tau_hi = (float)rc.tau;
    rc.tau_lo = (float)(rc.tau - (double)rc.tau_hi);
    rc.fold = !fixed && ctl->fold_pending;
    rc.fold_wd = ctl->fold_wgt;
    rc.fold_w = (float)rc.fold_wd;
    rc.cap = ctl->row_cap;
    rc.seed = mix32((unsigned)ctl->passes * 2u + 1u);
    const int cur = ctl->cur;
    const float* Xin = (const float*)(fixed ? Xin_fixed : (cur ? bf.X[1] : bf.X[0]));
    float* Xout = (float*)(fixed ? Xout_fixed : (cur ? bf.X[0] : bf.X[1]));
    float* Xb = (float*)bf.Xb;
    const float tau = rc.tau_hi;
    const float fw = rc.fold_w;
    const int hot = mk.hot;

    unsigned long long* acc_s = (unsigned long long*)smem;
    unsigned char* stages = smem + stage_offset(hot);
    for (int j = tid; j < hot; j += kThreads) acc_s[j] = 0ull;
    if (tid == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        mbar_init_fence();
    }
    __syncthreads();

    float dxf = 0.0f;
    int capped = 0, evals = 0;
    unsigned par0 = 0u, par1 = 0u;      // mbarrier phase parity of the two stages
    bool timed_out = false;
    int s = 0;
    int t = blockIdx.x;
    // thread 0 keeps the descriptor of the next tile in registers, loaded one
    // tile ahead, so issuing a tile's copies never waits on memory
    int2 nrr = make_int2(0, 0);
    longlong2 nee;
    nee.x = nee.y = 0;
    if (tid == 0 && t < mk.ntiles) {
        tile_issue(mk, Xin, Xb, bf.t, rc.fold, mk.tile_rows[t], mk.tile_ent[t], stages, &bar[0], &hdr[0]);
        if (t + (int)gridDim.x < mk.ntiles) {
            nrr = mk.tile_rows[t + gridDim.x];
            nee = mk.tile_ent[t + gridDim.x];
        }
    }

    for (; t < mk.ntiles; t += gridDim.x) {
        const int tn = t + gridDim.x;
        if (tid == 0 && tn < mk.ntiles) {
            tile_issue(mk, Xin, Xb, bf.t, rc.fold, nrr, nee, stages + (size_t)(s ^ 1) * kStageBytes, &bar[s ^ 1],
                       &hdr[s ^ 1]);
            if (tn + (int)gridDim.x < mk.ntiles) {
                nrr = mk.tile_rows[tn + gridDim.x];
                nee = mk.tile_ent[tn + gridDim.x];
            }
        }
        const bool ok = mbar_wait(&bar[s], s ? par1 : par0);
        if (__syncthreads_or(!ok)) { timed_out = true; break; }
        if (s) par1 ^= 1u; else par0 ^= 1u;

        // ================= solve tile t from stage s =================
        const unsigned char* st = stages + (size_t)s * kStageBytes;
        const float* su = (const float*)(st + kOffU);
        const float* sx = (const float*)(st + kOffX);
        const float* sxb = (const float*)(st + kOffXb);
        const int* sj = (const int*)(st + kOffJ);
        const long long* srp = (const long long*)(st + kOffRp);
        const double* sw = (const double*)(st + kOffW);
        const double* stp = (const double*)(st + kOffT);
        const TileHdr hd = hdr[s];
        const int nr = hd.rb - hd.ra;
        const long long A0 = hd.A;
        const int ro = hd.ra & 1;
        const int L0 = (int)(hd.ea - A0), L1 = (int)(hd.eb - A0);

        // ---- own entries: local positions Lb .. Lb + kTileE - 1; prices
        // are gathered first so that their latency overlaps the row setup ----
        const int Lb = tid * kTileE;
        float u[kTileE], x[kTileE], ph[kTileE], pl[kTileE], td[kTileE];
        int lr[kTileE], jj[kTileE];
        unsigned actm = 0u;           // bit k: entry k active (tau d < x) at the last evaluation
        {
            const float4* u4 = (const float4*)(su + Lb);
            const float4* x4 = (const float4*)(sx + Lb);
            const int4* j4 = (const int4*)(sj + Lb);
#pragma unroll
            for (int q = 0; q < kTileE / 4; q++) {
                const float4 a = u4[q], c = x4[q];
                const int4 g = j4[q];
                u[4 * q] = a.x; u[4 * q + 1] = a.y; u[4 * q + 2] = a.z; u[4 * q + 3] = a.w;
                x[4 * q] = c.x; x[4 * q + 1] = c.y; x[4 * q + 2] = c.z; x[4 * q + 3] = c.w;
                jj[4 * q] = g.x; jj[4 * q + 1] = g.y; jj[4 * q + 2] = g.z; jj[4 * q + 3] = g.w;
            }
#pragma unroll
            for (int k = 0; k < kTileE; k++) {
                const int L = Lb + k;
                td[k] = 0.0f;
                if (L < L0 || L >= L1) {
                    lr[k] = -1;
                    u[k] = 0.0f; x[k] = 0.0f; ph[k] = 0.0f; pl[k] = 0.0f;
                } else {
                    lr[k] = 0;
                    const float2 p = __ldg(bf.pff + jj[k]);
                    ph[k] = p.x;
                    pl[k] = p.y;
                }
            }
        }

        // ---- rows: offsets and the start y_0 = w / t_prev ----
        if (tid <= nr) R.off[tid] = (int)(srp[ro + tid] - A0);
        if (tid < nr) {
            const double tp = stp[ro + tid];
            ff y0 = ff_make(1.0f, 0.0f);
            if (tp > 0.0 && tp < 1e300) y0 = ff_div_fast(ff_from_double(sw[ro + tid]), ff_from_double(tp));
            if (!(y0.hi > 0.0f) || !isfinite(y0.hi)) y0 = ff_make(1.0f, 0.0f);
            R.yh[tid] = y0.hi;
            R.yl[tid] = y0.lo;
            R.s0[tid] = 0.0;
            R.C[tid] = 0.0f;
            R.A[tid] = 0.0f;
            R.Q[tid] = 0.0f;
            R.st[tid] = kRowEval;
            R.chg[tid] = 0;
            R.steps[tid] = 0;
            R.nev[tid] = 0;
            R.loh[tid] = 0.0f;
            R.lol[tid] = 0.0f;
            R.hih[tid] = INFINITY;
            R.hil[tid] = 0.0f;
        }
        __syncthreads();

        // ---- row of each own entry ----
        {
            int r = 0;
            const int Lf = max(Lb, L0);
            if (Lf < L1) {
                int lo = 0, hi = nr - 1;                // largest r with off[r] <= Lf
                while (lo < hi) {
                    const int mid = (lo + hi + 1) >> 1;
                    if (R.off[mid] <= Lf) lo = mid; else hi = mid - 1;
                }
                r = lo;
            }
#pragma unroll
            for (int k = 0; k < kTileE; k++) {
                if (lr[k] < 0) continue;
                const int L = Lb + k;
                while (R.off[r + 1] <= L) r++;
                lr[k] = r;
            }
        }

        // ---- sweeps: s0 (first sweep only), evaluations, activity checks ----
        bool first = true;
        while (true) {
            {
                ff sacc = ff_make(0.0f, 0.0f);
                float cC = 0.0f, cA = 0.0f, cQ = 0.0f, yh = 0.0f, yl = 0.0f;
                int rcur = -1, rst = kRowDone;
                bool chg = false;
#pragma unroll
                for (int k = 0; k < kTileE; k++) {
                    const int r = lr[k];
                    if (r < 0) continue;
                    if (r != rcur) {
                        if (rcur >= 0) {
                            if (first) shared_add_f64(&R.s0[rcur], (double)sacc.hi + (double)sacc.lo);
                            if (rst == kRowEval) {
                                shared_add_f32(&R.C[rcur], cC);
                                shared_add_f32(&R.A[rcur], cA);
                                shared_add_f32(&R.Q[rcur], cQ);
                            } else if (rst == kRowCheck && chg) {
                                atomicOr(&R.chg[rcur], 1);
                            }
                        }
                        rcur = r;
                        rst = R.st[r];
                        yh = R.yh[r];
                        yl = R.yl[r];
                        sacc = ff_make(0.0f, 0.0f);
                        cC = cA = cQ = 0.0f;
                        chg = false;
                    }
                    if (first) sacc = ff_add(sacc, two_prod(u[k], x[k]));
                    if (rst == kRowDone) continue;
                    const float uk = u[k];
                    const float d = fmaf(-uk, yl, fmaf(-uk, yh, ph[k]) + pl[k]);
                    const float tdk = tau * d;
                    td[k] = tdk;
                    const bool act = tdk < x[k];
                    const unsigned bit = 1u << k;
                    if (rst == kRowCheck) {
                        chg |= act != ((actm & bit) != 0u);
                    } else {
                        const float cr = fminf(tdk, x[k]);
                        cC = fmaf(uk, cr, cC);
                        cA = fmaf(uk, fabsf(cr), cA);
                        if (act) cQ = fmaf(uk, uk, cQ);
                    }
                    actm = act ? (actm | bit) : (actm & ~bit);
                }
                if (first) {
                    seg_sum_ff(rcur, sacc);
                    if (seg_head(rcur) && rcur >= 0) shared_add_f64(&R.s0[rcur], (double)sacc.hi + (double)sacc.lo);
                }
                const int key = (rcur >= 0 && rst == kRowEval) ? rcur : -1;
                seg_sum3(key, cC, cA, cQ);
                if (seg_head(key) && key >= 0) {
                    shared_add_f32(&R.C[key], cC);
                    shared_add_f32(&R.A[key], cA);
                    shared_add_f32(&R.Q[key], cQ);
                }
                if (rcur >= 0 && rst == kRowCheck && chg) atomicOr(&R.chg[rcur], 1);
            }
            __syncthreads();
            first = false;
            bool pending = false;
            if (tid < nr) {
                const int r = tid;
                const int rs = R.st[r];
                if (rs == kRowCheck) {
                    if (!R.chg[r]) {
                        // active set unchanged: the frozen model is exact at y
                        const double dy = ((double)R.yh[r] - (double)R.ymh[r]) + ((double)R.yl[r] - (double)R.yml[r]);
                        R.Cf[r] = (double)R.Cm[r] - (double)tau * (double)R.Qm[r] * dy;
                        R.st[r] = kRowDone;
                    } else {
                        R.chg[r] = 0;
                        R.st[r] = kRowEval;
                        pending = true;
                    }
                } else if (rs == kRowEval) {
                    const float yh = R.yh[r], yl = R.yl[r];
                    const float C = R.C[r], Ab = R.A[r], Q = R.Q[r];
                    R.C[r] = 0.0f;
                    R.A[r] = 0.0f;
                    R.Q[r] = 0.0f;
                    R.nev[r] += 1;
                    const ff s0 = ff_from_double(R.s0[r]);
                    const ff ws = ff_div_fast(ff_from_double(sw[ro + r]), ff_make(yh, yl));     // w / y
                    const ff D = ff_sub(s0, ws);
                    const float F = (D.hi - C) + D.lo;
                    // rounding bound of F: per-thread runs of kTileE terms, a warp
                    // scan, one atomic per warp; plus the float-float resolution of
                    // p and y seen through tau Q y
                    const float deg = (float)(R.off[r + 1] - R.off[r]);
                    const float cn = 1.2e-7f * (2.83f + 5.0f + sqrtf(deg * (1.0f / 256.0f) + 1.0f));
                    const float aQ = tau * Q;
                    const float floor = fmaf(cn, Ab, fmaf(3e-14f, aQ * yh, 2e-8f * ws.hi));
                    const int steps = R.steps[r] + 1;
                    R.steps[r] = steps;
                    bool fin = false;
                    if (fabsf(F) <= floor || steps >= rc.cap) {
                        fin = true;
                        if (fabsf(F) > floor) capped++;
                    } else {
                        if (F > 0.0f) { R.hih[r] = yh; R.hil[r] = yl; } else { R.loh[r] = yh; R.lol[r] = yl; }
                        const ff lo = ff_make(R.loh[r], R.lol[r]), hi = ff_make(R.hih[r], R.hil[r]);
                        // root of the frozen-active-set quadratic a d^2 + b d + c = 0,
                        // b = sum u x_new + tau Q y >= 0
                        const float bq = fmaf(aQ, yh, F + ws.hi);
                        const float cq = F * yh;
                        const float disc = fmaf(bq, bq, -4.0f * aQ * cq);
                        const float delta = __fdividef(-2.0f * cq, bq + sqrtf(fmaxf(disc, 0.0f)));
                        ff yn = ff_add_f(ff_make(yh, yl), delta);
                        // the frozen model may stand in for an evaluation at the new
                        // y only when its own rounding error (cn A) is as small as the
                        // final tolerance; far from the root evaluate again
                        bool model = cn * Ab <= 2e-8f * ws.hi;
                        if (!(ff_gt(yn, lo) && ff_gt(hi, yn))) {      // rounding left the bracket
                            yn = isinf(hi.hi) ? ff_make(2.0f * yh, 0.0f) : ff_mul_f(ff_add(lo, hi), 0.5f);
                            model = false;
                        }
                        if (yn.hi == yh && yn.lo == yl) {
                            fin = true;                                // no representable progress
                        } else {
                            if (model) {
                                R.ymh[r] = yh;
                                R.yml[r] = yl;
                                R.Cm[r] = C;
                                R.Qm[r] = Q;
                                R.st[r] = kRowCheck;
                            }
                            R.yh[r] = yn.hi;
                            R.yl[r] = yn.lo;
                            pending = true;
                        }
                    }
                    if (fin) {
                        R.Cf[r] = (double)C;
                        R.st[r] = kRowDone;
                    }
                }
            }
            if (!__syncthreads_or(pending)) break;
        }

        // ---- utilities of the rows ----
        if (tid < nr) {
            bf.t[hd.ra + tid] = R.s0[tid] - R.Cf[tid];
            evals += R.nev[tid];
        }

        // ---- x^{k+1}, average fold, column sums ----
        {
            float xo[kTileE], xbo[kTileE];
            if (rc.fold) {
                const float4* b4 = (const float4*)(sxb + Lb);
#pragma unroll
                for (int q = 0; q < kTileE / 4; q++) {
                    const float4 a = b4[q];
                    xbo[4 * q] = a.x; xbo[4 * q + 1] = a.y; xbo[4 * q + 2] = a.z; xbo[4 * q + 3] = a.w;
                }
            }
            // random bits: one mixed seed per thread and tile, then xorshift steps
            unsigned rs = sr_bits(A0 + Lb, rc.seed) | 1u;
#pragma unroll
            for (int k = 0; k < kTileE; k++) {
                xo[k] = 0.0f;
                rs ^= rs << 13;
                rs ^= rs >> 17;
                rs ^= rs << 5;
                if (lr[k] < 0) continue;
                const unsigned rb = rs;
                const float xn = td[k] < x[k] ? sr_add_fast(x[k], -td[k], rb) : 0.0f;
                xo[k] = xn;
                const float dd = xn - x[k];
                dxf = fmaf(dd, dd, dxf);
                if (rc.fold) {
                    const float xb = xbo[k];
                    xbo[k] = (fw == 1.0f) ? x[k] : sr_add_fast(xb, fw * (x[k] - xb), rb >> 16);
                }
                acc_add_fixed(acc_s, bf.acc, hot, jj[k], xn);
            }
            float* xg = Xout + A0 + Lb;
            float* bg = Xb + A0 + Lb;
            if (Lb >= L0 && Lb + kTileE <= L1) {
#pragma unroll
                for (int q = 0; q < kTileE / 4; q++) {
                    __stcs((float4*)xg + q, make_float4(xo[4 * q], xo[4 * q + 1], xo[4 * q + 2], xo[4 * q + 3]));
                    if (rc.fold) ((float4*)bg)[q] = make_float4(xbo[4 * q], xbo[4 * q + 1], xbo[4 * q + 2], xbo[4 * q + 3]);
                }
            } else {
#pragma unroll
                for (int k = 0; k < kTileE; k++) {
                    if (lr[k] < 0) continue;
                    __stcs(xg + k, xo[k]);
                    if (rc.fold) bg[k] = xbo[k];
                }
            }
        }
        __syncthreads();     // stage s and the row state are free again
        s ^= 1;
    }

    if (timed_out) {
        // a bulk copy never completed: report it, give the copies still in
        // flight a bounded time to land, and leave without touching results
        if (tid == 0) {
            atomicExch(&ctl->nan_flag, 2);
            mbar_wait(&bar[s], s ? par1 : par0);
            if (t + (int)gridDim.x < mk.ntiles) mbar_wait(&bar[s ^ 1], s ? par0 : par1);
        }
        __syncthreads();
        return;
    }

    // ---- rows longer than a tile: warp-chunked path ----
    for (int bi = 0; bi < mk.nb; bi++) {
        const Bucket bk = mk.buckets[bi];
        const int lane = tid & 31;
        while (true) {
            unsigned long long base = 0;
            if (lane == 0) base = atomicAdd(&ctl->work[bi], 1ull);
            base = __shfl_sync(0xffffffffu, base, 0);
            if ((long long)base >= bk.count) break;
            const int row = mk.row_order[bk.first + (long long)base];
            RowRegs Rg;
            Rg.b = mk.rp[row];
            Rg.e = mk.rp[row + 1];
            row_mixed_core<32, true>(mk, (const float*)mk.uv, Xin, Xout, Xb, bf.pff, bf.pff, acc_s, bf.acc, bf.t, rc,
                                     row, true, dxf, capped, evals, Rg);
        }
    }

    // ---- block epilogue: ||dx||^2 partial, counters, hot column sums ----
    double v = warp_sum_d((double)dxf);
    __shared__ double red[kWarps];
    __shared__ int capred, evred;
    if (tid == 0) capred = evred = 0;
    __syncthreads();
    if ((tid & 31) == 0) red[tid >> 5] = v;
    if (capped) atomicAdd(&capred, capped);
    if (evals) atomicAdd(&evred, evals);
    __syncthreads();
    if (tid == 0) {
        double a = 0.0;
        for (int w = 0; w < kWarps; w++) a += red[w];
        bf.part[blockIdx.x] = a;
        if (capred) atomicAdd((unsigned long long*)&ctl->capped, (unsigned long long)capred);
        if (evred) atomicAdd((unsigned long long*)&ctl->evals, (unsigned long long)evred);
    }
    for (int j = tid; j < hot; j += kThreads) {
        const unsigned long long a = acc_s[j];
        if (a) atomicAdd(&bf.acc[j], a);
    }
}

static void tile_attr() {
    static bool done = false;
    if (done) return;
    done = true;
    cudaFuncSetAttribute(tile_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
}

int tile_blocks(int hot) {
    tile_attr();
    int per = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, tile_kernel, kThreads, tile_smem_bytes(hot));
    const char* env = getenv("PDHCG_PROX_BLOCKS_PER_SM");
    if (env && atoi(env) > 0 && atoi(env) < per) per = atoi(env);
    return sm_count() * per;
}

void launch_tile(const DevMarket& mk, const IterBufs& b, Ctl* ctl, const void* x_in, void* x_out, int fixed,
                 cudaStream_t s) {
    tile_attr();
    tile_kernel<<<mk.nprox, kThreads, tile_smem_bytes(mk.hot), s>>>(mk, x_in, x_out, b, ctl, fixed);
}

}  // namespace pdhcg
