// Restarted PDHG (Alg. 1) for the linear Fisher market, FP64, on the GPU: the
// paper's comparator for PDHCG and a second, independent route to the same
// equilibrium prices.
//
// Saddle form of Section 2 with the buyer utilities t as primal variables and
// their defining constraints t_i = sum_j u_ij x_ij dualised by y.  One step
// (Eq. update-rule) is separable and closed form:
//   p_j <- p_j + sigma (sum_i (2 x^k - x^{k-1})_ij - 1)                 (Eq. update:py)
//   y_i <- y_i + sigma (2 t^k_i - t^{k-1}_i - sum_j u_ij (2 x^k - x^{k-1})_ij)
//   t_i <- positive root of t^2 + (tau y_i - t^k_i) t - tau w_i = 0       (Eq. update:t)
//   x_ij <- [x^k_ij - tau (p_j - u_ij y_i)]_+                             (Eq. update:x)
// By linearity only the column sums c^k = sum_i x^k_ij (m-vector) and the row
// utilities s^k_i = sum_j u_ij x^k_ij (n-vector) of the last two iterates are
// kept, never x^{k-1} itself, so one pass over the entries per iteration reads
// u, the good id and x, and writes x and its running average.
//
// Alg. 1: K inner steps with uniform averages (weights 1 / (k + 1)), then a
// restart from the averages.  Step sizes are constant: tau = eta / omega,
// sigma = eta omega with eta = eta0_scale / ||K||_2 (K the constraint operator
// of (x, t), its norm by power iteration on K^T K) and omega = ||p^0|| /
// ||(x^0, t^0)||.  The market is preprocessed as for PDHCG (row scaling of
// Section 5, goods relabelled, rows stored bucket by bucket) and the stopping
// test is the relative KKT error of Section 5 on (x, p), of the current point
// and of the average, every kkt_check_every steps.
#include <chrono>
#include <cmath>
#include <vector>

#include "common.cuh"
#include "prep.cuh"
#include "solver.cuh"

namespace pdhcg {
namespace {

constexpr int kPdThreads = 256;

__device__ __forceinline__ double pd_hash01(long long i) {
    // deterministic start vector of the power iteration, in [0.5, 1.5)
    return 0.5 + (double)(mix32((unsigned)i * 0x9E3779B1u + 0x7F4A7C15u) >> 8) * (1.0 / 16777216.0);
}

// ---- power iteration on K^T K, K(x, t) = (C x, t - U x) ----
__global__ void pd_pow_init_kernel(long long nnz, int n, double* a, double* b) {
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < nnz; q += (long long)gridDim.x * blockDim.x)
        a[q] = pd_hash01(q);
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) b[i] = pd_hash01(nnz + i);
}
// q = C a (column sums)
__global__ void pd_colsum_kernel(long long nnz, const int* __restrict__ cj, const double* __restrict__ a, double* q) {
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < nnz; e += (long long)gridDim.x * blockDim.x)
        atomicAdd(&q[cj[e]], a[e]);
}
// z = b - U a per row (one warp per row), then a'_ij = q_j - u_ij z_i, b' = z;
// partial sums of ||(a', b')||^2 per block
__global__ void __launch_bounds__(kPdThreads) pd_pow_rows_kernel(int n, const long long* __restrict__ rp,
                                                                 const int* __restrict__ cj,
                                                                 const double* __restrict__ u, double* a, double* b,
                                                                 const double* __restrict__ q, double* part) {
    const int lane = threadIdx.x & 31;
    const long long gw = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
    const long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
    double acc = 0.0;
    for (long long i = gw; i < n; i += nw) {
        const long long e0 = rp[i], e1 = rp[i + 1];
        double ua = 0.0;
        for (long long e = e0 + lane; e < e1; e += 32) ua = fma(u[e], a[e], ua);
        ua = warp_sum_d(ua);
        const double z = b[i] - ua;
        for (long long e = e0 + lane; e < e1; e += 32) {
            const double v = q[cj[e]] - u[e] * z;
            a[e] = v;
            acc = fma(v, v, acc);
        }
        if (lane == 0) {
            b[i] = z;
            acc = fma(z, z, acc);
        }
    }
    acc = warp_sum_d(acc);
    __shared__ double red[kPdThreads / 32];
    if (lane == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < kPdThreads / 32; w++) t += red[w];
        part[blockIdx.x] = t;
    }
}
__global__ void pd_sumsq_kernel(long long nnz, int n, const double* a, const double* b, double* part) {
    double acc = 0.0;
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < nnz; q += (long long)gridDim.x * blockDim.x)
        acc = fma(a[q], a[q], acc);
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) acc = fma(b[i], b[i], acc);
    acc = warp_sum_d(acc);
    __shared__ double red[8];
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); w++) t += red[w];
        part[blockIdx.x] = t;
    }
}
__global__ void pd_scale_kernel(long long nnz, int n, double* a, double* b, double f) {
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < nnz; q += (long long)gridDim.x * blockDim.x)
        a[q] *= f;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) b[i] *= f;
}

// ---- one PDHG step ----
// prices (Eq. update:py, first line) and their running average
__global__ void pd_price_kernel(int m, double* p, double* pbar, const double* __restrict__ ck,
                                const double* __restrict__ ckm1, double* cnew, double sigma, double wgt) {
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < m; j += gridDim.x * blockDim.x) {
        const double v = p[j] + sigma * (2.0 * ck[j] - ckm1[j] - 1.0);
        p[j] = v;
        pbar[j] += wgt * (v - pbar[j]);
        cnew[j] = 0.0;
    }
}

struct PdRow {
    double* t;      // t^k per row (in: t^k, out: t^{k+1})
    double* tm1;    // t^{k-1}
    double* s;      // s^k = u_i^T x^k_i
    double* sm1;    // s^{k-1}
    double* y;
    double* tbar;
    double* ybar;
};

// one warp per buyer: y (Eq. update:py, second line), t (Eq. update:t), x
// (Eq. update:x), the new row utility and column sums, the averages
__global__ void __launch_bounds__(kPdThreads) pd_rows_kernel(int n, const long long* __restrict__ rp,
                                                             const int* __restrict__ cj,
                                                             const double* __restrict__ u,
                                                             const double* __restrict__ w, double* x, double* xbar,
                                                             const double* __restrict__ p, double* cnew, PdRow R,
                                                             double tau, double sigma, double wgt) {
    const int lane = threadIdx.x & 31;
    const long long gw = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
    const long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
    for (long long i = gw; i < n; i += nw) {
        const double tk = R.t[i], tkm1 = R.tm1[i];
        const double yn = R.y[i] + sigma * (2.0 * tk - tkm1 - (2.0 * R.s[i] - R.sm1[i]));
        const double bq = tau * yn - tk;
        const double disc = sqrt(fma(bq, bq, 4.0 * tau * w[i]));
        const double tn = bq <= 0.0 ? 0.5 * (disc - bq) : (2.0 * tau * w[i]) / (disc + bq);
        const long long e0 = rp[i], e1 = rp[i + 1];
        double sn = 0.0;
        for (long long e = e0 + lane; e < e1; e += 32) {
            const double ue = u[e];
            const int j = cj[e];
            const double xn = fmax(fma(-tau, fma(-ue, yn, p[j]), x[e]), 0.0);
            x[e] = xn;
            xbar[e] += wgt * (xn - xbar[e]);
            sn = fma(ue, xn, sn);
            if (xn > 0.0) atomicAdd(&cnew[j], xn);
        }
        sn = warp_sum_d(sn);
        if (lane == 0) {
            R.tm1[i] = tk;
            R.t[i] = tn;
            R.sm1[i] = R.s[i];
            R.s[i] = sn;
            R.y[i] = yn;
            R.tbar[i] += wgt * (tn - R.tbar[i]);
            R.ybar[i] += wgt * (yn - R.ybar[i]);
        }
    }
}

// restart (Alg. 1): the averages become the new point; x^{k-1} := x^k, so the
// row utilities and column sums of the new x are recomputed for both slots
__global__ void __launch_bounds__(kPdThreads) pd_restart_rows_kernel(int n, const long long* __restrict__ rp,
                                                                     const int* __restrict__ cj,
                                                                     const double* __restrict__ u, double* x,
                                                                     const double* __restrict__ xbar, double* c,
                                                                     PdRow R) {
    const int lane = threadIdx.x & 31;
    const long long gw = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
    const long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
    for (long long i = gw; i < n; i += nw) {
        const long long e0 = rp[i], e1 = rp[i + 1];
        double sn = 0.0;
        for (long long e = e0 + lane; e < e1; e += 32) {
            const double v = xbar[e];
            x[e] = v;
            sn = fma(u[e], v, sn);
            if (v > 0.0) atomicAdd(&c[cj[e]], v);
        }
        sn = warp_sum_d(sn);
        if (lane == 0) {
            R.t[i] = R.tbar[i];
            R.tm1[i] = R.tbar[i];
            R.s[i] = sn;
            R.sm1[i] = sn;
            R.y[i] = R.ybar[i];
        }
    }
}
// initial row utilities s^0 = u^T x^0 (t^0 = s^0, y^0 = w / t^0)
__global__ void __launch_bounds__(kPdThreads) pd_init_rows_kernel(int n, const long long* __restrict__ rp,
                                                                  const double* __restrict__ u,
                                                                  const double* __restrict__ w,
                                                                  const double* __restrict__ x, PdRow R,
                                                                  double* part) {
    const int lane = threadIdx.x & 31;
    const long long gw = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
    const long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
    double acc = 0.0;
    for (long long i = gw; i < n; i += nw) {
        const long long e0 = rp[i], e1 = rp[i + 1];
        double sn = 0.0;
        for (long long e = e0 + lane; e < e1; e += 32) {
            sn = fma(u[e], x[e], sn);
            acc = fma(x[e], x[e], acc);
        }
        sn = warp_sum_d(sn);
        if (lane == 0) {
            R.t[i] = sn;
            R.tm1[i] = sn;
            R.s[i] = sn;
            R.sm1[i] = sn;
            R.y[i] = w[i] / sn;
            R.tbar[i] = sn;
            R.ybar[i] = R.y[i];
            acc = fma(sn, sn, acc);
        }
    }
    acc = warp_sum_d(acc);
    __shared__ double red[kPdThreads / 32];
    if (lane == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int k = 0; k < kPdThreads / 32; k++) t += red[k];
        part[blockIdx.x] = t;
    }
}

}  // namespace
}  // namespace pdhcg

using namespace pdhcg;

namespace {

int pd_row_grid(int n) {
    long long g = ((long long)n * 32 + kPdThreads - 1) / kPdThreads;
    return (int)std::max<long long>(1, std::min<long long>(g, 152LL * 16));
}
int pd_vec_grid(long long n) { return (int)std::max<long long>(1, std::min<long long>((n + 255) / 256, 4096)); }

double sum_parts(const double* dpart, int nb, cudaStream_t s, cudaError_t* err) {
    std::vector<double> h(nb);
    *err = cudaMemcpyAsync(h.data(), dpart, nb * sizeof(double), cudaMemcpyDeviceToHost, s);
    if (*err == cudaSuccess) *err = cudaStreamSynchronize(s);
    double t = 0.0;
    for (double v : h) t += v;
    return t;
}

double now_ms_pd() {
    using namespace std::chrono;
    return duration<double, std::milli>(steady_clock::now().time_since_epoch()).count();
}

}  // namespace

pdhcg_status pdhcg_fisher_solve_pdhg(pdhcg_handle h, const pdhcg_market* mk, const pdhcg_params* prm,
                                     int32_t restart_every, double* p_out, double* util_out, void* x_out,
                                     pdhcg_info* info) {
    if (!h || !mk || !prm || !p_out || restart_every <= 0) return PDHCG_ERR_INVALID;
    if (!(prm->tol > 0) || prm->max_iter <= 0 || prm->kkt_check_every <= 0 || !(prm->eta0_scale > 0))
        return PDHCG_ERR_INVALID;
    enter(h);
    session_end(h);
    const double t0 = now_ms_pd();
    pdhcg_status st = prepare_market(h, mk, false, true);      // FP64; X0 = 1/deg_j (reading R10)
    if (st != PDHCG_OK) return st;
    st = alloc_iter(h);
    if (st != PDHCG_OK) return st;
    Prepared& P = h->prep;
    const int n = P.n, m = P.m;
    const long long nnz = P.nnz;
    cudaStream_t s = h->stream;
    for (int k = 0; k < 8; k++) CK(ensure(h->pd[k], (size_t)n * sizeof(double)));
    PdRow R;
    R.t = (double*)h->pd[0].p;
    R.tm1 = (double*)h->pd[1].p;
    R.s = (double*)h->pd[2].p;
    R.sm1 = (double*)h->pd[3].p;
    R.y = (double*)h->pd[4].p;
    R.tbar = (double*)h->pd[5].p;
    R.ybar = (double*)h->pd[6].p;
    double* b = (double*)h->pd[7].p;
    double* x = (double*)h->X0.p;
    double* xbar = (double*)h->Xb.p;
    double* a = (double*)h->X1.p;                  // power-iteration vector
    double* p = (double*)h->p.p;
    double* pbar = (double*)h->pbar.p;
    double* C[3] = {(double*)h->C0.p, (double*)h->C1.p, (double*)h->C2.p};
    const int rg0 = pd_row_grid(n), vg0 = pd_vec_grid(nnz);
    CK(ensure(h->pd[8], (size_t)std::max(rg0, vg0) * sizeof(double)));     // one partial per block
    double* part = (double*)h->pd[8].p;
    const long long* rp = P.dm.rp;
    const int* cj = P.dm.cj;
    const double* u = (const double*)P.dm.uv;
    const double* w = P.dm.w;
    const int rg = pd_row_grid(n), vg = pd_vec_grid(nnz);
    cudaError_t err = cudaSuccess;

    CK(cudaMemsetAsync(h->acc.p, 0, 3 * (size_t)m * sizeof(unsigned long long), s));
    CK(cudaMemsetAsync(h->M.p, 0, m * sizeof(double), s));
    CK(cudaMemsetAsync(h->ctl.p, 0, sizeof(Ctl), s));
    // initial point: x^0 = 1/deg_j, p^0 = sum(w)/m, t^0 = u^T x^0, y^0 = w/t^0
    const double sum_w = device_sum(w, n, h->part2, s);
    const double p_init = sum_w / m;
    k_fill(p, m, p_init, s);
    pd_init_rows_kernel<<<rg, kPdThreads, 0, s>>>(n, rp, u, w, x, R, part);
    const double xt2 = sum_parts(part, rg, s, &err);
    CK(err);
    const double omega = std::sqrt((double)m) * p_init / std::sqrt(xt2);
    // ||K||_2 by power iteration on K^T K
    pd_pow_init_kernel<<<vg, 256, 0, s>>>(nnz, n, a, b);
    pd_sumsq_kernel<<<vg, 256, 0, s>>>(nnz, n, a, b, part);
    double nrm2 = sum_parts(part, vg, s, &err);
    CK(err);
    double lam = 0.0;
    for (int it = 0; it < 200; it++) {
        pd_scale_kernel<<<vg, 256, 0, s>>>(nnz, n, a, b, 1.0 / std::sqrt(nrm2));     // unit v
        CK(cudaMemsetAsync(C[2], 0, m * sizeof(double), s));
        pd_colsum_kernel<<<vg, 256, 0, s>>>(nnz, cj, a, C[2]);
        pd_pow_rows_kernel<<<rg, kPdThreads, 0, s>>>(n, rp, cj, u, a, b, C[2], part);   // K^T K v
        nrm2 = sum_parts(part, rg, s, &err);
        CK(err);
        lam = std::sqrt(nrm2);            // ||K^T K v||, v unit: the largest eigenvalue in the limit
    }
    const double normK = std::sqrt(lam) * 1.01;
    const double eta = prm->eta0_scale / normK;
    const double tau = eta / omega, sigma = eta * omega;
    // c^0 = C x^0 (x^{-1} := x^0), averages start at the initial point
    CK(cudaMemsetAsync(C[0], 0, m * sizeof(double), s));
    pd_colsum_kernel<<<vg, 256, 0, s>>>(nnz, cj, x, C[0]);
    CK(cudaMemcpyAsync(C[1], C[0], m * sizeof(double), cudaMemcpyDeviceToDevice, s));
    CK(cudaMemcpyAsync(xbar, x, nnz * sizeof(double), cudaMemcpyDeviceToDevice, s));
    CK(cudaMemcpyAsync(pbar, p, m * sizeof(double), cudaMemcpyDeviceToDevice, s));
    CK(cudaGetLastError());
    const double t_setup = now_ms_pd() - t0;

    // ---- Alg. 1: inner steps, checks, restarts from the average ----
    SolveResult r;
    r.setup_ms = t_setup;
    const double t_loop0 = now_ms_pd();
    long long total = 0, inner = 0;
    int restarts = 0;
    int ck = 0, ckm1 = 1, cnew = 2;
    bool converged = false, use_avg = false;
    pdhcg_status out = PDHCG_ERR_NOT_CONVERGED;
    KktOut kcur = {}, kavg = {};
    while (total < prm->max_iter) {
        inner++;
        const double wgt = 1.0 / (double)inner;
        pd_price_kernel<<<pd_vec_grid(m), 256, 0, s>>>(m, p, pbar, C[ck], C[ckm1], C[cnew], sigma, wgt);
        pd_rows_kernel<<<rg, kPdThreads, 0, s>>>(n, rp, cj, u, w, x, xbar, p, C[cnew], R, tau, sigma, wgt);
        const int old = ckm1;
        ckm1 = ck;
        ck = cnew;
        cnew = old;
        total++;
        if (total % prm->kkt_check_every == 0 || total == prm->max_iter) {
            KktBufs k0 = kkt_bufs(h, (double*)h->c_cur.p, (double*)h->t_cur.p, 0);
            launch_kkt(false, P.dm, x, p, k0, s);
            KktBufs k1 = kkt_bufs(h, (double*)h->c_avg.p, (double*)h->t_avg.p, 1);
            launch_kkt(false, P.dm, xbar, pbar, k1, s);
            KktOut ko[2];
            CK(cudaMemcpyAsync(ko, h->kout.p, 2 * sizeof(KktOut), cudaMemcpyDeviceToHost, s));
            CK(cudaStreamSynchronize(s));
            CK(cudaGetLastError());
            kcur = ko[0];
            kavg = ko[1];
            if (!(kcur.kkt == kcur.kkt) || !(kavg.kkt == kavg.kkt)) { out = PDHCG_ERR_NUMERIC; break; }
            use_avg = kavg.kkt < kcur.kkt;
            if (prm->verbose)
                fprintf(stderr, "[pdhg] it %lld kkt cur %.3e avg %.3e restarts %d\n", total, kcur.kkt, kavg.kkt,
                        restarts);
            if ((use_avg ? kavg.kkt : kcur.kkt) <= prm->tol) { converged = true; out = PDHCG_OK; break; }
            if ((now_ms_pd() - t_loop0) * 1e-3 > prm->time_limit_s) { out = PDHCG_ERR_TIMEOUT; break; }
        }
        if (inner == restart_every) {
            // restart from the averages (x^{-1} := x^0 of the new loop)
            CK(cudaMemcpyAsync(p, pbar, m * sizeof(double), cudaMemcpyDeviceToDevice, s));
            CK(cudaMemsetAsync(C[ck], 0, m * sizeof(double), s));
            pd_restart_rows_kernel<<<rg, kPdThreads, 0, s>>>(n, rp, cj, u, x, xbar, C[ck], R);
            CK(cudaMemcpyAsync(C[ckm1], C[ck], m * sizeof(double), cudaMemcpyDeviceToDevice, s));
            inner = 0;
            restarts++;
        }
    }
    CK(cudaStreamSynchronize(s));
    CK(cudaGetLastError());
    r.use_avg = use_avg;
    r.converged = converged;
    r.x = use_avg ? (void*)xbar : (void*)x;
    r.p = use_avg ? pbar : p;
    r.t = use_avg ? (double*)h->t_avg.p : (double*)h->t_cur.p;     // u^T x of the returned point (KKT pass)
    r.kkt = use_avg ? kavg : kcur;
    r.iters = r.passes = total;
    r.restarts = restarts;
    r.solve_ms = now_ms_pd() - t_loop0;
    pdhcg_status wst = write_outputs(h, r, p_out, util_out, x_out);
    if (wst != PDHCG_OK) return wst;
    // the equilibrium is the same whatever solver found it: backward may use it
    h->state.valid = (out == PDHCG_OK);
    h->state.kind = 0;
    h->state.res = r;
    fill_info(info, r, P, out);
    return out;
}
