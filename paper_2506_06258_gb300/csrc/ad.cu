// Arrow-Debreu exchange market by the fixed-point iteration of Alg. 4
// (Section 4): w^{k+1} = E p(w^k), where p(w) is the Fisher equilibrium price
// vector for budgets w (unique, Fact 1).  Each round is one Fisher solve of the
// already preprocessed market (the structure of U does not change, only w),
// warm-started from the previous round's allocation and prices.  Because
// sum_i e_ij = 1 and sum p = sum w (Fact 1), sum w is invariant; the new
// budgets are rescaled to the initial sum to remove the drift that inexact
// inner solves leave.  Stop: max_i |w^{k+1}_i - w^k_i| / max_i |w^k_i| < tol.
#include <cmath>
#include <vector>

#include "common.cuh"
#include "prep.cuh"
#include "solver.cuh"

using namespace pdhcg;

namespace {

// w_new = E p (caller good order), E in CSR
__global__ void e_times_p_kernel(int n, const long long* __restrict__ erp, const int* __restrict__ ecol,
                                 const double* __restrict__ eval, const double* __restrict__ p, double* __restrict__ out) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        double s = 0.0;
        for (long long q = erp[i]; q < erp[i + 1]; q++) s = fma(eval[q], p[ecol[q]], s);
        out[i] = s;
    }
}
// out_i = a_i * scale; also the per-block max |a_i - b_i| and max |b_i|
__global__ void rescale_change_kernel(int n, double* __restrict__ a, double scale, const double* __restrict__ b,
                                      double* part) {
    double mc = 0.0, mb = 0.0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        double v = a[i] * scale;
        a[i] = v;
        mc = fmax(mc, fabs(v - b[i]));
        mb = fmax(mb, fabs(b[i]));
    }
    mc = warp_max_d(mc);
    mb = warp_max_d(mb);
    __shared__ double r[32][2];
    if ((threadIdx.x & 31) == 0) { r[threadIdx.x >> 5][0] = mc; r[threadIdx.x >> 5][1] = mb; }
    __syncthreads();
    if (threadIdx.x == 0) {
        double x = 0.0, y = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); w++) { x = fmax(x, r[w][0]); y = fmax(y, r[w][1]); }
        part[2 * blockIdx.x] = x;
        part[2 * blockIdx.x + 1] = y;
    }
}

}  // namespace


pdhcg_status pdhcg_ad_solve(pdhcg_handle h, const pdhcg_market* mk, const int64_t* e_row_ptr, const int32_t* e_col,
                            const double* e_val, double outer_tol, int32_t max_outer, const pdhcg_params* prm,
                            double* p_out, double* w_out, int32_t* outer_out, pdhcg_info* info) {
    if (!h || !mk || !prm || !p_out || !(outer_tol > 0) || max_outer <= 0) return PDHCG_ERR_INVALID;
    const bool identity = (e_row_ptr == nullptr && e_col == nullptr && e_val == nullptr);
    if (!identity && (!e_row_ptr || !e_col || !e_val)) return PDHCG_ERR_INVALID;
    if (identity && mk->n != mk->m) return PDHCG_ERR_INVALID;
    const bool mixed = prm->prec == PDHCG_MIXED;
    enter(h);
    pdhcg_status st = prepare_market(h, mk, mixed, true);
    if (st != PDHCG_OK) return st;
    Prepared& P = h->prep;
    cudaStream_t s = h->stream;
    const int n = P.n, m = P.m;
    const size_t vb = mixed ? 4 : 8;
    cudaError_t err = cudaSuccess;
    const long long* erp = nullptr;
    const int* ecol = nullptr;
    const double* eval = nullptr;
    if (!identity) {
        std::vector<long long> rp0(2);
        erp = (const long long*)stage_in(h->ad_e_rp, e_row_ptr, (n + 1) * sizeof(long long), s, &err);
        CK(err);
        CK(cudaMemcpyAsync(rp0.data(), erp + n, sizeof(long long), cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        const long long ennz = rp0[0];
        if (ennz < 0) return PDHCG_ERR_INVALID;
        ecol = (const int*)stage_in(h->ad_e_col, e_col, ennz * sizeof(int), s, &err);
        eval = (const double*)stage_in(h->ad_e_val, e_val, ennz * sizeof(double), s, &err);
        CK(err);
    }
    h->tight_kappa = prm->tight_kappa;
    CK(ensure(h->ad_w, n * sizeof(double)));
    CK(ensure(h->ad_wn, n * sizeof(double)));
    CK(ensure(h->ad_p, m * sizeof(double)));
    CK(ensure(h->p0i, m * sizeof(double)));
    const double sum_w0 = device_sum((const double*)h->w.p, n, h->part2, s);
    // budgets in caller row order (ad_w); h->w holds them in the internal row order
    const int* perm = (const int*)h->perm.p;
    k_rows_to_caller(n, perm, (const double*)h->w.p, nullptr, (double*)h->ad_w.p, s);
    long long iters = 0, passes = 0, capped = 0, evals = 0;
    int restarts = 0, outer = 0;
    double solve_ms = 0.0, setup_ms = 0.0;
    SolveResult r;
    pdhcg_status out = PDHCG_ERR_NOT_CONVERGED;
    for (outer = 1; outer <= max_outer; outer++) {
        st = solve_prepared(h, *prm, outer > 1 ? (const double*)h->p0i.p : nullptr, outer > 1, &r);
        if (st != PDHCG_OK && st != PDHCG_ERR_NOT_CONVERGED) return st;
        iters += r.iters;
        passes += r.passes;
        restarts += r.restarts;
        capped += r.capped;
        evals += r.evals;
        solve_ms += r.solve_ms;
        setup_ms += r.setup_ms;
        // prices in caller order, then w_new = E p
        k_gather_goods(m, (const int*)h->rank.p, r.p, (double*)h->ad_p.p, s);
        if (identity)
            CK(cudaMemcpyAsync(h->ad_wn.p, h->ad_p.p, n * sizeof(double), cudaMemcpyDeviceToDevice, s));
        else
            e_times_p_kernel<<<(n + 255) / 256 > 4096 ? 4096 : (n + 255) / 256, 256, 0, s>>>(
                n, erp, ecol, eval, (const double*)h->ad_p.p, (double*)h->ad_wn.p);
        const double sum_wn = device_sum((const double*)h->ad_wn.p, n, h->part2, s);
        if (!(sum_wn > 0.0) || !std::isfinite(sum_wn)) return PDHCG_ERR_NUMERIC;
        const int nb = 256;
        rescale_change_kernel<<<nb, 256, 0, s>>>(n, (double*)h->ad_wn.p, sum_w0 / sum_wn, (const double*)h->ad_w.p,
                                                 (double*)h->part2.p);
        std::vector<double> part(2 * nb);
        CK(cudaMemcpyAsync(part.data(), h->part2.p, 2 * nb * sizeof(double), cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        double mc = 0.0, mb = 0.0;
        for (int b = 0; b < nb; b++) { mc = fmax(mc, part[2 * b]); mb = fmax(mb, part[2 * b + 1]); }
        const double change = mc / mb;
        if (prm->verbose) fprintf(stderr, "[pdhcg-ad] outer %d inner iters %lld kkt %.3e change %.3e\n", outer,
                                  r.iters, r.kkt.kkt, change);
        // warm start of the next round: current allocation and prices
        CK(cudaMemcpyAsync(h->p0i.p, r.p, m * sizeof(double), cudaMemcpyDeviceToDevice, s));
        if (r.x != h->X0.p) CK(cudaMemcpyAsync(h->X0.p, r.x, P.nnz * vb, cudaMemcpyDeviceToDevice, s));
        // budgets for the next round (the fixed-point map)
        CK(cudaMemcpyAsync(h->ad_w.p, h->ad_wn.p, n * sizeof(double), cudaMemcpyDeviceToDevice, s));
        k_rows_to_internal(n, perm, (const double*)h->ad_wn.p, (double*)h->w.p, s);
        if (!std::isfinite(change)) return PDHCG_ERR_NUMERIC;
        if (change < outer_tol) {
            out = (st == PDHCG_OK) ? PDHCG_OK : PDHCG_ERR_NOT_CONVERGED;
            break;
        }
    }
    if (outer > max_outer) outer = max_outer;
    // outputs: prices of the last solve (caller order), final budgets
    cudaError_t e2 = cudaSuccess;
    double* pd = (double*)out_loc(h->o_p, p_out, m * sizeof(double), &e2);
    double* wd = (double*)out_loc(h->o_u, w_out, n * sizeof(double), &e2);
    CK(e2);
    CK(cudaMemcpyAsync(pd, h->ad_p.p, m * sizeof(double), cudaMemcpyDeviceToDevice, s));
    if (wd) CK(cudaMemcpyAsync(wd, h->ad_w.p, n * sizeof(double), cudaMemcpyDeviceToDevice, s));
    CK(copy_out(p_out, pd, m * sizeof(double), s));
    CK(copy_out(w_out, wd, n * sizeof(double), s));
    CK(cudaStreamSynchronize(s));
    // the equilibrium saved for backward is that of the last Fisher solve; its
    // budgets are the previous round's (h->w now holds the next ones)
    h->state.valid = (out == PDHCG_OK) && identity;
    h->state.kind = 1;
    h->state.res = r;
    if (outer_out) *outer_out = outer;
    if (info) {
        r.iters = iters;
        r.passes = passes;
        r.restarts = restarts;
        r.capped = capped;
        r.evals = evals;
        r.solve_ms = solve_ms;
        r.setup_ms = setup_ms;
        fill_info(info, r, P, out);
    }
    return out;
}
