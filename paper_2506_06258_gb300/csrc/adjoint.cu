// Reverse-mode derivative of the equilibrium (pdhcg_fisher_backward).
//
// Derived from the KKT system of Section 3.2 (Eq. KKT-system-6..9) and Fact 1:
// on the tight graph G (edges with x_ij > 0 and p_j <= u_ij y_i (1 + kappa),
// y_i = w_i / t_i) the log-prices of goods and log y of buyers are node
// potentials v with v_j - v_i = log u_ij, and each connected component C keeps
// one free scale, fixed by sum_{j in C} p_j = sum_{i in C} w_i.  For
// f = sum_j r_j p_j + sum_i g_i t_i, with node weights h_j = r_j p_j,
// h_i = -g_i t_i, H_C = sum_C h and P_C = sum_C p:
//     df/dlog u_e = lambda_e,  B^T lambda = h - H_C pi    (pi_j = p_j / P_C)
// B being the edge-node incidence (+1 at the good, -1 at the buyer).  With
// L = B^T B (the Laplacian of G) and L z = h - H_C pi, lambda = B z, i.e.
// lambda_e = z_j - z_i.  L z = b is solved by conjugate gradients with a Jacobi
// preconditioner; L is singular along per-component constants and b is
// orthogonal to them, so CG converges to a solution whose differences are
// unique.  Then df/du_e = lambda_e / u_e on G (0 elsewhere) and
// df/dw_i = g_i t_i / w_i + H_C / P_C.
//
// Arrow-Debreu with E = I (w = p at a fixed point): with the component maps
// cg (good -> C) and cb (buyer -> C), lambda in R^K solves (I - Q) lambda = rho,
// Q[C, C'] = sum_{j in C, cb(j) = C'} pi_j, rho_C = sum_{j in C} pi_j r~_j.
// Q is row-stochastic and every component is recurrent (money is conserved per
// component), so the closed classes of Q are the weakly connected classes of
// the edges cg(j) - cb(j); each class keeps its own money at a fixed point, so
// the derivative holds it fixed: r~_j = r_j - (sum_class r p / sum_class p).
// The damped iteration lambda <- (lambda + rho + Q lambda) / 2, projected per
// class on sum_class P lambda = 0, converges; mu = r~ + lambda[cb] replaces r
// in the Fisher derivative.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "common.cuh"
#include "prep.cuh"
#include "solver.cuh"

namespace pdhcg {

struct AdjArgs {
    int n, m;
    long long nnz;
    const long long* rp;
    const int* cj;          // good id of each entry (in this derivative's good space)
    const void* uv;         // row-scaled utilities (float or double)
    int f32;
    const double* rowmax;
    const double* w;
    const void* x;          // allocation (float or double)
    const double* p;        // prices (good space)
    const double* t;        // row-scaled utilities t_i
    double kappa;
};

// ---- tight edges: x_ij > 0 and p_j <= u_ij y_i (1 + kappa) ----
__global__ void tight_kernel(AdjArgs a, int* ei, int* ej, long long* eq, unsigned long long* count,
                             unsigned long long cap) {
    const int lane = threadIdx.x & 31;
    const long long gw = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
    const long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
    for (long long i = gw; i < a.n; i += nw) {
        const double y = a.w[i] / a.t[i];
        // support: x_ij above 1e-9 of the row's largest allocation (first-order
        // iterates keep vanishing entries slightly positive for a while)
        double xm = 0.0;
        for (long long q = a.rp[i] + lane; q < a.rp[i + 1]; q += 32)
            xm = fmax(xm, a.f32 ? (double)((const float*)a.x)[q] : ((const double*)a.x)[q]);
        xm = warp_max_d(xm);
        for (long long q = a.rp[i] + lane; q < a.rp[i + 1]; q += 32) {
            const double x = a.f32 ? (double)((const float*)a.x)[q] : ((const double*)a.x)[q];
            if (!(x > 1e-9 * xm)) continue;
            const double u = a.f32 ? (double)((const float*)a.uv)[q] : ((const double*)a.uv)[q];
            const int j = a.cj[q];
            if (a.p[j] <= u * y * (1.0 + a.kappa)) {
                const unsigned long long k = atomicAdd(count, 1ull);
                if (k < cap) { ei[k] = (int)i; ej[k] = j; eq[k] = q; }
            }
        }
    }
}

// ---- connected components: min-label hooking + pointer jumping ----
__global__ void label_init_kernel(int nv, int* label) {
    for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < nv; v += gridDim.x * blockDim.x) label[v] = v;
}
__global__ void hook_kernel(int ne, int n, const int* ei, const int* ej, int* label, int* changed) {
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < ne; e += gridDim.x * blockDim.x) {
        const int a = label[ei[e]], b = label[n + ej[e]];
        if (a == b) continue;
        const int lo = min(a, b), hi = max(a, b);
        atomicMin(&label[hi], lo);
        *changed = 1;
    }
}
__global__ void jump_kernel(int nv, int* label, int* changed) {
    for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < nv; v += gridDim.x * blockDim.x) {
        int l = label[v];
        int ll = label[l];
        if (ll != l) { label[v] = ll; *changed = 1; }
    }
}

// ---- right-hand side: h - H_C pi ----
__global__ void comp_sums_kernel(int n, int m, const int* label, const double* p, const double* r,
                                 const double* g, const double* t, const double* rowmax, double* H, double* P) {
    const int nv = n + m;
    for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < nv; v += gridDim.x * blockDim.x) {
        const int c = label[v];
        if (v < n) {
            if (g) atomicAdd(&H[c], -g[v] * t[v] * rowmax[v]);
        } else {
            const int j = v - n;
            atomicAdd(&H[c], r[j] * p[j]);
            atomicAdd(&P[c], p[j]);
        }
    }
}
__global__ void rhs_kernel(int n, int m, const int* label, const double* p, const double* r, const double* g,
                           const double* t, const double* rowmax, const double* H, const double* P, double* b) {
    const int nv = n + m;
    for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < nv; v += gridDim.x * blockDim.x) {
        const int c = label[v];
        if (v < n) b[v] = g ? -g[v] * t[v] * rowmax[v] : 0.0;
        else {
            const int j = v - n;
            b[v] = r[j] * p[j] - H[c] * (P[c] > 0.0 ? p[j] / P[c] : 0.0);
        }
    }
}
__global__ void degree_kernel(int ne, int n, const int* ei, const int* ej, double* dg) {
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < ne; e += gridDim.x * blockDim.x) {
        atomicAdd(&dg[ei[e]], 1.0);
        atomicAdd(&dg[n + ej[e]], 1.0);
    }
}

// ---- CG pieces (scalars stay on the device) ----
struct CgScal {
    double rz, rz_new, pq, alpha, beta, rr, bb, rz0;
    unsigned int ticket;
    int stop;               // converged: further iterations leave z unchanged
};
__global__ void lap_kernel(int ne, int n, const int* ei, const int* ej, const double* z, double* y) {
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < ne; e += gridDim.x * blockDim.x) {
        const int i = ei[e], j = n + ej[e];
        const double d = z[i] - z[j];
        atomicAdd(&y[i], d);
        atomicAdd(&y[j], -d);
    }
}
// block partial dot products with a last-block finish; mode selects the formula
__device__ void finish_dot(double v, double* part, CgScal* S, int which) {
    v = warp_sum_d(v);
    __shared__ double red[32];
    __shared__ bool last;
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); w++) s += red[w];
        part[blockIdx.x] = s;
        __threadfence();
        last = atomicAdd(&S->ticket, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!last || threadIdx.x != 0) return;
    __threadfence();
    double s = 0.0;
    for (int b = 0; b < (int)gridDim.x; b++) s += ((volatile double*)part)[b];
    S->ticket = 0u;
    // iterations run in fixed-size graphs, so the ones after convergence must
    // leave the solution alone instead of dividing rounding noise by itself
    if (which == 0) {            // p . q  ->  alpha
        S->pq = s;
        S->alpha = (!S->stop && s > 0.0) ? S->rz / s : 0.0;
    } else if (which == 1) {     // r . z_new -> beta
        S->rz_new = s;
        if (!(s > 1e-26 * S->rz0)) S->stop = 1;
        S->beta = (!S->stop && S->rz > 0.0) ? s / S->rz : 0.0;
        S->rz = s;
    } else if (which == 2) {     // r . r
        S->rr = s;
    } else {                     // initial r . z
        S->rz = s;
        S->rz0 = s;
        S->stop = !(s > 0.0);
    }
}
__global__ void dot_pq_kernel(int nv, const double* p, const double* q, double* part, CgScal* S) {
    double v = 0.0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nv; i += gridDim.x * blockDim.x) v = fma(p[i], q[i], v);
    finish_dot(v, part, S, 0);
}
// z += alpha p; r -= alpha q; zz = r / D; partial r.zz ; q reset
__global__ void update_kernel(int nv, double* z, double* r, const double* p, double* q, const double* dg, double* zz,
                              double* part, CgScal* S) {
    const double alpha = S->alpha;
    double v = 0.0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nv; i += gridDim.x * blockDim.x) {
        z[i] = fma(alpha, p[i], z[i]);
        const double ri = fma(-alpha, q[i], r[i]);
        r[i] = ri;
        q[i] = 0.0;
        const double zi = dg[i] > 0.0 ? ri / dg[i] : 0.0;
        zz[i] = zi;
        v = fma(ri, zi, v);
    }
    finish_dot(v, part, S, 1);
}
__global__ void dir_kernel(int nv, double* p, const double* zz, CgScal* S) {
    const double beta = S->beta;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nv; i += gridDim.x * blockDim.x) p[i] = fma(beta, p[i], zz[i]);
}
__global__ void rr_kernel(int nv, const double* r, double* part, CgScal* S) {
    double v = 0.0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nv; i += gridDim.x * blockDim.x) v = fma(r[i], r[i], v);
    finish_dot(v, part, S, 2);
}
__global__ void cg_init_kernel(int nv, const double* b, double* z, double* r, double* p, double* q, const double* dg,
                               double* part, CgScal* S) {
    double v = 0.0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nv; i += gridDim.x * blockDim.x) {
        z[i] = 0.0;
        r[i] = b[i];
        q[i] = 0.0;
        const double zi = dg[i] > 0.0 ? b[i] / dg[i] : 0.0;
        p[i] = zi;
        v = fma(b[i], zi, v);
    }
    finish_dot(v, part, S, 3);
}

// ---- outputs ----
__global__ void grad_u_kernel(int ne, int n, const int* ei, const int* ej, const long long* eq, const double* z,
                              const void* uv, int f32, const double* rowmax, double* gu_int) {
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < ne; e += gridDim.x * blockDim.x) {
        const int i = ei[e];
        const long long q = eq[e];
        const double u = (f32 ? (double)((const float*)uv)[q] : ((const double*)uv)[q]) * rowmax[i];
        gu_int[q] = (z[n + ej[e]] - z[i]) / u;
    }
}
__global__ void grad_w_kernel(int n, const int* label, const double* g, const double* t, const double* rowmax,
                              const double* w, const double* H, const double* P, double* gw) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int c = label[i];
        double v = P[c] > 0.0 ? H[c] / P[c] : 0.0;
        if (g) v += g[i] * t[i] * rowmax[i] / w[i];
        gw[i] = v;
    }
}

// ---- Arrow-Debreu component system ----
// classes of components: hook the agent edges C(good j) - C(buyer of agent j)
__global__ void class_hook_kernel(int m, int n, const int* label, const int* agent_row, int* cl, int* changed) {
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < m; j += gridDim.x * blockDim.x) {
        const int a = cl[label[n + j]], b = cl[label[agent_row[j]]];
        if (a == b) continue;
        atomicMin(&cl[max(a, b)], min(a, b));
        *changed = 1;
    }
}
// per-class sums of r_j p_j and p_j, then r~_j = r_j - RP/PP of its class
__global__ void class_sums_kernel(int m, int n, const int* label, const int* cl, const double* r, const double* p,
                                  double* RP, double* PP) {
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < m; j += gridDim.x * blockDim.x) {
        const int c = cl[label[n + j]];
        atomicAdd(&RP[c], r[j] * p[j]);
        atomicAdd(&PP[c], p[j]);
    }
}
__global__ void class_center_kernel(int m, int n, const int* label, const int* cl, const double* r, const double* RP,
                                    const double* PP, double* rt) {
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < m; j += gridDim.x * blockDim.x) {
        const int c = cl[label[n + j]];
        rt[j] = r[j] - RP[c] / PP[c];
    }
}
// one damped step over component roots v: lam'_v = (lam_v + rho_v + (Q lam)_v) / 2,
// accumulating per-class sums of P_v lam'_v for the projection
__global__ void ad_step_kernel(int nv, const int* label, const int* cl, const double* P, const double* rho,
                               const double* qlam, const double* lam, double* lam_new, double* csum) {
    for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < nv; v += gridDim.x * blockDim.x) {
        if (label[v] != v) continue;
        const double nl = 0.5 * (lam[v] + rho[v] + qlam[v]);
        lam_new[v] = nl;
        atomicAdd(&csum[cl[v]], P[v] * nl);
    }
}
// projection per class; the largest change and the largest |lambda| (as bits
// of non-negative doubles, dmax[0] and dmax[1])
__global__ void ad_project_kernel(int nv, const int* label, const int* cl, const double* PPc, const double* csum,
                                  double* lam_new, const double* lam, unsigned long long* dmax) {
    for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < nv; v += gridDim.x * blockDim.x) {
        if (label[v] != v) continue;
        const int c = cl[v];
        const double nl = lam_new[v] - csum[c] / PPc[c];
        lam_new[v] = nl;
        const double d = fabs(nl - lam[v]);
        if (d > 0.0) atomicMax(&dmax[0], (unsigned long long)__double_as_longlong(d));
        if (nl != 0.0) atomicMax(&dmax[1], (unsigned long long)__double_as_longlong(fabs(nl)));
    }
}
__global__ void ad_pi_kernel(int n, int m, const int* label, const double* p, const double* P, const double* rt,
                             double* rho, double* pi) {
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < m; j += gridDim.x * blockDim.x) {
        const int c = label[n + j];
        const double v = P[c] > 0.0 ? p[j] / P[c] : 0.0;
        pi[j] = v;
        atomicAdd(&rho[c], v * rt[j]);
    }
}
// out_C = sum_{j in C} pi_j lam[cb(j)]   (agent j = good j; its buyer is row j)
__global__ void ad_q_kernel(int n, int m, const int* label, const int* agent_row, const double* pi, const double* lam,
                            double* out) {
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < m; j += gridDim.x * blockDim.x) {
        const int c = label[n + j];
        atomicAdd(&out[c], pi[j] * lam[label[agent_row[j]]]);
    }
}
__global__ void ad_mu_kernel(int n, int m, const int* label, const int* agent_row, const double* rt, const double* lam,
                             double* mu) {
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < m; j += gridDim.x * blockDim.x)
        mu[j] = rt[j] + lam[label[agent_row[j]]];
}

}  // namespace pdhcg

using namespace pdhcg;

namespace {

// Slack of the tight-edge test: the caller's, else 100 x the KKT error the
// solve reached (within [1e-9, 1e-3]): support edges are tight to about the
// KKT error, and edges that are tight only to within a wider margin belong to
// a different (nearby) equilibrium structure.
double eff_kappa(double user, double kkt) {
    if (user > 0.0) return user;
    return std::min(1e-3, std::max(1e-9, 100.0 * kkt));
}

int gsz(long long n) {
    long long b = (n + 255) / 256;
    return (int)std::max<long long>(1, std::min<long long>(b, 4096));
}


// Fisher derivative core on one (possibly block-diagonal) market.
// r, g in the derivative's good / row space; outputs grad_u (entry order of a.cj)
// and grad_w.
pdhcg_status adjoint_core(pdhcg_handle h, const AdjArgs& a, const double* r, const double* g, double* gu, double* gw,
                          int max_cg, double* cg_resid, int* n_edges, int* n_comp, int* label_out_copy) {
    cudaStream_t s = h->stream;
    const int n = a.n, m = a.m, nv = n + m;
    DevBuf* B = h->adj;
    const unsigned long long cap = (unsigned long long)std::min<long long>(a.nnz, 4LL * nv + 4096);
    CK(ensure(B[0], cap * sizeof(int)));
    CK(ensure(B[1], cap * sizeof(int)));
    CK(ensure(B[2], cap * sizeof(long long)));
    CK(ensure(B[3], 64));
    CK(ensure(B[4], (size_t)nv * sizeof(int)));
    CK(ensure(B[5], 2 * (size_t)nv * sizeof(double)));      // H, P by label
    CK(ensure(B[6], 6 * (size_t)nv * sizeof(double)));      // b z r p q zz
    CK(ensure(B[7], (size_t)nv * sizeof(double)));          // degree
    CK(ensure(B[8], 4096 * sizeof(double)));
    CK(ensure(B[9], sizeof(CgScal)));
    int* ei = (int*)B[0].p;
    int* ej = (int*)B[1].p;
    long long* eq = (long long*)B[2].p;
    unsigned long long* cnt = (unsigned long long*)B[3].p;
    int* changed = (int*)((char*)B[3].p + 16);
    int* label = (int*)B[4].p;
    double* H = (double*)B[5].p;
    double* P = H + nv;
    double* vb = (double*)B[6].p;
    double *bb = vb, *z = vb + nv, *rr = vb + 2 * (size_t)nv, *pp = vb + 3 * (size_t)nv, *qq = vb + 4 * (size_t)nv,
           *zz = vb + 5 * (size_t)nv;
    double* dg = (double*)B[7].p;
    double* part = (double*)B[8].p;
    CgScal* S = (CgScal*)B[9].p;
    CK(cudaMemsetAsync(B[3].p, 0, 64, s));
    tight_kernel<<<gsz((long long)n * 32), 256, 0, s>>>(a, ei, ej, eq, cnt, cap);
    unsigned long long ne_h = 0;
    CK(cudaMemcpyAsync(&ne_h, cnt, 8, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    CK(cudaGetLastError());
    if (ne_h > cap) return PDHCG_ERR_NUMERIC;     // far from a non-degenerate equilibrium
    const int ne = (int)ne_h;
    *n_edges = ne;
    label_init_kernel<<<gsz(nv), 256, 0, s>>>(nv, label);
    for (int round = 0; round < 200; round++) {
        CK(cudaMemsetAsync(changed, 0, 4, s));
        if (ne) hook_kernel<<<gsz(ne), 256, 0, s>>>(ne, n, ei, ej, label, changed);
        for (int jmp = 0; jmp < 4; jmp++) jump_kernel<<<gsz(nv), 256, 0, s>>>(nv, label, changed);
        int ch = 0;
        CK(cudaMemcpyAsync(&ch, changed, 4, cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        if (!ch) break;
        if (round == 199) return PDHCG_ERR_NUMERIC;
    }
    CK(cudaMemsetAsync(H, 0, 2 * (size_t)nv * sizeof(double), s));
    comp_sums_kernel<<<gsz(nv), 256, 0, s>>>(n, m, label, a.p, r, g, a.t, a.rowmax, H, P);
    rhs_kernel<<<gsz(nv), 256, 0, s>>>(n, m, label, a.p, r, g, a.t, a.rowmax, H, P, bb);
    CK(cudaMemsetAsync(dg, 0, (size_t)nv * sizeof(double), s));
    if (ne) degree_kernel<<<gsz(ne), 256, 0, s>>>(ne, n, ei, ej, dg);
    CK(cudaMemsetAsync(S, 0, sizeof(CgScal), s));
    const int nbv = std::min(gsz(nv), 1024);
    // ||b||^2 for the stopping rule
    rr_kernel<<<nbv, 256, 0, s>>>(nv, bb, part, S);
    CgScal Sh;
    CK(cudaMemcpyAsync(&Sh, S, sizeof(CgScal), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    const double bnorm2 = Sh.rr;
    cg_init_kernel<<<nbv, 256, 0, s>>>(nv, bb, z, rr, pp, qq, dg, part, S);
    double res = bnorm2 > 0.0 ? 1.0 : 0.0;
    int it = 0;
    if (bnorm2 > 0.0 && ne > 0) {
        // 32 CG iterations per captured graph, residual checked between graphs
        const int K = 32;
        cudaGraph_t graph;
        cudaGraphExec_t exec;
        CK(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
        for (int k = 0; k < K; k++) {
            lap_kernel<<<gsz(ne), 256, 0, s>>>(ne, n, ei, ej, pp, qq);
            dot_pq_kernel<<<nbv, 256, 0, s>>>(nv, pp, qq, part, S);
            update_kernel<<<nbv, 256, 0, s>>>(nv, z, rr, pp, qq, dg, zz, part, S);
            dir_kernel<<<nbv, 256, 0, s>>>(nv, pp, zz, S);
        }
        rr_kernel<<<nbv, 256, 0, s>>>(nv, rr, part, S);
        cudaMemcpyAsync(&h->host->kout[0], &S->rr, sizeof(double), cudaMemcpyDeviceToHost, s);
        CK(cudaStreamEndCapture(s, &graph));
        {
            const cudaError_t ie = cudaGraphInstantiate(&exec, graph, 0);
            if (ie != cudaSuccess) cudaGraphDestroy(graph);
            CK(ie);
        }
        for (it = 0; it < max_cg; it += K) {
            cudaError_t ce = cudaGraphLaunch(exec, s);
            if (ce == cudaSuccess) ce = cudaStreamSynchronize(s);
            if (note_error(ce, "adjoint CG") != cudaSuccess) {
                cudaGraphExecDestroy(exec);
                cudaGraphDestroy(graph);
                return PDHCG_ERR_CUDA;
            }
            res = std::sqrt(h->host->kout[0].r_primal / bnorm2);
            if (!(res > 1e-10)) break;
        }
        cudaGraphExecDestroy(exec);
        cudaGraphDestroy(graph);
    }
    *cg_resid = res;
    CK(cudaMemsetAsync(gu, 0, a.nnz * sizeof(double), s));
    if (ne) grad_u_kernel<<<gsz(ne), 256, 0, s>>>(ne, n, ei, ej, eq, z, a.uv, a.f32, a.rowmax, gu);
    grad_w_kernel<<<gsz(n), 256, 0, s>>>(n, label, g, a.t, a.rowmax, a.w, H, P, gw);
    CK(cudaGetLastError());
    // number of components (roots)
    std::vector<int> lab(nv);
    CK(cudaMemcpyAsync(lab.data(), label, nv * sizeof(int), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    int kc = 0;
    for (int v = 0; v < nv; v++) kc += lab[v] == v;
    *n_comp = kc;
    (void)label_out_copy;
    return res <= 1e-8 || ne == 0 ? PDHCG_OK : PDHCG_ERR_NOT_CONVERGED;
}

__global__ void scatter_int_kernel(int m, const int* rank, const double* src, double* dst) {
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < m; j += gridDim.x * blockDim.x) dst[rank[j]] = src[j];
}
// Arrow-Debreu budgets at the fixed point: agent j (caller row j) owns caller
// good j, so w_j = p_j, stored at internal row inv[j]
__global__ void ad_weq_kernel(int m, const int* rank, const int* inv, const double* p_int, double* w_eq) {
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < m; j += gridDim.x * blockDim.x) w_eq[inv[j]] = p_int[rank[j]];
}
__global__ void axpy_const_kernel(int m, double* v, double c) {
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < m; j += gridDim.x * blockDim.x) v[j] += c;
}
__global__ void dot2_kernel(int m, const double* a, const double* b, double* out) {
    double v = 0.0, s = 0.0;
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < m; j += gridDim.x * blockDim.x) {
        v = fma(a[j], b[j], v);
        s += b[j];
    }
    v = warp_sum_d(v);
    s = warp_sum_d(s);
    if ((threadIdx.x & 31) == 0) { atomicAdd(&out[0], v); atomicAdd(&out[1], s); }
}

}  // namespace

pdhcg_status pdhcg_fisher_backward(pdhcg_handle h, const double* grad_p, const double* grad_util, double* grad_u,
                                   double* grad_w) {
    if (!h || !grad_p || !grad_u) return PDHCG_ERR_INVALID;
    if (!h->state.valid) return PDHCG_ERR_NO_STATE;
    enter(h);
    cudaStream_t s = h->stream;
    const SavedState& st = h->state;
    cudaError_t err = cudaSuccess;
    DevBuf* B = h->adj;
    if (st.kind == 2) {
        // batched: the markets form one block-diagonal market in global ids
        const int n = h->bt_N, m = h->bt_M;
        const long long nnz = h->bt_NNZ;
        const double* gp = (const double*)stage_in(h->in_p0, grad_p, m * sizeof(double), s, &err);
        const double* gt = (const double*)stage_in(h->in_x0, grad_util, n * sizeof(double), s, &err);
        double* gu = (double*)out_loc(h->o_x, grad_u, nnz * sizeof(double), &err);
        double* gw = (double*)out_loc(h->o_u, grad_w, n * sizeof(double), &err);
        CK(err);
        CK(ensure(B[12], n * sizeof(double)));
        if (!gw) gw = (double*)B[12].p;
        AdjArgs a = {};
        a.n = n;
        a.m = m;
        a.nnz = nnz;
        a.rp = (const long long*)h->bt[21].p;
        a.cj = (const int*)h->bt[19].p;
        a.uv = h->bt[0].p;
        a.f32 = h->bt_mixed ? 1 : 0;
        a.rowmax = (const double*)h->bt[5].p;
        a.w = (const double*)h->bt[20].p;
        a.x = h->bt[18].p;
        a.p = (const double*)h->bt[22].p;
        a.t = (const double*)h->bt[23].p;
        a.kappa = eff_kappa(h->tight_kappa, h->bt_kkt_max);
        double res;
        int ne, kc;
        pdhcg_status r = adjoint_core(h, a, gp, gt, gu, gw, 200000, &res, &ne, &kc, nullptr);
        if (r != PDHCG_OK && r != PDHCG_ERR_NOT_CONVERGED) return r;
        CK(copy_out(grad_u, gu, nnz * sizeof(double), s));
        CK(copy_out(grad_w, gw, n * sizeof(double), s));
        CK(cudaStreamSynchronize(s));
        return r;
    }
    const Prepared& P = h->prep;
    const int n = P.n, m = P.m;
    const long long nnz = P.nnz;
    const double* gp = (const double*)stage_in(h->in_p0, grad_p, m * sizeof(double), s, &err);
    const double* gt = (const double*)stage_in(h->in_x0, grad_util, n * sizeof(double), s, &err);
    double* gu = (double*)out_loc(h->o_x, grad_u, nnz * sizeof(double), &err);
    double* gw = (double*)out_loc(h->o_u, grad_w, n * sizeof(double), &err);
    CK(err);
    CK(ensure(B[10], m * sizeof(double)));
    CK(ensure(B[11], n * sizeof(double)));
    CK(ensure(B[12], n * sizeof(double)));
    CK(ensure(B[13], 4 * (size_t)(n + m) * sizeof(double)));
    CK(ensure(B[17], n * sizeof(double)));
    CK(ensure(B[18], nnz * sizeof(double)));
    double* r_int = (double*)B[10].p;
    double* w_eq = (double*)B[11].p;
    // the derivative is computed in the internal row order (rows stored bucket
    // by bucket) and mapped back to the caller's rows and entries at the end
    const int* perm = (const int*)h->perm.p;
    double* gw_int = (double*)B[12].p;
    double* gu_int = (double*)B[18].p;
    double* gt_int = nullptr;
    if (gt) {
        gt_int = (double*)B[17].p;
        k_rows_to_internal(n, perm, gt, gt_int, s);
    }
    scatter_int_kernel<<<gsz(m), 256, 0, s>>>(m, (const int*)h->rank.p, gp, r_int);
    const SolveResult& R = st.res;
    if (st.kind == 1) {
        // budgets at the fixed point are the prices of the own goods: w_i = p_i
        ad_weq_kernel<<<gsz(m), 256, 0, s>>>(m, (const int*)h->rank.p, (const int*)h->inv.p, R.p, w_eq);
    } else {
        CK(cudaMemcpyAsync(w_eq, h->w.p, n * sizeof(double), cudaMemcpyDeviceToDevice, s));
    }
    AdjArgs a = {};
    a.n = n;
    a.m = m;
    a.nnz = nnz;
    a.rp = (const long long*)h->rp.p;
    a.cj = (const int*)h->cj.p;
    a.uv = h->uv.p;
    a.f32 = P.mixed ? 1 : 0;
    a.rowmax = (const double*)h->rowmax.p;
    a.w = w_eq;
    a.x = R.x;
    a.p = R.p;
    a.t = R.t;
    a.kappa = eff_kappa(h->tight_kappa, R.kkt.kkt);
    if (st.kind == 1) {
        // ---- Arrow-Debreu: replace r by mu (see the file comment) ----
        const int nv = n + m;
        CK(ensure(B[13], 8 * (size_t)nv * sizeof(double)));
        CK(ensure(B[14], 64));
        CK(ensure(B[15], m * sizeof(int)));
        CK(ensure(B[16], (size_t)nv * sizeof(int)));
        double* base = (double*)B[13].p;
        double* rt = base;                        // [m]
        double* pi = base + nv;                   // [m]
        double* rho = base + 2 * (size_t)nv;      // by component root
        double* lam = base + 3 * (size_t)nv;
        double* lamn = base + 4 * (size_t)nv;
        double* qlam = base + 5 * (size_t)nv;
        double* csum = base + 6 * (size_t)nv;     // by class root
        double* PPc = base + 7 * (size_t)nv;      // by class root (also RP during centring)
        unsigned long long* dmax = (unsigned long long*)B[14].p;
        int* changed = (int*)((char*)B[14].p + 16);
        int* cl = (int*)B[16].p;
        // components of the tight graph (one derivative pass computes them)
        double res0;
        int ne0, kc0;
        pdhcg_status r0 = adjoint_core(h, a, r_int, nullptr, gu_int, gw_int, 1, &res0, &ne0, &kc0, nullptr);
        if (r0 != PDHCG_OK && r0 != PDHCG_ERR_NOT_CONVERGED) return r0;
        const int* label = (const int*)h->adj[4].p;
        const double* Pc = (const double*)h->adj[5].p + nv;
        {
            std::vector<int> agent_row(m);
            for (int j = 0; j < m; j++) agent_row[P.rank[j]] = P.inv[j];     // internal good -> its owner's internal row
            CK(cudaMemcpyAsync(B[15].p, agent_row.data(), m * sizeof(int), cudaMemcpyHostToDevice, s));
        }
        const int* agent_row = (const int*)B[15].p;
        // closed classes of components
        label_init_kernel<<<gsz(nv), 256, 0, s>>>(nv, cl);
        for (int round = 0; round < 200; round++) {
            CK(cudaMemsetAsync(changed, 0, 4, s));
            class_hook_kernel<<<gsz(m), 256, 0, s>>>(m, n, label, agent_row, cl, changed);
            for (int jmp = 0; jmp < 4; jmp++) jump_kernel<<<gsz(nv), 256, 0, s>>>(nv, cl, changed);
            int ch = 0;
            CK(cudaMemcpyAsync(&ch, changed, 4, cudaMemcpyDeviceToHost, s));
            CK(cudaStreamSynchronize(s));
            if (!ch) break;
            if (round == 199) return PDHCG_ERR_NUMERIC;
        }
        // r~ = r - per-class (r.p / sum p)
        CK(cudaMemsetAsync(csum, 0, 2 * (size_t)nv * sizeof(double), s));
        class_sums_kernel<<<gsz(m), 256, 0, s>>>(m, n, label, cl, r_int, R.p, csum, PPc);
        class_center_kernel<<<gsz(m), 256, 0, s>>>(m, n, label, cl, r_int, csum, PPc, rt);
        // rho, pi; P per class for the projection
        CK(cudaMemsetAsync(rho, 0, (size_t)nv * sizeof(double), s));
        CK(cudaMemsetAsync(lam, 0, (size_t)nv * sizeof(double), s));
        CK(cudaMemsetAsync(PPc, 0, (size_t)nv * sizeof(double), s));
        ad_pi_kernel<<<gsz(m), 256, 0, s>>>(n, m, label, R.p, Pc, rt, rho, pi);
        class_sums_kernel<<<gsz(m), 256, 0, s>>>(m, n, label, cl, r_int, R.p, csum, PPc);   // PPc = class price totals
        // damped, projected iteration, 16 steps per captured graph
        cudaGraph_t graph;
        cudaGraphExec_t exec;
        CK(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
        cudaMemsetAsync(dmax, 0, 16, s);
        for (int k = 0; k < 16; k++) {
            cudaMemsetAsync(qlam, 0, (size_t)nv * sizeof(double), s);
            cudaMemsetAsync(csum, 0, (size_t)nv * sizeof(double), s);
            ad_q_kernel<<<gsz(m), 256, 0, s>>>(n, m, label, agent_row, pi, lam, qlam);
            ad_step_kernel<<<gsz(nv), 256, 0, s>>>(nv, label, cl, Pc, rho, qlam, lam, lamn, csum);
            if (k == 15) cudaMemsetAsync(dmax, 0, 16, s);
            ad_project_kernel<<<gsz(nv), 256, 0, s>>>(nv, label, cl, PPc, csum, lamn, lam, dmax);
            cudaMemcpyAsync(lam, lamn, (size_t)nv * sizeof(double), cudaMemcpyDeviceToDevice, s);
        }
        cudaMemcpyAsync(&h->host->kout[0], dmax, 16, cudaMemcpyDeviceToHost, s);
        CK(cudaStreamEndCapture(s, &graph));
        {
            const cudaError_t ie = cudaGraphInstantiate(&exec, graph, 0);
            if (ie != cudaSuccess) cudaGraphDestroy(graph);
            CK(ie);
        }
        bool ok = false;
        for (int it = 0; it < 40000; it += 16) {
            cudaError_t ce = cudaGraphLaunch(exec, s);
            if (ce == cudaSuccess) ce = cudaStreamSynchronize(s);
            if (note_error(ce, "adjoint fixed point") != cudaSuccess) break;
            double d, lmax;
            memcpy(&d, &h->host->kout[0], 8);
            memcpy(&lmax, (const char*)&h->host->kout[0] + 8, 8);
            // the last step changed lambda by at most 1e-13 of its size
            if (!(d > 1e-13 * std::max(1.0, lmax))) { ok = true; break; }
        }
        cudaGraphExecDestroy(exec);
        cudaGraphDestroy(graph);
        if (!ok) return PDHCG_ERR_NOT_CONVERGED;
        ad_mu_kernel<<<gsz(m), 256, 0, s>>>(n, m, label, agent_row, rt, lam, r_int);
        CK(cudaGetLastError());
    }
    double res;
    int ne, kc;
    pdhcg_status r = adjoint_core(h, a, r_int, gt_int, gu_int, gw_int, 200000, &res, &ne, &kc, nullptr);
    if (r != PDHCG_OK && r != PDHCG_ERR_NOT_CONVERGED) return r;
    k_entries(n, perm, (const long long*)h->urp.p, (const long long*)h->rp.p, gu_int, gu, 8, true, s);
    if (gw) k_rows_to_caller(n, perm, gw_int, nullptr, gw, s);
    CK(copy_out(grad_u, gu, nnz * sizeof(double), s));
    if (gw) CK(copy_out(grad_w, gw, n * sizeof(double), s));
    CK(cudaStreamSynchronize(s));
    return r;
}
