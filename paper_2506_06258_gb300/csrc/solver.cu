// Host driver and C ABI of libpdhcg.so (declared in include/pdhcg.h).
//
// pdhcg_fisher_solve runs Alg. 2 (restarted PDHCG) with the Section 5
// enhancements:
//   preprocessing   validation (Assumption 1), row scaling, relabelling of
//                   goods by degree, row buckets by degree        (once, device)
//   chunk           one CUDA graph: K_chk accepted iterations of
//                   [price, prox, dual] (+ slack passes for rejected steps),
//                   the average flush, the KKT of the current point and of the
//                   average, and a device->host copy of 2 KktOut + Ctl
//   host decision   termination on the relative KKT error, adaptive restart
//                   (beta_suff 0.2, beta_nec 0.8, beta_art 0.2) and the primal
//                   weight update (theta 0.2, range check every 3 restarts)
// The step-size rule runs on the device after every pass (dual kernel).
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <vector>

#include "common.cuh"
#include "prep.cuh"
#include "solver.cuh"

using namespace pdhcg;

// ---------------------------------------------------------------------------
// small utilities
// ---------------------------------------------------------------------------
namespace pdhcg {

static thread_local char g_last_error[512] = "no error";

cudaError_t note_error(cudaError_t e, const char* what) {
    if (e != cudaSuccess) {
        snprintf(g_last_error, sizeof(g_last_error), "%s (%s) in %s", cudaGetErrorString(e), cudaGetErrorName(e), what);
        cudaGetLastError();   // clear a non-sticky error so the next call starts clean
    }
    return e;
}

cudaError_t ensure(DevBuf& b, size_t bytes) {
    if (bytes == 0) bytes = 16;
    if (b.cap >= bytes) return cudaSuccess;
    if (b.p) cudaFree(b.p);
    b.p = nullptr;
    b.cap = 0;
    cudaError_t e = cudaMalloc(&b.p, bytes);
    if (e == cudaSuccess) b.cap = bytes;
    return e;
}

bool is_device_ptr(const void* p) {
    if (!p) return false;
    cudaPointerAttributes a;
    cudaError_t e = cudaPointerGetAttributes(&a, p);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// Make `src` (host or device) available on the device; returns the device pointer.
const void* stage_in(DevBuf& buf, const void* src, size_t bytes, cudaStream_t s, cudaError_t* err) {
    if (!src) return nullptr;
    if (is_device_ptr(src)) return src;
    cudaError_t e = ensure(buf, bytes);
    if (e == cudaSuccess) e = cudaMemcpyAsync(buf.p, src, bytes, cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) {
        *err = e;
        return nullptr;
    }
    return buf.p;
}

// Device location for an output; copy_out() moves it to the caller afterwards.
void* out_loc(DevBuf& buf, void* dst, size_t bytes, cudaError_t* err) {
    if (!dst) return nullptr;
    if (is_device_ptr(dst)) return dst;
    cudaError_t e = ensure(buf, bytes);
    if (e != cudaSuccess) {
        *err = e;
        return nullptr;
    }
    return buf.p;
}
cudaError_t copy_out(void* dst, const void* loc, size_t bytes, cudaStream_t s) {
    if (!dst || dst == loc) return cudaSuccess;
    return cudaMemcpyAsync(dst, loc, bytes, cudaMemcpyDeviceToHost, s);
}

__global__ void sum_kernel(const double* a, long long n, double* part) {
    double s = 0.0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) s += a[i];
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
__global__ void chunk_begin_kernel(Ctl* ctl) {
    if (!ctl->nan_flag) ctl->active = 1;
    ctl->chunk_acc = 0;
}

double device_sum(const double* a, long long n, DevBuf& scratch, cudaStream_t s) {
    const int nb = 256;
    ensure(scratch, nb * sizeof(double));
    sum_kernel<<<nb, 256, 0, s>>>(a, n, (double*)scratch.p);
    std::vector<double> h(nb);
    cudaMemcpyAsync(h.data(), scratch.p, nb * sizeof(double), cudaMemcpyDeviceToHost, s);
    cudaStreamSynchronize(s);
    double t = 0.0;
    for (double v : h) t += v;
    return t;
}

}  // namespace pdhcg

static double now_ms() {
    using namespace std::chrono;
    return duration<double, std::milli>(steady_clock::now().time_since_epoch()).count();
}


// ---------------------------------------------------------------------------
// preprocessing (step a0): validation, row scaling, relabelling, buckets
// ---------------------------------------------------------------------------
pdhcg_status prepare_market(pdhcg_handle h, const pdhcg_market* mk, bool mixed, bool init_x) {
    cudaStream_t s = h->stream;
    if (!mk || mk->n <= 0 || mk->m <= 0 || mk->nnz <= 0 || !mk->row_ptr || !mk->col || !mk->val || !mk->w)
        return PDHCG_ERR_INVALID;
    Prepared& P = h->prep;
    h->state.valid = false;          // the buffers of a saved equilibrium are about to be reused
    const int n = mk->n, m = mk->m;
    const long long nnz = mk->nnz;
    const bool f32 = mk->val_type == PDHCG_VAL_F32;
    cudaError_t err = cudaSuccess;
    const long long* rp = (const long long*)stage_in(h->in_rp, mk->row_ptr, (n + 1) * sizeof(long long), s, &err);
    const int* col = (const int*)stage_in(h->in_col, mk->col, nnz * sizeof(int), s, &err);
    const void* val = stage_in(h->in_val, mk->val, nnz * (f32 ? 4 : 8), s, &err);
    const double* w = (const double*)stage_in(h->in_w, mk->w, n * sizeof(double), s, &err);
    CK(err);
    // our own copy of the caller's row_ptr (the caller's buffers are not kept):
    // outputs per entry are mapped back through it
    CK(ensure(h->urp, (n + 1) * sizeof(long long)));
    CK(cudaMemcpyAsync(h->urp.p, rp, (n + 1) * sizeof(long long), cudaMemcpyDeviceToDevice, s));
    // validation
    CK(ensure(h->err, 16));
    CK(cudaMemsetAsync(h->err.p, 0, 16, s));
    k_validate(n, m, nnz, rp, col, val, f32 ? 1 : 0, w, (unsigned int*)h->err.p, s);
    CK(ensure(h->deg, m * sizeof(int)));
    CK(cudaMemsetAsync(h->deg.p, 0, m * sizeof(int), s));
    k_col_degree(nnz, col, m, (int*)h->deg.p, s);
    unsigned int errh = 0;
    std::vector<int> deg(m);
    std::vector<long long> rph(n + 1);
    CK(cudaMemcpyAsync(&errh, h->err.p, sizeof(unsigned int), cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(deg.data(), h->deg.p, m * sizeof(int), cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(rph.data(), rp, (n + 1) * sizeof(long long), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    if (errh) {
        h->last_err = errh;
        return PDHCG_ERR_INVALID;
    }
    for (int j = 0; j < m; j++)
        if (deg[j] == 0) {
            h->last_err = ERR_EMPTY_COL;
            return PDHCG_ERR_INVALID;
        }
    // goods by decreasing degree: rank[j] = internal id of caller good j
    std::vector<int> order(m);
    for (int j = 0; j < m; j++) order[j] = j;
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return deg[a] > deg[b]; });
    P.rank.assign(m, 0);
    P.deg_int.assign(m, 0);
    for (int r = 0; r < m; r++) {
        P.rank[order[r]] = r;
        P.deg_int[r] = deg[order[r]];
    }
    CK(ensure(h->rank, m * sizeof(int)));
    CK(cudaMemcpyAsync(h->rank.p, P.rank.data(), m * sizeof(int), cudaMemcpyHostToDevice, s));
    DevMarket& D = P.dm;
    D = DevMarket{};
    D.n = n;
    D.m = m;
    D.nnz = nnz;
    D.nb = 0;
    D.mixed = mixed ? 1 : 0;
    // rows stored bucket by bucket (caller order within a bucket): internal row
    // r is caller row perm[r], so the row kernel, which solves one bucket after
    // another, streams the arrays in memory order
    std::vector<int> perm;
    {
        // rows by degree bucket
        const int caps[4] = {4 * kSlots, 8 * kSlots, 16 * kSlots, 32 * kSlots};
        const int gs[4] = {4, 8, 16, 32};
        std::vector<long long> cnt(5, 0);
        std::vector<unsigned char> bk(n);
        for (int i = 0; i < n; i++) {
            long long d = rph[i + 1] - rph[i];
            int b = 4;
            for (int q = 0; q < 4; q++)
                if (d <= caps[q]) { b = q; break; }
            bk[i] = (unsigned char)b;
            cnt[b]++;
        }
        std::vector<long long> start(5, 0);
        for (int b = 1; b < 5; b++) start[b] = start[b - 1] + cnt[b - 1];
        perm.assign(n, 0);
        {
            std::vector<long long> pos = start;
            for (int i = 0; i < n; i++) perm[pos[bk[i]]++] = i;
        }
        for (int b = 0; b < 5; b++) {
            if (!cnt[b]) continue;
            Bucket B;
            B.g = b < 4 ? gs[b] : 32;
            B.chunks = b < 4 ? 0 : 1;
            B.first = start[b];
            B.count = cnt[b];
            D.buckets[D.nb++] = B;
        }
    }
    P.inv.assign(n, 0);
    for (int r = 0; r < n; r++) P.inv[perm[r]] = r;
    std::vector<long long> irp(n + 1);
    irp[0] = 0;
    for (int r = 0; r < n; r++) irp[r + 1] = irp[r] + (rph[perm[r] + 1] - rph[perm[r]]);
    CK(ensure(h->perm, n * sizeof(int)));
    CK(ensure(h->inv, n * sizeof(int)));
    CK(ensure(h->rp, (n + 1 + 2) * sizeof(long long)));   // +2: bulk copies read whole 16-byte pairs
    CK(ensure(h->w, (n + 2) * sizeof(double)));
    CK(cudaMemcpyAsync(h->perm.p, perm.data(), n * sizeof(int), cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(h->inv.p, P.inv.data(), n * sizeof(int), cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(h->rp.p, irp.data(), (n + 1) * sizeof(long long), cudaMemcpyHostToDevice, s));
    k_rows_to_internal(n, (const int*)h->perm.p, w, (double*)h->w.p, s);
    if (mixed) {
        CK(ensure(h->wff, (n + 2) * sizeof(float2)));
        k_w_to_ff(n, (const double*)h->w.p, (float2*)h->wff.p, s);
    }
    // scaled utilities, relabelled goods, initial x
    const size_t vb = mixed ? 4 : 8;
    CK(ensure(h->cj, (nnz + kPadEntries) * sizeof(int)));
    CK(ensure(h->uv, (nnz + kPadEntries) * vb));
    CK(ensure(h->rowmax, n * sizeof(double)));
    CK(ensure(h->X0, (nnz + kPadEntries) * vb));
    CK(ensure(h->degint, m * sizeof(int)));
    CK(cudaMemcpyAsync(h->degint.p, P.deg_int.data(), m * sizeof(int), cudaMemcpyHostToDevice, s));
    k_scale(mixed, n, rp, col, val, f32 ? 1 : 0, (const int*)h->rank.p, (const int*)h->deg.p,
            (const int*)h->inv.p, (const long long*)h->rp.p, (double*)h->rowmax.p, h->uv.p, (int*)h->cj.p, h->X0.p,
            init_x ? 1 : 0, s);
    CK(cudaGetLastError());
    D.rp = (const long long*)h->rp.p;
    D.cj = (const int*)h->cj.p;
    D.uv = h->uv.p;
    D.w = (const double*)h->w.p;
    D.wff = mixed ? (const float2*)h->wff.p : nullptr;
    // hot goods in shared memory: as many as fit, but flushing them (blocks x
    // hot atomics) must stay small against nnz
    long long hot = std::min<long long>(m, mixed ? 4096 : 8192);
    long long lim = nnz / (8LL * prox_blocks(mixed, (int)hot));
    if (hot > lim) hot = lim;
    if (hot < 0) hot = 0;
    D.hot = (int)hot;
    D.nprox = prox_blocks(mixed, D.hot);
    // ||K||_2 = sqrt(max_j deg_j) for the column-sum operator on supp U
    int maxdeg = P.deg_int[0];
    P.normK = std::sqrt((double)maxdeg);
    double inv_deg_sum = 0.0;
    for (int j = 0; j < m; j++) inv_deg_sum += 1.0 / (double)deg[j];
    P.x0_norm = std::sqrt(inv_deg_sum);          // ||x^0|| with x_ij = 1/deg_j
    P.n = n;
    P.m = m;
    P.nnz = nnz;
    P.mixed = mixed;
    P.ready = true;
    return PDHCG_OK;
}

// ---------------------------------------------------------------------------
// iteration workspace
// ---------------------------------------------------------------------------
pdhcg_status alloc_iter(pdhcg_handle h) {
    Prepared& P = h->prep;
    const size_t vb = P.mixed ? 4 : 8;
    const int m = P.m, n = P.n;
    const long long nnz = P.nnz;
    CK(ensure(h->X1, (nnz + kPadEntries) * vb));
    CK(ensure(h->Xb, (nnz + kPadEntries) * vb));
    CK(ensure(h->Xr, (nnz + kPadEntries) * vb));
    DevBuf* gv[] = {&h->p, &h->pc, &h->pbar, &h->prs, &h->C0, &h->C1, &h->C2, &h->c_cur, &h->c_avg, &h->M};
    for (DevBuf* b : gv) CK(ensure(*b, m * sizeof(double)));
    CK(ensure(h->pff, m * sizeof(float2)));
    CK(ensure(h->acc, 3 * (size_t)m * sizeof(unsigned long long)));
    CK(ensure(h->t, (n + 2) * sizeof(double)));   // +2: read by 16-byte bulk copies
    CK(ensure(h->t_cur, n * sizeof(double)));
    CK(ensure(h->t_avg, n * sizeof(double)));
    CK(ensure(h->part, std::max(max_prox_blocks(), dist_blocks()) * sizeof(double)));
    CK(ensure(h->part2, 2 * 1024 * sizeof(double)));
    CK(ensure(h->kpart, kkt_blocks() * sizeof(KktPart)));
    CK(ensure(h->ndpart, kkt_blocks() * sizeof(float)));
    CK(ensure(h->pff_p, m * sizeof(float2)));
    CK(ensure(h->pff_pb, m * sizeof(float2)));
    CK(ensure(h->gpart, 4 * 64 * sizeof(double)));
    CK(ensure(h->ctl, sizeof(Ctl)));
    CK(ensure(h->kout, 2 * sizeof(KktOut)));
    if (!h->host) {
        CK(cudaMallocHost((void**)&h->host, sizeof(HostMirror)));
        memset(h->host, 0, sizeof(HostMirror));
    }
    return PDHCG_OK;
}

static IterBufs iter_bufs(pdhcg_handle h) {
    IterBufs b = {};
    b.X[0] = h->X0.p;
    b.X[1] = h->X1.p;
    b.Xb = h->Xb.p;
    b.p = (double*)h->p.p;
    b.pc = (double*)h->pc.p;
    b.pff = (float2*)h->pff.p;
    b.pbar = (double*)h->pbar.p;
    b.C[0] = (double*)h->C0.p;
    b.C[1] = (double*)h->C1.p;
    b.C[2] = (double*)h->C2.p;
    b.acc = (unsigned long long*)h->acc.p;
    b.t = (double*)h->t.p;
    b.yst = h->prep.mixed ? (float2*)h->t.p : nullptr;   // MIXED keeps y = w / s in the same buffer
    b.part = (double*)h->part.p;
    b.part2 = (double*)h->part2.p;
    b.pff_p = h->prep.mixed ? (float2*)h->pff_p.p : nullptr;
    b.pff_pb = h->prep.mixed ? (float2*)h->pff_pb.p : nullptr;
    return b;
}

KktBufs kkt_bufs(pdhcg_handle h, double* c_out, double* t_out, int slot) {
    KktBufs k = {};
    k.acc = (unsigned long long*)h->acc.p;
    k.M = (unsigned long long*)h->M.p;
    k.c_out = c_out;
    k.t_out = t_out;
    k.part = (KktPart*)h->kpart.p;
    k.gpart = (double*)h->gpart.p;
    k.out = (KktOut*)h->kout.p + slot;
    k.ctl = (Ctl*)h->ctl.p;
    k.nd_part = (float*)h->ndpart.p;
    k.pff = slot == 0 ? (const float2*)h->pff_p.p : (const float2*)h->pff_pb.p;
    return k;
}

// Warm start of the row kernel from the utilities t_cur of the current point:
// FP64 keeps s = t, MIXED keeps y = w / t as float-float.
static void set_row_state(pdhcg_handle h, cudaStream_t s) {
    const Prepared& P = h->prep;
    if (P.mixed) k_t_to_y(P.n, (const double*)h->w.p, (const double*)h->t_cur.p, (float2*)h->t.p, s);
    else cudaMemcpyAsync(h->t.p, h->t_cur.p, P.n * sizeof(double), cudaMemcpyDeviceToDevice, s);
}

// restart test of Section 5 (PDLP/PDHCG adaptive restarts)
static bool restart_decision(double kc, double k_rs, double k_prev, long long inner, long long total,
                             const pdhcg_params& prm) {
    if (kc <= prm.beta_suff * k_rs) return true;
    if (kc <= prm.beta_nec * k_rs && kc > k_prev) return true;
    if ((double)inner >= prm.beta_art * (double)total) return true;
    return false;
}

// ---------------------------------------------------------------------------
// the iteration loop on a prepared market; w already on the device (h->w)
// ---------------------------------------------------------------------------
void session_end(pdhcg_handle h) {
    Session& S = h->sess;
    if (S.exec) cudaGraphExecDestroy(S.exec);
    if (S.graph) cudaGraphDestroy(S.graph);
    S.exec = nullptr;
    S.graph = nullptr;
    for (int i = 0; i < S.n_ev; i++) cudaEventDestroy(S.ev[i]);
    S.n_ev = 0;
    S.active = false;
}

pdhcg_status session_begin(pdhcg_handle h, const pdhcg_params& prm, const double* p0_int_dev) {
    session_end(h);
    cudaStream_t s = h->stream;
    Prepared& P = h->prep;
    Session& S = h->sess;
    S = Session();
    S.prm = prm;
    const bool mixed = P.mixed;
    const int m = P.m, n = P.n;
    const long long nnz = P.nnz;
    pdhcg_status st = alloc_iter(h);
    if (st != PDHCG_OK) return st;
    const double t0 = now_ms();
    // budgets as float-float for the MIXED row kernel (the Arrow-Debreu loop
    // changes h->w between solves)
    if (mixed) k_w_to_ff(n, (const double*)h->w.p, (float2*)h->wff.p, s);
    const double sum_w = device_sum((const double*)h->w.p, n, h->part2, s);
    // initial point (reading: x_ij = 1/deg_j, p_j = sum(w)/m; omega_0 = ||p0||/||x0||)
    const double p_init = sum_w / m;
    if (p0_int_dev) CK(cudaMemcpyAsync(h->p.p, p0_int_dev, m * sizeof(double), cudaMemcpyDeviceToDevice, s));
    else k_fill((double*)h->p.p, m, p_init, s);
    S.omega0 = (std::sqrt((double)m) * p_init) / P.x0_norm;
    S.omega = S.omega0;
    const double eta0 = prm.eta0_scale / P.normK;
    const size_t vb = mixed ? 4 : 8;
    CK(cudaMemcpyAsync(h->pbar.p, h->p.p, m * sizeof(double), cudaMemcpyDeviceToDevice, s));
    CK(cudaMemcpyAsync(h->prs.p, h->p.p, m * sizeof(double), cudaMemcpyDeviceToDevice, s));
    CK(cudaMemcpyAsync(h->Xr.p, h->X0.p, nnz * vb, cudaMemcpyDeviceToDevice, s));
    CK(cudaMemsetAsync(h->acc.p, 0, 3 * (size_t)m * sizeof(unsigned long long), s));
    CK(cudaMemsetAsync(h->M.p, mixed ? 0x7f : 0, m * sizeof(double), s));
    if (mixed) {
        launch_to_ff(m, (const double*)h->p.p, (float2*)h->pff_p.p, s);
        launch_to_ff(m, (const double*)h->p.p, (float2*)h->pff_pb.p, s);
    }
    Ctl c0 = {};
    c0.eta = eta0;
    c0.omega = S.omega0;
    c0.eta0 = eta0;
    c0.eta_min = prm.eta_lo * eta0;
    c0.eta_max_abs = prm.eta_hi * eta0;
    c0.tau = eta0 / S.omega0;
    c0.sigma = eta0 * S.omega0;
    c0.cur = 0;
    c0.ck = 0;
    c0.ckm1 = 1;
    c0.cnew = 2;
    c0.active = 1;
    c0.chunk_quota = prm.kkt_check_every;
    c0.row_cap = prm.row_solve_max_iter;
    c0.sections = mixed ? 0 : prm.section_count;     // the K-section search is an FP64 row solve
    c0.sec_tol = prm.section_tol > 0 ? prm.section_tol : 1e-8;
    CK(cudaMemcpyAsync(h->ctl.p, &c0, sizeof(Ctl), cudaMemcpyHostToDevice, s));
    IterBufs bf = iter_bufs(h);
    Ctl* ctl = (Ctl*)h->ctl.p;
    // initial column sums and KKT of the starting point
    KktBufs kc = kkt_bufs(h, (double*)h->c_cur.p, (double*)h->t_cur.p, 0);
    launch_kkt(mixed, P.dm, h->X0.p, (const double*)h->p.p, kc, s);
    // utilities of the starting point: the row kernel's warm start y_0 = w / t
    set_row_state(h, s);
    CK(cudaMemcpyAsync(h->C0.p, h->c_cur.p, m * sizeof(double), cudaMemcpyDeviceToDevice, s));
    CK(cudaMemcpyAsync(h->C1.p, h->c_cur.p, m * sizeof(double), cudaMemcpyDeviceToDevice, s));
    CK(cudaMemcpyAsync(&h->host->kout[0], h->kout.p, sizeof(KktOut), cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(&h->host->ctl, h->ctl.p, sizeof(Ctl), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    CK(cudaGetLastError());
    S.kkt_rs = h->host->kout[0].kkt;
    S.kkt_prev = INFINITY;
    S.best = h->host->kout[0];
    // ---- capture one chunk ----
    const int slack = 8;
    const int passes = prm.kkt_check_every + slack;
    const bool timing = prm.timing && passes <= 80;
    if (timing) {
        S.n_ev = 2 * passes + 2;
        for (int i = 0; i < S.n_ev; i++) CK(cudaEventCreate(&S.ev[i]));
    }
    CK(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
    chunk_begin_kernel<<<1, 1, 0, s>>>(ctl);
    for (int q = 0; q < passes; q++) {
        launch_price(mixed, P.dm, bf, ctl, s);
        if (timing) cudaEventRecordWithFlags(S.ev[2 * q], s, cudaEventRecordExternal);
        launch_prox(mixed, P.dm, bf, ctl, s);
        if (timing) cudaEventRecordWithFlags(S.ev[2 * q + 1], s, cudaEventRecordExternal);
        launch_dual(mixed, P.dm, bf, ctl, s);
        launch_fold(mixed, P.dm, bf, ctl, s);
    }
    launch_flush(mixed, P.dm, bf, ctl, s);
    if (timing) cudaEventRecordWithFlags(S.ev[2 * passes], s, cudaEventRecordExternal);
    {
        KktBufs k0 = kkt_bufs(h, (double*)h->c_cur.p, (double*)h->t_cur.p, 0);
        k0.xsel[0] = h->X0.p;
        k0.xsel[1] = h->X1.p;
        k0.sel = &ctl->cur;
        launch_kkt(mixed, P.dm, nullptr, (const double*)h->p.p, k0, s);
        KktBufs k1 = kkt_bufs(h, (double*)h->c_avg.p, (double*)h->t_avg.p, 1);
        launch_kkt(mixed, P.dm, h->Xb.p, (const double*)h->pbar.p, k1, s);
    }
    if (timing) cudaEventRecordWithFlags(S.ev[2 * passes + 1], s, cudaEventRecordExternal);
    cudaMemcpyAsync(h->host->kout, h->kout.p, 2 * sizeof(KktOut), cudaMemcpyDeviceToHost, s);
    cudaMemcpyAsync(&h->host->ctl, h->ctl.p, sizeof(Ctl), cudaMemcpyDeviceToHost, s);
    cudaError_t ce = cudaStreamEndCapture(s, &S.graph);
    if (ce != cudaSuccess) return PDHCG_ERR_CUDA;
    ce = cudaGraphInstantiate(&S.exec, S.graph, 0);
    if (ce != cudaSuccess) {
        session_end(h);
        return PDHCG_ERR_CUDA;
    }
    {
        size_t nn = 0;
        cudaGraphGetNodes(S.graph, nullptr, &nn);
        std::vector<cudaGraphNode_t> nodes(nn);
        cudaGraphGetNodes(S.graph, nodes.data(), &nn);
        for (auto nd : nodes) {
            cudaGraphNodeType t;
            cudaGraphNodeGetType(nd, &t);
            if (t == cudaGraphNodeTypeKernel) S.graph_kernels++;
        }
    }
    S.t_setup = now_ms() - t0;
    S.active = true;
    S.status = PDHCG_ERR_NOT_CONVERGED;
    if (S.kkt_rs <= prm.tol) {
        S.converged = true;
        S.status = PDHCG_OK;
    }
    return PDHCG_OK;
}

// Run up to `chunks` check periods; stops early on convergence or a limit.
pdhcg_status session_step(pdhcg_handle h, long long chunks) {
    Session& S = h->sess;
    if (!S.active) return PDHCG_ERR_INVALID;
    if (S.status != PDHCG_ERR_NOT_CONVERGED) return S.status;
    cudaStream_t s = h->stream;
    Prepared& P = h->prep;
    const pdhcg_params& prm = S.prm;
    const bool mixed = P.mixed;
    const int m = P.m;
    const long long nnz = P.nnz;
    const size_t vb = mixed ? 4 : 8;
    const int passes = prm.kkt_check_every + 8;
    const double t_loop0 = now_ms();
    for (long long ch = 0; ch < chunks; ch++) {
        const long long passes_before = h->host->ctl.passes;
        cudaError_t ce = cudaGraphLaunch(S.exec, s);
        S.launches += S.graph_kernels;
        if (ce == cudaSuccess) ce = cudaStreamSynchronize(s);
        if (ce != cudaSuccess) { S.status = PDHCG_ERR_CUDA; break; }
        Ctl& c = h->host->ctl;
        if (S.n_ev) {
            float ms = 0.0f;
            for (int q = 0; q < passes; q++) {
                if (note_error(cudaEventElapsedTime(&ms, S.ev[2 * q], S.ev[2 * q + 1]), "event timing") == cudaSuccess)
                    S.prox_ms += ms;
            }
            S.prox_launches += c.passes - passes_before;
            if (note_error(cudaEventElapsedTime(&ms, S.ev[2 * passes], S.ev[2 * passes + 1]), "event timing") ==
                cudaSuccess)
                S.kkt_ms += ms;
        }
        const KktOut kcur = h->host->kout[0], kavg = h->host->kout[1];
        if (c.nan_flag || !(kcur.kkt == kcur.kkt)) {
            S.status = PDHCG_ERR_NUMERIC;
            S.use_avg = false;
            S.best = kcur;
            break;
        }
        S.use_avg = kavg.kkt < kcur.kkt;
        S.best = S.use_avg ? kavg : kcur;
        const double kc = S.best.kkt;
        if (prm.verbose)
            fprintf(stderr, "[pdhcg] it %lld passes %lld kkt cur %.3e (p %.2e d %.2e g %.2e) avg %.3e eta %.3e omega %.3e "
                    "restarts %d\n", c.iters, c.passes, kcur.kkt, kcur.r_primal, kcur.r_dual, kcur.r_gap, kavg.kkt, c.eta,
                    c.omega, S.restarts);
        if (kc <= prm.tol) { S.converged = true; S.status = PDHCG_OK; break; }
        if (c.iters >= prm.max_iter || c.passes >= 4 * prm.max_iter + 10000) {
            S.status = PDHCG_ERR_NOT_CONVERGED;
            S.t_loop += now_ms() - t_loop0;
            return PDHCG_ERR_NOT_CONVERGED;
        }
        if ((S.t_loop + now_ms() - t_loop0) * 1e-3 > prm.time_limit_s) { S.status = PDHCG_ERR_TIMEOUT; break; }
        const long long inner = c.iters - S.iters_at_restart;
        if (restart_decision(kc, S.kkt_rs, S.kkt_prev, inner, c.iters, prm)) {
            void* Xc = c.cur ? h->X1.p : h->X0.p;
            double* Cbuf[3] = {(double*)h->C0.p, (double*)h->C1.p, (double*)h->C2.p};
            const double* csrc = S.use_avg ? (const double*)h->c_avg.p : (const double*)h->c_cur.p;
            if (S.use_avg) {
                CK(cudaMemcpyAsync(Xc, h->Xb.p, nnz * vb, cudaMemcpyDeviceToDevice, s));
                CK(cudaMemcpyAsync(h->p.p, h->pbar.p, m * sizeof(double), cudaMemcpyDeviceToDevice, s));
                CK(cudaMemcpyAsync(h->t_cur.p, h->t_avg.p, P.n * sizeof(double), cudaMemcpyDeviceToDevice, s));
            }
            CK(cudaMemcpyAsync(Cbuf[c.ck], csrc, m * sizeof(double), cudaMemcpyDeviceToDevice, s));
            CK(cudaMemcpyAsync(Cbuf[c.ckm1], csrc, m * sizeof(double), cudaMemcpyDeviceToDevice, s));
            set_row_state(h, s);
            // distances to the previous restart point, then remember this one
            const int nb = dist_blocks();
            std::vector<double> pa(nb), pb(nb);
            S.launches += 2;
            k_dist_copy(mixed, nnz, Xc, h->Xr.p, (double*)h->part.p, s);
            CK(cudaMemcpyAsync(pa.data(), h->part.p, nb * sizeof(double), cudaMemcpyDeviceToHost, s));
            CK(cudaStreamSynchronize(s));
            k_dist_copy(false, m, h->p.p, h->prs.p, (double*)h->part.p, s);
            CK(cudaMemcpyAsync(pb.data(), h->part.p, nb * sizeof(double), cudaMemcpyDeviceToHost, s));
            CK(cudaStreamSynchronize(s));
            double dx2 = 0.0, dp2 = 0.0;
            for (double v : pa) dx2 += v;
            for (double v : pb) dp2 += v;
            const double dx = std::sqrt(dx2), dp = std::sqrt(dp2);
            S.restarts++;
            if (dx > 1e-300 && dp > 1e-300)
                S.omega = std::exp(prm.theta * std::log(dp / dx) + (1.0 - prm.theta) * std::log(S.omega));
            if (prm.omega_reset_every > 0 && S.restarts % prm.omega_reset_every == 0) {
                if (!(S.omega >= S.omega0 / prm.omega_range && S.omega <= S.omega0 * prm.omega_range))
                    S.omega = S.omega0;
            }
            c.omega = S.omega;
            c.tau = c.eta / S.omega;
            c.sigma = c.eta * S.omega;
            c.sum_eta = 0.0;
            c.fold_pending = 0;
            c.fold_wgt = 1.0;
            c.xf_n = 0;
            c.xf_folded = 0;
            CK(cudaMemcpyAsync(h->ctl.p, &c, sizeof(Ctl), cudaMemcpyHostToDevice, s));
            S.kkt_rs = kc;
            S.kkt_prev = INFINITY;
            S.iters_at_restart = c.iters;
            S.use_avg = false;        // the restarted point now lives in the current buffers
        } else {
            S.kkt_prev = kc;
        }
    }
    S.t_loop += now_ms() - t_loop0;
    return S.status;
}

void session_result(pdhcg_handle h, SolveResult* res) {
    Session& S = h->sess;
    const Ctl& c = h->host->ctl;
    res->use_avg = S.use_avg;
    res->x = S.use_avg ? h->Xb.p : (c.cur ? h->X1.p : h->X0.p);
    res->p = S.use_avg ? (double*)h->pbar.p : (double*)h->p.p;
    res->t = S.use_avg ? (double*)h->t_avg.p : (double*)h->t_cur.p;
    res->kkt = S.best;
    res->iters = c.iters;
    res->passes = c.passes;
    res->restarts = S.restarts;
    res->capped = c.capped;
    res->evals = c.evals;
    res->solve_ms = S.t_loop;
    res->setup_ms = S.t_setup;
    res->converged = S.converged;
    res->prox_ms = S.prox_ms;
    res->prox_launches = S.prox_launches;
    res->kkt_ms = S.kkt_ms;
    res->launches = S.launches;
}

pdhcg_status solve_prepared(pdhcg_handle h, const pdhcg_params& prm, const double* p0_int_dev, bool warm_x,
                            SolveResult* res) {
    (void)warm_x;
    pdhcg_status st = session_begin(h, prm, p0_int_dev);
    if (st != PDHCG_OK) return st;
    st = session_step(h, 1LL << 62);
    session_result(h, res);
    session_end(h);
    return st;
}

// ---------------------------------------------------------------------------
// C ABI (C linkage comes from the declarations in pdhcg.h)
// ---------------------------------------------------------------------------

const char* pdhcg_status_string(pdhcg_status s) {
    switch (s) {
        case PDHCG_OK: return "ok";
        case PDHCG_ERR_INVALID: return "invalid argument or market (Assumption 1)";
        case PDHCG_ERR_CUDA: return "CUDA error";
        case PDHCG_ERR_OOM: return "out of device memory";
        case PDHCG_ERR_NOT_CONVERGED: return "iteration limit reached before tolerance";
        case PDHCG_ERR_NUMERIC: return "non-finite value in the iterates";
        case PDHCG_ERR_TIMEOUT: return "time limit reached before tolerance";
        case PDHCG_ERR_NO_STATE: return "no saved equilibrium on this handle";
    }
    return "unknown status";
}

int32_t pdhcg_version(void) { return PDHCG_VERSION_MAJOR * 100 + PDHCG_VERSION_MINOR; }

const char* pdhcg_last_error(void) { return g_last_error; }

void pdhcg_default_params(pdhcg_params* p) {
    if (!p) return;
    memset(p, 0, sizeof(*p));
    p->tol = 1e-6;
    p->max_iter = 1000000;
    p->time_limit_s = 1e9;
    p->prec = PDHCG_MIXED;
    p->kkt_check_every = 64;
    p->beta_suff = 0.2;
    p->beta_nec = 0.8;
    p->beta_art = 0.2;
    p->theta = 0.2;
    p->eta_lo = 0.01;
    p->eta_hi = 3.0;
    p->eta0_scale = 0.9;
    p->omega_reset_every = 3;
    p->omega_range = 100.0;
    p->row_solve_max_iter = 64;
    p->tight_kappa = 0.0;
    p->verbose = 0;
}

void enter(pdhcg_handle h) {
    if (h->owns_stream) {
        cudaEventRecord(h->entry_ev, h->user_stream);
        cudaStreamWaitEvent(h->stream, h->entry_ev, 0);
    }
}

pdhcg_status pdhcg_create(pdhcg_handle* hp, void* stream) {
    if (!hp) return PDHCG_ERR_INVALID;
    pdhcg_handle h = new (std::nothrow) pdhcg_handle_s();
    if (!h) return PDHCG_ERR_OOM;
    h->user_stream = (cudaStream_t)stream;
    h->stream = h->user_stream;
    if (cudaGetDevice(&h->device) != cudaSuccess) {
        delete h;
        return PDHCG_ERR_CUDA;
    }
    if (h->user_stream == 0) {
        if (cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&h->entry_ev, cudaEventDisableTiming) != cudaSuccess) {
            delete h;
            return PDHCG_ERR_CUDA;
        }
        h->owns_stream = true;
    }
    *hp = h;
    return PDHCG_OK;
}

pdhcg_status pdhcg_destroy(pdhcg_handle h) {
    if (!h) return PDHCG_ERR_INVALID;
    cudaStreamSynchronize(h->stream);
    session_end(h);
    h->release();
    if (h->owns_stream) {
        cudaStreamDestroy(h->stream);
        cudaEventDestroy(h->entry_ev);
    }
    delete h;
    return PDHCG_OK;
}

static pdhcg_status check_params(const pdhcg_params* prm) {
    if (!prm) return PDHCG_ERR_INVALID;
    if (!(prm->tol > 0) || prm->max_iter <= 0 || prm->kkt_check_every <= 0 || prm->row_solve_max_iter <= 0)
        return PDHCG_ERR_INVALID;
    if (!(prm->eta_lo > 0) || !(prm->eta_hi >= prm->eta_lo) || !(prm->eta0_scale > 0)) return PDHCG_ERR_INVALID;
    if (prm->prec != PDHCG_FP64 && prm->prec != PDHCG_MIXED) return PDHCG_ERR_INVALID;
    if (prm->section_count < 0 || prm->section_count == 1 || prm->section_count > 1024 || prm->section_tol < 0)
        return PDHCG_ERR_INVALID;
    return PDHCG_OK;
}


// write p (caller order), utilities and x; fill info
pdhcg_status write_outputs(pdhcg_handle h, const SolveResult& r, double* p_out, double* util_out, void* x_out) {
    cudaStream_t s = h->stream;
    Prepared& P = h->prep;
    cudaError_t err = cudaSuccess;
    double* pd = (double*)out_loc(h->o_p, p_out, P.m * sizeof(double), &err);
    double* ud = (double*)out_loc(h->o_u, util_out, P.n * sizeof(double), &err);
    const size_t vb = P.mixed ? 4 : 8;
    void* xd = out_loc(h->o_x, x_out, P.nnz * vb, &err);
    CK(err);
    if (pd) k_gather_goods(P.m, (const int*)h->rank.p, r.p, pd, s);
    if (ud) k_rows_to_caller(P.n, (const int*)h->perm.p, r.t, (const double*)h->rowmax.p, ud, s);
    if (xd) k_entries(P.n, (const int*)h->perm.p, (const long long*)h->urp.p, (const long long*)h->rp.p, r.x, xd,
                      (int)vb, true, s);
    CK(copy_out(p_out, pd, P.m * sizeof(double), s));
    CK(copy_out(util_out, ud, P.n * sizeof(double), s));
    CK(copy_out(x_out, xd, P.nnz * vb, s));
    CK(cudaStreamSynchronize(s));
    return PDHCG_OK;
}

void fill_info(pdhcg_info* info, const SolveResult& r, const Prepared& P, pdhcg_status st) {
    if (!info) return;
    info->iters = r.iters;
    info->passes = r.passes;
    info->restarts = r.restarts;
    info->kkt = r.kkt.kkt;
    info->r_primal = r.kkt.r_primal;
    info->r_dual = r.kkt.r_dual;
    info->r_gap = r.kkt.r_gap;
    info->solve_ms = r.solve_ms;
    info->setup_ms = r.setup_ms;
    info->bytes_moved = (double)r.passes * (double)P.nnz * (P.mixed ? 24.0 : 44.0);
    info->row_solve_capped = (int32_t)std::min<long long>(r.capped, 2147483647LL);
    info->status = st;
    info->prox_ms = r.prox_ms;
    info->prox_launches = r.prox_launches;
    info->kkt_ms = r.kkt_ms;
    info->kernel_launches = r.launches;
    info->row_solve_evals = r.evals;
}

pdhcg_status pdhcg_fisher_begin(pdhcg_handle h, const pdhcg_market* mk, const pdhcg_params* prm,
                                const double* p0, const void* x0) {
    if (!h || !mk) return PDHCG_ERR_INVALID;
    pdhcg_status st = check_params(prm);
    if (st != PDHCG_OK) return st;
    enter(h);
    session_end(h);
    const double t0 = now_ms();
    const bool mixed = prm->prec == PDHCG_MIXED;
    st = prepare_market(h, mk, mixed, x0 == nullptr);
    if (st != PDHCG_OK) return st;
    Prepared& P = h->prep;
    cudaStream_t s = h->stream;
    cudaError_t err = cudaSuccess;
    if (x0) {
        const void* xd = stage_in(h->in_x0, x0, P.nnz * (mixed ? 4 : 8), s, &err);
        CK(err);
        k_entries(P.n, (const int*)h->perm.p, (const long long*)h->urp.p, (const long long*)h->rp.p, xd, h->X0.p,
                  mixed ? 4 : 8, false, s);
    }
    const double* p0i = nullptr;
    if (p0) {
        const double* pd = (const double*)stage_in(h->in_p0, p0, P.m * sizeof(double), s, &err);
        CK(err);
        CK(ensure(h->p0i, P.m * sizeof(double)));
        k_scatter_goods(P.m, (const int*)h->rank.p, pd, (double*)h->p0i.p, s);
        p0i = (const double*)h->p0i.p;
    }
    const double t_prep = now_ms() - t0;
    h->tight_kappa = prm->tight_kappa;
    st = session_begin(h, *prm, p0i);
    h->sess.t_setup += t_prep;
    h->state.valid = false;
    return st;
}

pdhcg_status pdhcg_fisher_step(pdhcg_handle h, int32_t chunks, pdhcg_info* info) {
    if (!h || chunks < 0) return PDHCG_ERR_INVALID;
    pdhcg_status st = session_step(h, chunks);
    if (info) {
        SolveResult r;
        session_result(h, &r);
        fill_info(info, r, h->prep, st);
    }
    return st;
}

pdhcg_status pdhcg_fisher_end(pdhcg_handle h, double* p_out, double* util_out, void* x_out, pdhcg_info* info) {
    if (!h || !h->sess.active) return PDHCG_ERR_INVALID;
    SolveResult r;
    session_result(h, &r);
    const pdhcg_status st = h->sess.status;
    session_end(h);
    if (p_out || util_out || x_out) {
        pdhcg_status wst = write_outputs(h, r, p_out, util_out, x_out);
        if (wst != PDHCG_OK) return wst;
    }
    h->state.valid = (st == PDHCG_OK);
    h->state.kind = 0;
    h->state.res = r;
    fill_info(info, r, h->prep, st);
    return st;
}

pdhcg_status pdhcg_fisher_solve(pdhcg_handle h, const pdhcg_market* mk, const pdhcg_params* prm,
                                const double* p0, const void* x0, double* p_out, double* util_out, void* x_out,
                                pdhcg_info* info) {
    if (!h || !mk || !p_out) return PDHCG_ERR_INVALID;
    pdhcg_status st = pdhcg_fisher_begin(h, mk, prm, p0, x0);
    if (st != PDHCG_OK) return st;
    st = session_step(h, 1LL << 62);
    if (st != PDHCG_OK && st != PDHCG_ERR_NOT_CONVERGED && st != PDHCG_ERR_TIMEOUT && st != PDHCG_ERR_NUMERIC) {
        session_end(h);
        return st;
    }
    return pdhcg_fisher_end(h, p_out, util_out, x_out, info);
}

pdhcg_status pdhcg_row_prox(pdhcg_handle h, const pdhcg_market* mk, pdhcg_precision prec, const void* x_in,
                            const double* p, double tau, void* x_new, double* s_out, double* c_out) {
    if (!h || !mk || !x_in || !p || !x_new || !(tau > 0)) return PDHCG_ERR_INVALID;
    if (prec != PDHCG_FP64 && prec != PDHCG_MIXED) return PDHCG_ERR_INVALID;
    const bool mixed = prec == PDHCG_MIXED;
    enter(h);
    pdhcg_status st = prepare_market(h, mk, mixed, false);
    if (st != PDHCG_OK) return st;
    st = alloc_iter(h);
    if (st != PDHCG_OK) return st;
    Prepared& P = h->prep;
    cudaStream_t s = h->stream;
    cudaError_t err = cudaSuccess;
    const size_t vb = mixed ? 4 : 8;
    const void* xi = stage_in(h->in_x0, x_in, P.nnz * vb, s, &err);
    const double* pd = (const double*)stage_in(h->in_p0, p, P.m * sizeof(double), s, &err);
    CK(err);
    CK(ensure(h->p0i, P.m * sizeof(double)));
    k_scatter_goods(P.m, (const int*)h->rank.p, pd, (double*)h->p0i.p, s);
    void* xo = out_loc(h->o_x, x_new, P.nnz * vb, &err);
    double* so = (double*)out_loc(h->o_u, s_out, P.n * sizeof(double), &err);
    double* co = (double*)out_loc(h->o_p, c_out, P.m * sizeof(double), &err);
    CK(err);
    CK(cudaMemsetAsync(h->acc.p, 0, P.m * sizeof(unsigned long long), s));
    // x in the internal row order: X0 in, X1 out
    const int* perm = (const int*)h->perm.p;
    const long long* urp = (const long long*)h->urp.p;
    k_entries(P.n, perm, urp, P.dm.rp, xi, h->X0.p, (int)vb, false, s);
    launch_prox_fixed(mixed, P.dm, h->X0.p, h->X1.p, (const double*)h->p0i.p, tau, (unsigned long long*)h->acc.p,
                      (double*)h->t.p, (double*)h->c_cur.p, (double*)h->part.p, (Ctl*)h->ctl.p, s);
    CK(cudaGetLastError());
    k_entries(P.n, perm, urp, P.dm.rp, h->X1.p, xo, (int)vb, true, s);
    if (so) {
        if (mixed) {
            k_max_scaled_t(P.n, P.dm.rp, (const float*)P.dm.uv, (const double*)h->t.p, (double*)h->t_avg.p, s);
            k_rows_to_caller(P.n, perm, (const double*)h->t_avg.p, nullptr, so, s);
        } else {
            k_rows_to_caller(P.n, perm, (const double*)h->t.p, nullptr, so, s);
        }
    }
    if (co) k_gather_goods(P.m, (const int*)h->rank.p, (const double*)h->c_cur.p, co, s);
    CK(copy_out(x_new, xo, P.nnz * vb, s));
    CK(copy_out(s_out, so, P.n * sizeof(double), s));
    CK(copy_out(c_out, co, P.m * sizeof(double), s));
    CK(cudaStreamSynchronize(s));
    return PDHCG_OK;
}

pdhcg_status pdhcg_kkt(pdhcg_handle h, const pdhcg_market* mk, pdhcg_precision prec, const void* x,
                       const double* p, double* out) {
    if (!h || !mk || !x || !p || !out) return PDHCG_ERR_INVALID;
    if (prec != PDHCG_FP64 && prec != PDHCG_MIXED) return PDHCG_ERR_INVALID;
    const bool mixed = prec == PDHCG_MIXED;
    enter(h);
    pdhcg_status st = prepare_market(h, mk, mixed, false);
    if (st != PDHCG_OK) return st;
    st = alloc_iter(h);
    if (st != PDHCG_OK) return st;
    Prepared& P = h->prep;
    cudaStream_t s = h->stream;
    cudaError_t err = cudaSuccess;
    const size_t vb = mixed ? 4 : 8;
    const void* xd = stage_in(h->in_x0, x, P.nnz * vb, s, &err);
    const double* pd = (const double*)stage_in(h->in_p0, p, P.m * sizeof(double), s, &err);
    CK(err);
    CK(ensure(h->p0i, P.m * sizeof(double)));
    k_scatter_goods(P.m, (const int*)h->rank.p, pd, (double*)h->p0i.p, s);
    CK(cudaMemsetAsync(h->acc.p, 0, P.m * sizeof(unsigned long long), s));
    CK(cudaMemsetAsync(h->M.p, mixed ? 0x7f : 0, P.m * sizeof(double), s));
    CK(cudaMemsetAsync(h->ctl.p, 0, sizeof(Ctl), s));
    if (mixed) launch_to_ff(P.m, (const double*)h->p0i.p, (float2*)h->pff_p.p, s);
    k_entries(P.n, (const int*)h->perm.p, (const long long*)h->urp.p, P.dm.rp, xd, h->X0.p, (int)vb, false, s);
    KktBufs kb = kkt_bufs(h, nullptr, nullptr, 0);
    launch_kkt(mixed, P.dm, h->X0.p, (const double*)h->p0i.p, kb, s);
    KktOut o;
    CK(cudaMemcpyAsync(&o, h->kout.p, sizeof(KktOut), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    CK(cudaGetLastError());
    out[0] = o.r_primal;
    out[1] = o.r_dual;
    out[2] = o.r_gap;
    out[3] = o.kkt;
    return PDHCG_OK;
}
