// Handle, workspace and host-side driver state shared by solver.cu, ad.cu,
// batched.cu and adjoint.cu.
#pragma once
#include <vector>

#include "common.cuh"

namespace pdhcg {

struct DevBuf {
    void* p = nullptr;
    size_t cap = 0;
    void release() {
        if (p) cudaFree(p);
        p = nullptr;
        cap = 0;
    }
};

cudaError_t ensure(DevBuf& b, size_t bytes);
// remembers the last failing CUDA call for pdhcg_last_error()
cudaError_t note_error(cudaError_t e, const char* what);

#define CK(x)                                                          \
    do {                                                               \
        cudaError_t e_ = pdhcg::note_error((x), #x);                   \
        if (e_ != cudaSuccess) {                                       \
            if (e_ == cudaErrorMemoryAllocation) return PDHCG_ERR_OOM; \
            return PDHCG_ERR_CUDA;                                     \
        }                                                              \
    } while (0)
bool is_device_ptr(const void* p);
const void* stage_in(DevBuf& buf, const void* src, size_t bytes, cudaStream_t s, cudaError_t* err);
void* out_loc(DevBuf& buf, void* dst, size_t bytes, cudaError_t* err);
cudaError_t copy_out(void* dst, const void* loc, size_t bytes, cudaStream_t s);
double device_sum(const double* a, long long n, DevBuf& scratch, cudaStream_t s);

// Market after preprocessing (step a0).
struct Prepared {
    bool ready = false;
    bool mixed = true;
    int n = 0, m = 0;
    long long nnz = 0;
    DevMarket dm;
    std::vector<int> rank;      // caller good j -> internal id
    std::vector<int> deg_int;   // column degree by internal id
    std::vector<int> inv;       // caller row i -> internal row (rows stored bucket by bucket)
    double normK = 1.0;         // ||K||_2 = sqrt(max_j deg_j)
    double x0_norm = 1.0;       // ||x^0||_2 for x_ij = 1/deg_j
};

struct SolveResult {
    bool use_avg = false;
    bool converged = false;
    void* x = nullptr;      // internal buffers holding the returned point
    double* p = nullptr;
    double* t = nullptr;
    KktOut kkt = {};
    long long iters = 0, passes = 0, capped = 0, evals = 0;
    int restarts = 0;
    double solve_ms = 0.0, setup_ms = 0.0;
    double prox_ms = 0.0, kkt_ms = 0.0;
    long long prox_launches = 0;
    long long launches = 0;
};

struct HostMirror {     // pinned
    KktOut kout[2];
    Ctl ctl;
};

// A Fisher solve in progress (pdhcg_fisher_begin .. pdhcg_fisher_end).
struct Session {
    bool active = false;
    pdhcg_params prm;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    double omega = 1.0, omega0 = 1.0;
    int restarts = 0;
    long long iters_at_restart = 0;
    double kkt_rs = 0.0, kkt_prev = 0.0;
    bool converged = false, use_avg = false;
    pdhcg_status status = PDHCG_ERR_NOT_CONVERGED;
    KktOut best = {};
    double t_setup = 0.0, t_loop = 0.0;
    // optional CUDA-event timing of the row kernel and the KKT evaluations
    int n_ev = 0;
    cudaEvent_t ev[2 * 80 + 4];
    double prox_ms = 0.0, kkt_ms = 0.0;
    long long prox_launches = 0;
    long long graph_kernels = 0;     // kernel nodes in the chunk graph
    long long launches = 0;          // kernels launched by session_step
};

struct SavedState {
    bool valid = false;
    int kind = 0;           // 0 Fisher, 1 Arrow-Debreu (E = I), 2 batched
    SolveResult res;
};

}  // namespace pdhcg

struct pdhcg_handle_s {
    cudaStream_t stream = 0;        // where the library's work runs
    cudaStream_t user_stream = 0;   // the stream given to pdhcg_create
    bool owns_stream = false;       // stream 0 given: work runs on an owned stream
    cudaEvent_t entry_ev = nullptr;
    int device = 0;
    unsigned int last_err = 0;
    pdhcg::Prepared prep;
    pdhcg::SavedState state;
    pdhcg::Session sess;
    // staged caller inputs / outputs
    pdhcg::DevBuf in_rp, in_col, in_val, in_w, in_x0, in_p0, o_p, o_u, o_x;
    // market
    pdhcg::DevBuf rp, urp, perm, inv, w, wff, err, deg, degint, rank, cj, uv, rowmax, p0i;
    // iterates
    pdhcg::DevBuf X0, X1, Xb, Xr;
    pdhcg::DevBuf p, pc, pff, pbar, prs, C0, C1, C2, c_cur, c_avg, M, acc, t, t_cur, t_avg;
    pdhcg::DevBuf part, part2, kpart, gpart, ctl, kout, pff_p, pff_pb, ndpart;
    // extra buffers of the AD loop, the batched solver and the adjoint
    pdhcg::DevBuf ad_w, ad_wn, ad_p, ad_e_rp, ad_e_col, ad_e_val;
    pdhcg::DevBuf bt[24];
    int bt_table_mixed[5] = {-1, -1, -1, -1, -1};   // autotuned lanes per row by degree class
    int bt_table_fp64[5] = {-1, -1, -1, -1, -1};
    int batch_B = 0;
    int bt_N = 0, bt_M = 0;           // sizes of the last batched solve (for backward)
    long long bt_NNZ = 0;
    bool bt_mixed = true;
    double tight_kappa = 0.0;   // 0: automatic (from the KKT error of the solve)
    double bt_kkt_max = 0.0;    // largest KKT error of the last batched solve
    pdhcg::DevBuf adj[24];
    pdhcg::DevBuf pd[16];         // restarted PDHG (pdhg.cu)
    pdhcg::HostMirror* host = nullptr;

    void release() {
        pdhcg::DevBuf* all[] = {&in_rp, &in_col, &in_val, &in_w, &in_x0, &in_p0, &o_p, &o_u, &o_x,
                                &rp, &urp, &perm, &inv, &w, &wff, &err, &deg, &degint, &rank, &cj, &uv, &rowmax, &p0i,
                                &X0, &X1, &Xb, &Xr, &p, &pc, &pff, &pbar, &prs, &C0, &C1, &C2, &c_cur,
                                &c_avg, &M, &acc, &t, &t_cur, &t_avg, &part, &part2, &kpart, &gpart, &ctl,
                                &kout, &pff_p, &pff_pb, &ndpart, &ad_w, &ad_wn, &ad_p, &ad_e_rp, &ad_e_col, &ad_e_val};
        for (auto* b : all) b->release();
        for (auto& b : bt) b.release();
        for (auto& b : adj) b.release();
        for (auto& b : pd) b.release();
        if (host) cudaFreeHost(host);
        host = nullptr;
    }
};

pdhcg_status prepare_market(pdhcg_handle h, const pdhcg_market* mk, bool mixed, bool init_x);
// iteration workspace of a prepared market (shared with the PDHG solver)
pdhcg_status alloc_iter(pdhcg_handle h);
// buffers of one KKT evaluation (slot 0: current point, 1: average)
pdhcg::KktBufs kkt_bufs(pdhcg_handle h, double* c_out, double* t_out, int slot);
// Order the library stream after the caller's legacy default stream (a graph
// cannot be captured on stream 0, so such handles work on a stream of their own).
void enter(pdhcg_handle h);
pdhcg_status solve_prepared(pdhcg_handle h, const pdhcg_params& prm, const double* p0_int_dev, bool warm_x,
                            pdhcg::SolveResult* res);
pdhcg_status session_begin(pdhcg_handle h, const pdhcg_params& prm, const double* p0_int_dev);
pdhcg_status session_step(pdhcg_handle h, long long chunks);
void session_result(pdhcg_handle h, pdhcg::SolveResult* res);
void session_end(pdhcg_handle h);
pdhcg_status write_outputs(pdhcg_handle h, const pdhcg::SolveResult& r, double* p_out, double* util_out,
                           void* x_out);
void fill_info(pdhcg_info* info, const pdhcg::SolveResult& r, const pdhcg::Prepared& P, pdhcg_status st);
