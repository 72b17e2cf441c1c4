/*
 * pdhcg.h -- C ABI of libpdhcg.so: restarted PDHCG for linear Fisher markets
 * and the Arrow-Debreu fixed point, on one NVIDIA GB300 (sm_103a).
 *
 * Method: Liu, Huang, Li, Ge, Ye, "PDHCG: A Scalable First-Order Method for
 * Large-Scale Competitive Market Equilibrium Computation".
 *
 *   Eisenberg-Gale program (Eq. 1):   max_x sum_i w_i log(sum_j u_ij x_ij)
 *                                     s.t. sum_i x_ij = 1, x >= 0,
 *   solved through its saddle form (Eq. pdhcg:primal-dual-formulation) by
 *   Alg. 2 (restarted PDHCG) with the Section 5 enhancements (row scaling,
 *   adaptive restarts, adaptive step size and primal weight), stopped on the
 *   relative KKT error of Section 5.
 *
 * Conventions (all entry points):
 *   - A market is n buyers x m goods.  U is CSR: row_ptr[n+1] (int64,
 *     row_ptr[0] = 0), col[nnz] (int32, strictly increasing within a row),
 *     val[nnz] (u_ij > 0, finite).  Budgets w[n] > 0 (double).
 *   - Assumption 1 of the paper (every row and every column has an entry) is
 *     required; violations return PDHCG_ERR_INVALID.
 *   - Pointer location: every array argument may be HOST or DEVICE memory; the
 *     library detects which (cudaPointerGetAttributes) and copies host inputs
 *     to its device workspace and device results to host outputs inside the
 *     call.  Pinned host memory makes those copies faster.
 *   - Ownership: the caller owns every argument and allocates every output.
 *     The library never keeps a caller pointer after a call returns.  The
 *     handle owns its device workspace, which grows to the largest problem
 *     seen and is released by pdhcg_destroy.
 *   - Streams: all device work is ordered on the stream given to
 *     pdhcg_create (0 = legacy default stream).  Every call is synchronous
 *     on return (it reads a convergence status from the device).
 *   - Errors: functions return a pdhcg_status; outputs are unspecified unless
 *     the status is PDHCG_OK or PDHCG_ERR_NOT_CONVERGED (then they hold the
 *     best iterate found).  A handle is used by one host thread at a time.
 */
#ifndef PDHCG_H
#define PDHCG_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define PDHCG_VERSION_MAJOR 0
#define PDHCG_VERSION_MINOR 1

typedef enum {
    PDHCG_OK = 0,
    PDHCG_ERR_INVALID = 1,        /* bad argument or Assumption 1 violated       */
    PDHCG_ERR_CUDA = 2,           /* a CUDA runtime call failed                   */
    PDHCG_ERR_OOM = 3,            /* device allocation failed                     */
    PDHCG_ERR_NOT_CONVERGED = 4,  /* iteration or time limit reached before tol   */
    PDHCG_ERR_NUMERIC = 5,        /* NaN/Inf detected in the iterates             */
    PDHCG_ERR_TIMEOUT = 6,        /* time_limit_s exceeded                         */
    PDHCG_ERR_NO_STATE = 7        /* backward called without a saved equilibrium   */
} pdhcg_status;

typedef enum {
    PDHCG_FP64 = 0,   /* "plain": FP64 storage and arithmetic everywhere          */
    PDHCG_MIXED = 1   /* FP32 storage of u, x, x-bar; per-entry arithmetic in FP32
                         with float-float (about 48-bit) evaluation of the
                         cancellation-prone row terms; column sums in exact
                         64-bit fixed point; every reduction, norm, KKT residual
                         and restart test in FP64                               */
} pdhcg_precision;

/* Value type of a market's val array. */
typedef enum { PDHCG_VAL_F64 = 0, PDHCG_VAL_F32 = 1 } pdhcg_valtype;

typedef struct {
    int32_t n;                 /* buyers                                  */
    int32_t m;                 /* goods                                   */
    int64_t nnz;               /* stored utilities = row_ptr[n]           */
    const int64_t* row_ptr;    /* [n+1]                                   */
    const int32_t* col;        /* [nnz]                                   */
    const void* val;           /* [nnz] double or float (val_type)        */
    pdhcg_valtype val_type;
    const double* w;           /* [n] budgets                             */
} pdhcg_market;

typedef struct {
    double tol;                /* stop when relative KKT error <= tol (Section 5)   */
    int64_t max_iter;          /* cap on accepted PDHCG iterations                   */
    double time_limit_s;       /* wall-clock cap, checked every kkt_check_every     */
    pdhcg_precision prec;
    int32_t kkt_check_every;   /* iterations between KKT / restart checks (64)      */
    double beta_suff;          /* 0.2  adaptive restart, Section 5                  */
    double beta_nec;           /* 0.8                                               */
    double beta_art;           /* 0.2                                               */
    double theta;              /* 0.2  primal-weight smoothing, Section 5           */
    double eta_lo;             /* 0.01 lower bound of eta / eta_0, Section 5        */
    double eta_hi;             /* 3.0  upper bound of eta / eta_0, Section 5        */
    double eta0_scale;         /* 0.9  eta_0 = eta0_scale / ||K||_2                  */
    int32_t omega_reset_every; /* 3    restarts between primal-weight range checks  */
    double omega_range;        /* 100  allowed range omega_0 / r .. omega_0 * r     */
    int32_t row_solve_max_iter;/* cap on active-set rounds of one row solve (64)    */
    double tight_kappa;        /* relative slack defining tight edges (backward);
                                  0: 100 x the KKT error reached, in [1e-9, 1e-3]   */
    int32_t verbose;           /* 0 silent, 1 one line per check to stderr          */
    int32_t timing;            /* 1: time every row-kernel launch with CUDA events
                                  (fills pdhcg_info.prox_ms / prox_launches)        */
    int32_t batch_lanes;       /* batched solves: lanes per row.  0 (default): the
                                  autotuner's choice per degree class; 4, 8, 16, 32:
                                  that many lanes per row, rows held in registers
                                  (a market whose longest row does not fit takes the
                                  narrowest width that fits, or the chunked path);
                                  64: the chunked long-row path (32 lanes streaming
                                  the row) for every market.  Other values:
                                  PDHCG_ERR_INVALID                                  */
    int32_t section_count;     /* FP64 single-market solves: 0 (default) = the exact
                                  active-set root of each row subproblem; K >= 2 = the
                                  K-section search of Section 2.2 (K candidates per
                                  round, each with its image bracketing the root),
                                  at most row_solve_max_iter rounds                  */
    double section_tol;        /* relative bracket width at which the K-section
                                  search stops (0 = 1e-8, the paper's)               */
} pdhcg_params;

typedef struct {
    int64_t iters;             /* accepted PDHCG iterations                         */
    int64_t passes;            /* row passes (accepted + rejected step attempts)    */
    int32_t restarts;
    double kkt, r_primal, r_dual, r_gap;   /* of the returned point              */
    double solve_ms;           /* device+host time of the iteration loop         */
    double setup_ms;           /* validation, preprocessing, uploads              */
    double bytes_moved;        /* algorithmic HBM bytes of the row passes         */
    int32_t row_solve_capped;  /* rows whose solve hit row_solve_max_iter          */
    pdhcg_status status;
    double prox_ms;            /* device time of the row-kernel launches (timing=1) */
    int64_t prox_launches;     /* row-kernel launches that did a pass (timing=1)    */
    double kkt_ms;             /* device time of the KKT evaluations (timing=1)     */
    int64_t kernel_launches;   /* library kernels launched by the iteration loop    */
    int64_t row_solve_evals;   /* MIXED: evaluations of the row equation, summed over
                                  rows and passes (0 for FP64 and batched solves)   */
} pdhcg_info;

typedef struct pdhcg_handle_s* pdhcg_handle;

/* ---------------------------------------------------------------------------
 * Library plumbing
 * ------------------------------------------------------------------------- */
const char* pdhcg_status_string(pdhcg_status s);
/* Text of the last CUDA error met by a library call on this host thread
 * ("no error" if none); meant for diagnostics after PDHCG_ERR_CUDA. */
const char* pdhcg_last_error(void);
int32_t pdhcg_version(void);      /* major * 100 + minor */

/* Defaults: tol 1e-6, max_iter 1e6, time limit 1e9 s, MIXED, check every 64,
 * betas 0.2/0.8/0.2 and theta 0.2 (Section 5), eta in [0.01, 3] eta_0
 * (Section 5), eta0_scale 0.9, omega reset every 3 restarts (Section 5),
 * omega_range 100, 64 row-solve rounds, tight_kappa 0 (automatic). */
void pdhcg_default_params(pdhcg_params* prm);

/* Create a handle bound to a CUDA stream (cudaStream_t passed as void*) on the
 * current device.  Allocates no workspace yet. */
pdhcg_status pdhcg_create(pdhcg_handle* h, void* stream);
pdhcg_status pdhcg_destroy(pdhcg_handle h);

/* ---------------------------------------------------------------------------
 * Fisher equilibrium (Alg. 2, Section 2.2; enhancements and stopping rule of
 * Section 5).
 *
 * p_out[m]      equilibrium prices (unique, Fact 1)
 * util_out[n]   buyer utilities t_i = sum_j u_ij x_ij in the caller's units
 *               (unique, Fact 1); may be NULL
 * x_out[nnz]    allocation on supp U in CSR order, of the precision's value
 *               type (double for FP64, float for MIXED); may be NULL
 * p0, x0        optional warm start (NULL = x_ij = 1/deg_j, p_j = sum w / m)
 * info          may be NULL
 * ------------------------------------------------------------------------- */
pdhcg_status pdhcg_fisher_solve(pdhcg_handle h, const pdhcg_market* mk, const pdhcg_params* prm,
                                const double* p0, const void* x0,
                                double* p_out, double* util_out, void* x_out, pdhcg_info* info);

/* The same solve in three calls, for callers that interleave their own work
 * or time a fixed number of check periods:
 *   pdhcg_fisher_begin  validation, preprocessing, initial point (as above)
 *   pdhcg_fisher_step   run `chunks` check periods, each kkt_check_every
 *                       accepted iterations followed by the KKT evaluation and
 *                       the restart / termination decision; returns PDHCG_OK
 *                       once the tolerance is met (further steps do nothing),
 *                       PDHCG_ERR_NOT_CONVERGED while it is not, or an error
 *                       (TIMEOUT, NUMERIC, CUDA).  info (may be NULL) receives
 *                       the running totals.
 *   pdhcg_fisher_end    write the outputs of the best current candidate
 *                       (same arguments as pdhcg_fisher_solve) and release the
 *                       iteration graph.
 * pdhcg_fisher_solve == begin, step until done, end. */
pdhcg_status pdhcg_fisher_begin(pdhcg_handle h, const pdhcg_market* mk, const pdhcg_params* prm,
                                const double* p0, const void* x0);
pdhcg_status pdhcg_fisher_step(pdhcg_handle h, int32_t chunks, pdhcg_info* info);
pdhcg_status pdhcg_fisher_end(pdhcg_handle h, double* p_out, double* util_out, void* x_out, pdhcg_info* info);

/* ---------------------------------------------------------------------------
 * Arrow-Debreu exchange market by the fixed-point iteration of Alg. 4
 * (Section 4):  w^{k+1} = E p(w^k), each p(w) a Fisher solve warm-started
 * from the previous one.  E is n x m CSR (e_row_ptr, e_col, e_val); all three
 * NULL means E = I (requires n == m: agent i owns one unit of good i).
 * mk->w holds the initial budgets w^0.  Stops when
 *   max_i |w^{k+1}_i - w^k_i| / max_i |w^k_i| < outer_tol
 * or after max_outer rounds.  p_out[m], w_out[n] (the final budgets).
 * info (may be NULL) accumulates the inner iterations; info->iters is the sum,
 * *outer_out (may be NULL) receives the number of outer rounds.
 * ------------------------------------------------------------------------- */
pdhcg_status pdhcg_ad_solve(pdhcg_handle h, const pdhcg_market* mk,
                            const int64_t* e_row_ptr, const int32_t* e_col, const double* e_val,
                            double outer_tol, int32_t max_outer, const pdhcg_params* prm,
                            double* p_out, double* w_out, int32_t* outer_out, pdhcg_info* info);

/* ---------------------------------------------------------------------------
 * B independent Fisher markets solved together (each to prm->tol).  Market b
 * owns rows [row_off[b], row_off[b+1]), goods [good_off[b], good_off[b+1]) and
 * entries [nnz_off[b], nnz_off[b+1]); row_ptr is the global CSR over all rows
 * (row_ptr[row_off[b]] == nnz_off[b]); col holds LOCAL good ids (0..m_b-1).
 * p_out[sum m_b], util_out[sum n_b] (may be NULL), info_out[B] (may be NULL).
 * Returns PDHCG_OK only if every market converged.
 * ------------------------------------------------------------------------- */
pdhcg_status pdhcg_fisher_solve_batched(pdhcg_handle h, int32_t B,
                                        const int64_t* row_off, const int64_t* good_off,
                                        const int64_t* nnz_off, const int64_t* row_ptr,
                                        const int32_t* col, const void* val, pdhcg_valtype val_type,
                                        const double* w, const pdhcg_params* prm,
                                        double* p_out, double* util_out, pdhcg_info* info_out);

/* ---------------------------------------------------------------------------
 * Reverse-mode derivative of the equilibrium of the LAST successful
 * pdhcg_fisher_solve / pdhcg_fisher_solve_batched / pdhcg_ad_solve on this
 * handle.  For f = sum_j grad_p[j] p_j + sum_i grad_util[i] t_i it returns
 * grad_u[nnz] = df/du_ij (CSR order of that market) and grad_w[n] = df/dw_i.
 * The derivative follows from the KKT system of Section 3.2 (Eq.
 * KKT-system-6..9) at a non-degenerate equilibrium: on the tight graph G
 * (edges with p_j <= u_ij y_i (1 + tight_kappa) and x_ij > 0) prices and
 * y = w/t are log-potentials fixed by log u_ij up to one scale per connected
 * component, the scale being set by sum_C p = sum_C w (Fact 1).  The adjoint
 * edge flows solve a graph-Laplacian system by conjugate gradients.  For an
 * Arrow-Debreu solve the fixed point w = E p(w) is differentiated as well
 * (adjoint fixed-point iteration).  grad_util may be NULL (zero).
 * ------------------------------------------------------------------------- */
pdhcg_status pdhcg_fisher_backward(pdhcg_handle h, const double* grad_p, const double* grad_util,
                                   double* grad_u, double* grad_w);

/* ---------------------------------------------------------------------------
 * Restarted PDHG (Alg. 1, Section 2.1), the paper's comparator for PDHCG, in
 * FP64 whatever prm->prec says.  The saddle form keeps the buyer utilities t
 * as primal variables with dual variables y for t_i = u_i^T x_i; each step is
 * the closed-form update of Eq. update:py (p and y), Eq. update:t (t) and Eq.
 * update:x (x = [x - tau (p - u y)]_+).  Every restart_every steps the iterates
 * restart from their uniform averages (Alg. 1).  Constant step sizes tau =
 * eta / omega, sigma = eta omega with eta = prm->eta0_scale / ||K||_2 (||K||_2
 * by power iteration on the GPU) and omega = ||p^0|| / ||(x^0, t^0)||.  Stops
 * when the relative KKT error of Section 5 of the current point or of the
 * average is <= prm->tol (checked every prm->kkt_check_every steps), or on
 * prm->max_iter / prm->time_limit_s.  Outputs as pdhcg_fisher_solve (x_out is
 * double); the equilibrium it returns is saved for pdhcg_fisher_backward.
 * ------------------------------------------------------------------------- */
pdhcg_status pdhcg_fisher_solve_pdhg(pdhcg_handle h, const pdhcg_market* mk, const pdhcg_params* prm,
                                     int32_t restart_every, double* p_out, double* util_out, void* x_out,
                                     pdhcg_info* info);

/* ---------------------------------------------------------------------------
 * Building blocks of one iteration, exposed so that each step can be checked
 * on its own at any size.  They run the same kernels as the solver.
 *
 * pdhcg_row_prox: the primal update of Alg. 2 (Section 2.2, Eq. bisection with
 * the utility factor u_ij restored, as in Eq. KKT-system-6): for every buyer i
 * solve s = sum_j u_ij [x_ij - tau p_j + tau w_i u_ij / s]_+ and return
 * x_new[nnz] (value type of prec) and s_out[n] (may be NULL), on the
 * ROW-SCALED market (each row divided by its maximum, Section 5), together
 * with the exact column sums c_out[m] = sum_i x_new_ij (may be NULL).
 * x_in uses the value type of prec; p[m] is double.
 * ------------------------------------------------------------------------- */
pdhcg_status pdhcg_row_prox(pdhcg_handle h, const pdhcg_market* mk, pdhcg_precision prec,
                            const void* x_in, const double* p, double tau,
                            void* x_new, double* s_out, double* c_out);

/* pdhcg_kkt: relative primal residual, dual residual and primal-dual gap of
 * Section 5 ("Criteria") for the point (x, p) of the row-scaled market, with
 * t_i = u_i^T x_i and y = w/t; out[0..3] = r_primal, r_dual, r_gap, max of
 * the three.  x uses the value type of prec. */
pdhcg_status pdhcg_kkt(pdhcg_handle h, const pdhcg_market* mk, pdhcg_precision prec,
                       const void* x, const double* p, double* out);

/* pdhcg_kkt_noalloc: the same three residuals as pdhcg_kkt, for callers that
 * cannot allocate device memory at the moment they need them: code running
 * inside an allocator or memory-pool callback (allocating there re-enters the
 * allocator), a process whose device memory another framework has reserved in
 * full, or a real-time loop that forbids allocation after start-up.  The paper
 * has no counterpart to this entry point.
 *   mk: DEVICE pointers only, the caller's CSR and row order; val may be
 *       FP64 or FP32 (val_type), scaled per row by its maximum as pdhcg_kkt
 *       does; every row must hold at least one entry.
 *   x[nnz] (double), p[m] (double): DEVICE pointers, caller order.
 *   out[4]: host or device; r_primal, r_dual, r_gap, max of the three.
 *   stream: cudaStream_t as void* (0 = legacy default stream).
 * The call is synchronous (it ends with a copy to the host and a stream
 * synchronisation), so it must not be issued on a stream that is being
 * captured into a CUDA graph; it returns PDHCG_ERR_INVALID on such a stream.
 * No call allocates: all scratch lives in one file-scope device array sized
 * for at most 262144 goods (about 4 MiB, held by every device that loads the
 * library until the process exits).  PDHCG_ERR_INVALID is returned for larger
 * m, host input pointers, an empty row, and out-of-range row pointers or
 * column indices (checked in the kernel, which skips the bad entry).  The
 * first call made with a given device current looks the array's device
 * address up (cudaGetSymbolAddress).  The array is shared by every call: each
 * call clears what must start at zero, and calls that overlap on the GPU
 * (other streams or host threads) race, so callers must serialise them. */
pdhcg_status pdhcg_kkt_noalloc(const pdhcg_market* mk, const double* x, const double* p, double* out,
                               void* stream);

#ifdef __cplusplus
}
#endif
#endif /* PDHCG_H */
