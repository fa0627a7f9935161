/*
 * condipm — condensed-space interior-point KKT solves on one GB300 (sm_103a).
 *
 * C ABI of libcondipm.so.  Every compute step runs in this library's own CUDA kernels.
 *
 * Conventions (all entry points):
 *  - Pointers are DEVICE pointers owned by the caller unless the argument says "host".
 *    The library never frees or keeps caller pointers beyond the call.
 *  - Index arrays are int32, CSR row pointers are int32 (nnz < 2^31), values FP64.
 *  - Work is ordered on the given cudaStream_t (0 = legacy default stream; blocking and
 *    non-blocking streams both work).  Calls do not synchronize the stream unless stated
 *    ("synchronizes").  The set-up calls (ipm_opf_create*, ipm_symbolic*, ipm_state_create*,
 *    ipm_batch_create) wait for the given stream's earlier work, run their own device work on
 *    the legacy default stream and return with it finished; the handles they create then work
 *    on the stream given at creation (IPM state, batch) or at each call.
 *  - Library-owned state lives in opaque handles; all their device memory is allocated by
 *    the *_create / ipm_symbolic calls and released by *_destroy.  The numeric calls
 *    (ipm_condense, ipm_factor, ipm_solve, ipm_aug_solve, hykkt_cg) allocate nothing.
 *  - Return value: IPM_OK (0), a positive numerical event, or a negative usage/CUDA error.
 *    No call throws or aborts across the ABI.
 *
 * Notation (paper, Section 2): x in R^n; J = [G; H] stacks the m_e equality rows G on
 * the m_i inequality rows H (m = m_e + m_i rows); W is the Hessian of the Lagrangian;
 * Sigma_x the bound-barrier diagonal; D_H = D_s + delta_w the slack diagonal.
 */
#ifndef CONDIPM_H
#define CONDIPM_H

#include <stdint.h>
#include <cuda_runtime.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
  IPM_OK = 0,
  IPM_ERR_NOT_PD = 1,       /* Cholesky met a pivot <= 0 or non-finite (inertia wrong) */
  IPM_ERR_CG_MAXIT = 2,     /* HyKKT CG hit its iteration limit */
  IPM_ERR_NONFINITE = 3,    /* NaN/Inf in inputs or results */
  IPM_ERR_TIMEOUT = 4,      /* a bounded device wait gave up */
  IPM_ERR_RESTORATION = 5,  /* line search failed (batched solves; the single-problem IPM
                               then runs its restoration phase, and returns this code when that
                               phase fails) */
  IPM_ERR_INERTIA = 6,      /* inertia correction failed: delta_w reached 1e40 */
  IPM_ERR_MAXITER = 7,      /* iteration limit reached before convergence (batched solves) */
  IPM_ERR_INFEASIBLE = 8,   /* the restoration phase converged to a stationary point of the
                               constraint violation without reducing it: locally infeasible */
  IPM_ERR_BAD_ARG = -1,
  IPM_ERR_OOM = -2,
  IPM_ERR_CUDA = -3
};

/* Text of the last error recorded by any call (thread-shared, overwritten by later errors). */
const char *ipm_last_error_message(void);

typedef struct ipm_sym_s *ipm_sym_t; /* symbolic analysis of one sparsity pattern */
typedef struct ipm_num_s *ipm_num_t; /* numeric factor storage + workspaces for one pattern */

/* ipm_symbolic — symbolic analysis, once per sparsity pattern (paper Section 5, "cuDSS
 * analysis": ordering, elimination tree and supernodes, reused across iterations).
 *
 * Pattern of the condensed matrix K = W + Sigma_x + delta_w I + J^T D J (Eq. (K_1), (9),
 * (13)): pat(W) united with the diagonal and pat(J^T J).  Computed entirely on the GPU:
 * graph of K, nested-dissection ordering (project-defined deterministic rule), elimination
 * tree, column structures of L, relaxed supernodes (ipm_symbolic_relaxed with (8, 5)),
 * condensation index maps and the level schedule.
 *   n            number of primal variables
 *   m            rows of J (m_e + m_i)
 *   J_rowptr     [m+1] CSR row pointers of J (device)
 *   J_colind     [nnzJ] CSR column indices of J, each row strictly increasing (device)
 *   nnzJ         J_rowptr[m] (host value)
 *   W_rowptr     [n+1] CSR row pointers of the LOWER triangle of W, diagonal included (device)
 *   W_colind     [nnzW] column indices (col <= row, strictly increasing per row) (device)
 *   nnzW         W_rowptr[n] (host value)
 *   out          receives the handle.
 * Synchronizes the stream.  Errors: IPM_ERR_BAD_ARG on sizes/NULLs, IPM_ERR_OOM, IPM_ERR_CUDA.
 */
int ipm_symbolic(int n, int m, const int *J_rowptr, const int *J_colind, int nnzJ,
                 const int *W_rowptr, const int *W_colind, int nnzW, cudaStream_t stream,
                 ipm_sym_t *out);
/* ipm_symbolic with the supernode partition's parameters (the shape of the supernodal panels).
 * A supernode is a run f..l of consecutive columns with parent(k) = k+1 (a chain of the
 * elimination tree), width <= 64, whose panel holds in every column k the rows k..l and
 * struct(L_l) (explicit zeros where struct(L_k) has none).  Scanning the columns in order,
 * column l+1 joins f..l when parent(l) = l+1, the width stays <= 64, and the width is <= relax_w,
 * or the panel has no explicit zero, or (relax_den > 0) its explicit zeros are at most 1/relax_den
 * of its entries.  (1, 0) gives the fundamental supernodes.  The paper leaves the symbolic
 * analysis to the sparse solver (Section 5); relaxed amalgamation and its parameters are this
 * library's choice, and the same rule runs in the oracle.  IPM_ERR_BAD_ARG unless
 * 1 <= relax_w <= 64 and relax_den >= 0. */
int ipm_symbolic_relaxed(int n, int m, const int *J_rowptr, const int *J_colind, int nnzJ,
                         const int *W_rowptr, const int *W_colind, int nnzW, int relax_w,
                         int relax_den, cudaStream_t stream, ipm_sym_t *out);

/* Sizes of a symbolic analysis (host outputs; NULL outputs are skipped).
 *   nnz_k       structural entries of the lower triangle of K (diagonal included)
 *   nsuper      number of supernodes
 *   nnz_offdiag entries of L below the diagonal (sum of column counts - n)
 *   panel_len   FP64 slots of the supernodal panel storage
 *   nlevels     levels of the supernodal elimination tree
 *   flops       textbook factorization flop count sum_j eta_j (eta_j + 3)              */
int ipm_symbolic_info(ipm_sym_t sym, int64_t *nnz_k, int *nsuper, int64_t *nnz_offdiag,
                      int64_t *panel_len, int *nlevels, double *flops);

/* Number of kernels launched so far by the numeric entry points of this process. */
long long ipm_launch_count(void);

/* Copies the symbolic result to HOST buffers (for bit-exact checks):
 *   perm [n]        perm[k] = original variable at elimination position k
 *   parent [n]      elimination tree over positions (-1 = root)
 *   sptr [nsuper+1] first position of each supernode
 *   colptr [n+1]    int64 column pointers of the below-diagonal structure of L
 *   rowind [nnz_offdiag] row positions, increasing within each column
 * NULL pointers are skipped.  Synchronizes. */
int ipm_symbolic_export(ipm_sym_t sym, int *perm, int *parent, int *sptr, int64_t *colptr,
                        int *rowind);

/* Copies the supernodal layout to HOST buffers: srow_ptr [nsuper+1], srow [srow_ptr[nsuper]]
 * (rows of each supernode, own columns first), lptr [nsuper+1] (panel offsets; panel s is
 * column-major with leading dimension srow_ptr[s+1]-srow_ptr[s]).  NULLs skipped.
 * Synchronizes. */
int ipm_symbolic_export_panels(ipm_sym_t sym, int *srow_ptr, int *srow, int64_t *lptr);

void ipm_symbolic_destroy(ipm_sym_t sym);

/* Numeric storage for one pattern.  precision: 64 (FP64 panels and factor) or 32 (the
 * condensation sums are formed in FP64 and stored in FP32, the factorization runs in FP32, the
 * triangular solves read the FP32 factor and compute in FP64; the factored matrix carries a
 * relative diagonal shift of 2^-20).  ipm_aug_solve and hykkt_cg then reach FP64 accuracy by
 * conjugate gradients in FP64 on K preconditioned by the FP32 factor, which converges while
 * cond(K) * 2^-24 stays moderate; otherwise they return IPM_ERR_NOT_PD (the caller then
 * switches to a precision-64 handle).  Allocates the panel values and every workspace. */
int ipm_num_create(ipm_sym_t sym, int precision, ipm_num_t *out);

/* HOST outputs: the handle's precision and the FP64 preconditioned-CG iterations spent by the
 * last ipm_aug_solve / hykkt_cg on an FP32 factor (0 for FP64 handles). */
int ipm_num_info(ipm_num_t num, int *precision, int *last_pcg_iters);
void ipm_num_destroy(ipm_num_t num);

/* Copies the panel values (panel_len doubles: the lower triangle of P K P^T after
 * ipm_condense, L after ipm_factor) to a HOST buffer.  Synchronizes. */
int ipm_num_export(ipm_num_t num, double *Lx_host);

/* ipm_condense — K = W + diag(sigma_x) + delta_w I + J^T diag(d_row) J written straight into
 * the supernodal panels of L (fill entries zeroed) (Eq. (K_1): K = W + delta_w I + H^T D_H H;
 * Eq. (9): K_gamma = K + gamma G^T G; Eq. (13): K_tau = W + delta_w I + H_tau^T D_H H_tau).
 *   W_val [nnzW]    values of the lower triangle of W in the pattern given to ipm_symbolic
 *   sigma_x [n]     bound-barrier diagonal Sigma_x (0 for free variables)
 *   J_val [nnzJ]    values of J in its pattern
 *   d_row [m]       per-row weight: gamma on HyKKT equality rows, D_H on inequality rows
 *   delta_w         primal regularization
 * Deterministic: each panel entry is one fixed-order sum, no atomics.  The value pointers are
 * kept: FP32 handles multiply by K in FP64 during ipm_aug_solve / hykkt_cg, so they must stay
 * valid and unchanged until the solves that follow. */
int ipm_condense(ipm_sym_t sym, ipm_num_t num, const double *W_val, const double *sigma_x,
                 const double *J_val, const double *d_row, double delta_w, cudaStream_t stream);

/* ipm_factor — supernodal Cholesky P K P^T = L L^T in place (Section 3: Cholesky of the
 * SPD condensed matrix; positive definiteness stands in for the inertia test, Eq. (7)).
 * One persistent kernel runs all panel and update tasks in a topological order; tasks wait on
 * dependency counters with a bounded number of polls.
 *   d_info  DEVICE int: set to -1 on success, -2 if a device wait gave up (the factor is then
 *           invalid and ipm_num_status reports IPM_ERR_TIMEOUT), else the smallest elimination
 *           position whose pivot was <= 0 or non-finite.  The call does not read it back.
 * The panels then hold L.  Returns IPM_OK unless a usage/CUDA error occurred. */
int ipm_factor(ipm_sym_t sym, ipm_num_t num, int *d_info, cudaStream_t stream);

/* Device status of the last factorization / solves of this handle: IPM_OK or IPM_ERR_TIMEOUT
 * (a bounded wait gave up; later solves do nothing until the next ipm_factor).  HOST output.
 * Synchronizes the device. */
int ipm_num_status(ipm_num_t num, int *status);

/* Number of ~0.2 us polls a device wait may take before it gives up (default 2^23, about
 * 2 s).  Process-wide.  IPM_ERR_BAD_ARG if polls < 1. */
int ipm_set_spin_limit(long long polls);

/* Test hook: raises the number of updates supernode `supernode` waits for by `extra`, so that
 * the next ipm_factor meets a wait that nothing satisfies (exercises the timeout path
 * without any fault).  Destroy the symbolic handle afterwards. */
int ipm_debug_add_dependency(ipm_sym_t sym, int supernode, int extra);

/* Debugging aid: while on (nonzero), every floating-point device buffer that the KKT and IPM
 * entry points allocate afterwards (symbolic, numeric, OPF, IPM-state and batch handles, their
 * temporaries, the batch's instance pool) starts filled with bytes 0xFF, a NaN in FP64 and FP32,
 * instead of undefined contents (or zeros, for the batch pool), so that any entry a kernel reads
 * before writing it shows up as NaN in the results.  Integer buffers and the MLP's (zeroed)
 * buffers are left as they are.  Process-wide, off by default; costs one memset per
 * allocation.  Always IPM_OK. */
int ipm_debug_poison_allocations(int on);

/* ipm_solve — x = K^{-1} b with the factor: y = P b, L z = y, L^T w = z, x = P^T w.
 *   b [n x nrhs], x [n x nrhs] device, column-major with leading dimension n (x may alias b);
 *   nrhs >= 1 right-hand sides, solved one after another in stream order. */
int ipm_solve(ipm_sym_t sym, ipm_num_t num, const double *b, double *x, int nrhs,
              cudaStream_t stream);

/* ipm_solve_noalloc — the solve of ipm_solve (x = K^{-1} b, same factor, same kernels) for
 * callers that cannot allocate device memory when they call: a runtime that hands out all
 * device memory itself at start-up, a process with a fixed memory budget, a latency-critical
 * loop that must not enter the allocator.  The paper has no counterpart; this is a library
 * convenience.  The call allocates nothing: its scratch (the permuted work vector and the
 * dependency counters) is a static device array of the library, sized for n and the number of
 * supernodes up to 262144 (2^18), which every GPU that loads the library holds until exit.
 *   b [n], x [n] device (may alias); d_status: DEVICE int, receives IPM_OK or IPM_ERR_TIMEOUT
 *   (a bounded wait gave up; x is then invalid) in stream order, and the call returns without
 *   waiting; or NULL: the call then synchronizes the stream and returns that status itself.
 * The first call on each device looks up the array's device address (cudaGetSymbolAddress),
 * so make that first call before any stream capture.  All calls share the array and it keeps
 * the last call's contents (the counters are cleared by each call); calls that overlap on the
 * GPU (other streams, other threads) race on it — serialize them.
 * IPM_ERR_BAD_ARG (with a message) when n or the supernode count exceeds 262144. */
int ipm_solve_noalloc(ipm_sym_t sym, ipm_num_t num, const double *b, double *x, int *d_status,
                      cudaStream_t stream);

/* ipm_aug_solve — LiftedKKT solve (Section 3.2, Eq. (13)) of the augmented system with the
 * slack block eliminated (all rows inequality rows):
 *     [ W + Sigma_x + delta_w I   J^T      ] [dx]   [a]
 *     [ J                        -D_H^{-1} ] [dz] = [b]
 * by K dx = a + J^T D_H b, dz = D_H (J dx - b), followed by Richardson iterative refinement
 * on this system in FP64 (Section 2.2 "Iterative refinement") until the backward error
 * eta = ||res||_inf / (||A||_inf ||sol||_inf + ||rhs||_inf) <= tol, it stops halving, or
 * max_refine steps.  Requires a successful ipm_factor of the matching K.
 *   a [n], b [m], dx [n], dz [m];  d_eta (device double), d_steps (device int) receive the
 *   final backward error and the refinement steps taken.
 * Synchronizes once per refinement step (host decides whether to continue).  With an FP32
 * factor each condensed solve is FP64 conjugate gradients on K preconditioned by the factor;
 * IPM_ERR_NOT_PD is returned when they meet negative curvature or reach neither a relative
 * residual nor a normwise backward error of 1e-14 in 100 iterations (regularize more, as after a failed factorization). */
int ipm_aug_solve(ipm_sym_t sym, ipm_num_t num, const double *W_val, const double *sigma_x,
                  const double *J_val, const double *d_row, double delta_w, const double *a,
                  const double *b, double *dx, double *dz, int max_refine, double tol,
                  double *d_eta, int *d_steps, cudaStream_t stream);

/* hykkt_cg — HyKKT (Section 3.1, Eq. (10)).  With the first m_e rows of J being G and the
 * rest H, solves the augmented system
 *     [ W + Sigma_x + delta_w I   G^T   H^T      ] [dx]   [a  ]
 *     [ G                         0     0        ] [dy] = [b_G]
 *     [ H                         0    -D_H^{-1} ] [dz]   [b_H]
 * using the factor of K_gamma = W + Sigma_x + delta_w I + H^T D_H H + gamma G^T G
 * (ipm_condense with d_row = [gamma..., D_H...]): r1 = a + H^T D_H b_H, r2 = b_G,
 * CG from dy = 0 on (G K_gamma^{-1} G^T) dy = G K_gamma^{-1}(r1 + gamma G^T r2) - r2 until
 * ||r_k||_2 <= max(rtol ||r_0||_2, 1e-14) or maxit; then
 * dx = K_gamma^{-1}(r1 + gamma G^T r2 - G^T dy) and dz = D_H (H dx - b_H).  When the normwise
 * backward error of (dx, dy, dz) on the augmented system above exceeds 1e-10, the solution is
 * refined on that system (Sec. 2.2): the residual is solved by the same procedure and added, at
 * most three times, until the error is below 1e-10 or stops halving.  The refinement reads
 * W_val, sigma_x and delta_w as passed to the last ipm_condense on num: those device arrays must
 * still hold the values they held then.
 *   d_row [m] as passed to ipm_condense (d_row[0..m_e) = gamma).
 *   a [n], b [m], dx [n], dy [m_e], dz [m - m_e]
 *   h_iters, h_relres: HOST outputs (CG iterations of all solves, final ||r||/||r_0|| of the
 *   first CG).
 * Returns IPM_ERR_CG_MAXIT if maxit was reached; with an FP32 factor, IPM_ERR_NOT_PD as for
 * ipm_aug_solve.  Synchronizes (convergence tests). */
int hykkt_cg(ipm_sym_t sym, ipm_num_t num, int m_e, const double *J_val, const double *d_row,
             double gamma, const double *a, const double *b, double rtol, int maxit, double *dx,
             double *dy, double *dz, int *h_iters, double *h_relres, cudaStream_t stream);

/* ---------------------------------------------------------------------------------------
 * AC optimal power flow model (the NLP (1) the benchmarks solve; its derivative evaluation is
 * the "AD" part of an IPM iteration, Section 5).  Variables x = [V | theta | Pg | Qg],
 * equalities g = [P balance | Q balance | theta_ref], inequalities
 * h = [|S_from|^2 - rate^2 | |S_to|^2 - rate^2] (h <= 0), cost sum c2 (100 Pg)^2 + c1 (100 Pg).
 */
typedef struct ipm_opf_s *ipm_opf_t;

/* All array arguments are HOST arrays (copied).  Branch k joins f_bus[k] -> t_bus[k] (pi model,
 * series r + j x, total charging b, limit rate); generator g sits at gen_bus[g] (gen_bus[0] is
 * the reference bus); xl/xu are the n = 2nb+2ng variable bounds (+-inf where absent).
 * Builds the sparsity patterns of J and of the lower triangle of W on the GPU.
 * Synchronizes.  IPM_ERR_BAD_ARG on out-of-range bus indices. */
int ipm_opf_create(int nb, int nbr, int ng, const int *f_bus, const int *t_bus, const double *r,
                   const double *x, const double *b, const double *rate, const double *pd,
                   const double *qd, const int *gen_bus, const double *c2, const double *c1,
                   const double *xl, const double *xu, cudaStream_t stream, ipm_opf_t *out);
/* The same grid in the flow-variable formulation (the shape of the paper's instances): branch
 * flows p_end, q_end (2 nbr each, from ends then to ends) are free variables after [V | theta |
 * Pg | Qg]; equalities [P balance | Q balance | theta_ref | p_end - P_end(V, theta) |
 * q_end - Q_end(V, theta)], inequalities p_end^2 + q_end^2 - rate^2 <= 0.  n = 2 nb + 2 ng +
 * 4 nbr, m_e = 2 nb + 1 + 4 nbr, m_i = 2 nbr.  Arguments as for ipm_opf_create (xl, xu: the
 * 2 nb + 2 ng compact bounds).  The IPM starts every flow variable at the flow of its start
 * voltages. */
int ipm_opf_create_flow(int nb, int nbr, int ng, const int *f_bus, const int *t_bus,
                        const double *r, const double *x, const double *b, const double *rate,
                        const double *pd, const double *qd, const int *gen_bus, const double *c2,
                        const double *c1, const double *xl, const double *xu,
                        cudaStream_t stream, ipm_opf_t *out);
int ipm_opf_info(ipm_opf_t opf, int *n, int *m_e, int *m_i, int *nnzJ, int *nnzW);
/* Copies the handle's patterns into caller buffers (host or device; NULLs skipped): CSR of J
 * (J_rowptr [m_e+m_i+1], J_colind [nnzJ]) and CSR of the lower triangle of W (W_rowptr [n+1],
 * W_colind [nnzW]); columns increase within each row.  Synchronizes. */
int ipm_opf_patterns(ipm_opf_t opf, int *J_rowptr, int *J_colind, int *W_rowptr, int *W_colind);
/* Evaluates at x (device): f (device scalar, may be NULL), grad [n] (may be NULL),
 * g [m_e], h [m_i], J_val [nnzJ] (may be NULL) and, when W_val is not NULL, W_val [nnzW] =
 * sigma_f grad^2 f + sum y_i grad^2 g_i + sum z_j grad^2 h_j (y [m_e], z [m_i]). */
int ipm_opf_eval(ipm_opf_t opf, const double *x, const double *y, const double *z,
                 double sigma_f, double *f, double *grad, double *g, double *h, double *J_val,
                 double *W_val, cudaStream_t stream);
/* Replaces the loads (pd, qd: nb values each, HOST or device; MW / 100 per bus) of a model, for
 * a new scenario of the same grid.  Stream-ordered. */
int ipm_opf_set_loads(ipm_opf_t opf, const double *pd, const double *qd, cudaStream_t stream);
void ipm_opf_destroy(ipm_opf_t opf);

/* ---------------------------------------------------------------------------------------
 * Interior-point iterations on the GPU (Section 2: barrier problem (5), Newton step (K_3) solved
 * in condensed form by LiftedKKT or HyKKT; Ipopt's filter line search, barrier update, inertia
 * correction and multiplier safeguards as cited in Section 2.2).
 */
typedef struct {
  int kkt;          /* 0 = LiftedKKT (Section 3.2), 1 = HyKKT (Section 3.1), 2 = dual-regularized
                       condensed form with delta_c = 1/gamma (Remark in Section 3): one condensed
                       solve of K + G^T G / delta_c refined on the regularized augmented system */
  double tol;       /* scaled KKT tolerance (e.g. 1e-6) */
  double gamma;     /* gamma of forms 1 and 2; <= 0: ||K||_inf / ||G||_inf^2 every iteration
                       (Golub & Greif, recommended in Section 3.1), ||K|| bounded by the row sums
                       of |W + Sigma_x| + |H|^T |D_s| |H| */
  double tau;       /* LiftedKKT relaxation; <= 0 means tau = tol */
  double mu0;       /* initial barrier parameter; <= 0 means 0.1 */
  double cg_rtol;   /* HyKKT CG relative residual; <= 0 means 1e-10 */
  int max_refine;   /* LiftedKKT refinement steps; < 0 means 10 */
  int cg_maxit;     /* HyKKT CG iteration limit; <= 0 means m_e */
  int precision;    /* factorization precision: 64 or 32; 0 means 64.  With 32 the state
                       switches to an FP64 factor for good at the first iteration whose
                       FP32-preconditioned FP64 refinement does not converge (late IPM
                       iterations are too ill-conditioned for an FP32 factor) */
  int sn_relax_w;   /* supernode partition (ipm_symbolic_relaxed); <= 0 means (8, 5) */
  int sn_relax_den;
  int no_resto;     /* nonzero: no feasibility restoration phase (a failed line search ends the
                       solve with IPM_ERR_RESTORATION) */
} ipm_options;

typedef struct {
  int k;            /* iteration index */
  int status;       /* 0 running, 1 converged, else an IPM_ERR_* code among IPM_ERR_INERTIA,
                       IPM_ERR_RESTORATION, IPM_ERR_INFEASIBLE, IPM_ERR_TIMEOUT and
                       IPM_ERR_NONFINITE */
  double mu, kkt_err, alpha, delta_w, obj, eta, theta;
  int n_factor, cg_iters, refine_steps, ls_steps;
  int precision;    /* factorization precision used by this iteration (32 or 64) */
  double gamma;     /* gamma used by this iteration (forms 1 and 2) */
  int pcg_iters;    /* FP64 CG iterations over the FP32 factor in this step's solves (0 in FP64;
                       also the CG after a stagnating refinement) */
  int resto;        /* 1: this call made an iteration of the restoration phase (mu, kkt_err,
                       theta, alpha and delta_w then belong to the restoration problem); 2: the
                       line search failed and the call started the phase; 0 otherwise */
} ipm_iter_info;

typedef struct ipm_state_s *ipm_state_t;

/* Creates the iterate for an OPF problem: flat start pushed inside the bounds, Ipopt gradient
 * scaling of the objective and of each constraint row at the start, s = max(-h, 0.01), y = 0,
 * z = v = 1, bound multipliers 1; runs ipm_symbolic on the model pattern and allocates every
 * workspace.  The opf handle must outlive the state.  Synchronizes. */
int ipm_state_create(ipm_opf_t opf, const ipm_options *opt, cudaStream_t stream,
                     ipm_state_t *out);
/* As ipm_state_create from the caller's point x0 (HOST, n values) instead of the flat start:
 * x0 is pushed inside the bounds, and the scaling, slacks and multipliers are set there as in
 * ipm_state_create.  IPM_ERR_BAD_ARG when x0 is NULL.  Synchronizes. */
int ipm_state_create_at(ipm_opf_t opf, const ipm_options *opt, const double *x0,
                        cudaStream_t stream, ipm_state_t *out);
/* One IPM iteration (or the convergence test that ends the solve): evaluate, test E_0 <= tol,
 * update mu, inertia-corrected condensed KKT solve, fraction to the boundary, filter line search,
 * update.  When the line search finds no acceptable step the call enters the feasibility
 * restoration phase of the filter method (Waechter & Biegler 2006, Sec. 3.3, cited in
 * Section 2.2), and the following calls make its iterations (host_info->resto = 1): an IPM on
 *   min rho sum(p + q) + zeta/2 ||D_R (x - x_R)||^2   s.t.  c(x) - p + q = 0, p, q >= 0,
 * c the IPM rows at the failing point x_R, rho = 1000, zeta = sqrt(mu_R), D_R = min(1, 1/|x_R|),
 * mu_R = max(mu, ||c||_inf), p and q eliminated row by row from its Newton system, which is then
 * solved by the refined condensed solve on the pattern of the main condensed matrix.  The phase
 * ends at the first point whose violation is at most 0.9 times that of x_R and that the filter
 * (with x_R's entry) accepts; the IPM goes on there with y = z = 0.  Status
 * IPM_ERR_INFEASIBLE: the phase converged to a stationary point of its problem first (a local
 * minimizer of the violation); IPM_ERR_RESTORATION: its own line search failed or it ran 500
 * iterations.  host_info (HOST) receives the iteration record; after convergence or a failure
 * further calls return the final status without work.  Synchronizes.  Returns a negative code
 * only on usage/CUDA errors (numerical failures are reported in host_info->status). */
int ipm_step(ipm_state_t state, ipm_iter_info *host_info);
/* Copies x [n] to a HOST buffer (NULL skipped) and the unscaled objective f(x) to *obj (HOST). */
int ipm_state_export(ipm_state_t state, double *x, double *obj);
/* Checkpoint of the iteration between two ipm_step calls (the paper has no counterpart; it reuses
 * one symbolic analysis across solves of a pattern): the primal-dual iterate (x, s, y, z, v, zl,
 * zu), the row scaling, mu, tau, the filter, delta_last, the iteration count and status, in one
 * HOST buffer of doubles.  *len (HOST) receives the length needed; buf = NULL only asks for it.
 * IPM_ERR_BAD_ARG when cap is smaller, or while the state is in the restoration phase.
 * Synchronizes. */
int ipm_state_save(ipm_state_t state, double *buf, int64_t cap, int64_t *len);
/* Puts a saved checkpoint into a state created for the same model and options (sizes, format
 * and length checked: IPM_ERR_BAD_ARG otherwise); the next ipm_step continues the saved
 * iteration.  A checkpoint taken after the FP32 factor stopped serving continues in FP64.
 * Synchronizes. */
int ipm_state_load(ipm_state_t state, const double *buf, int64_t len);
/* Copies the KKT system that the last completed ipm_step solved, and its solution, to HOST
 * buffers (any pointer may be NULL).  The system is the augmented system (K_2) with the slack
 * block eliminated (Sec. 2.2, the system that iterative refinement runs on; Sec. 3.1-3.2):
 *   [ W + Sigma_x + delta_w I   J^T ] [dx ]   [a]
 *   [ J                         -E  ] [dyz] = [b],   E = diag(1 / d_row) on condensed rows,
 * E = 0 on the first *m_e rows (HyKKT keeps the equalities; *m_e = 0 for the other forms).
 * W_val [nnzW]: lower-triangular Hessian values in the model's W pattern (scaled multipliers and
 * objective); sigma [n]; J_val [nnzJ]: the scaled Jacobian in the model's J pattern (rows
 * [G; H], m = m_e0 + m_i0); d_row [m]: the row weights the condensed matrix was built with
 * (LiftedKKT: the two relaxed rows of an equality merged, D1 + D2; HyKKT: gamma on G rows; a
 * step of the restoration phase: 1/E_r on every row, *m_e = 0 for every form);
 * *delta_w; a [n], b [m]: right-hand sides; dx [n], dyz [m]: the refined solution (HyKKT: dy
 * over the G rows, then dz).  Returns IPM_ERR_BAD_ARG before the first step.  Synchronizes. */
int ipm_state_export_kkt(ipm_state_t state, double *W_val, double *sigma, double *J_val,
                         double *d_row, double *delta_w, double *a, double *b, double *dx,
                         double *dyz, int *m_e);
void ipm_state_destroy(ipm_state_t state);

/* ---------------------------------------------------------------- batched interior-point solves
 * Many OPF instances advanced together (LiftedKKT, HyKKT or the dual-regularized form; FP64): the
 * batched form of the method.
 * Instances whose model patterns (J and lower W) are equal share one symbolic analysis (the
 * paper reuses the analysis of a pattern across iterations, Section 5); instances may have
 * different sizes.  Each launch of the condensation, the factorization (level by level through
 * each instance's elimination tree: one block, or one thread-block cluster for the big
 * instances, per instance) and the triangular solves covers every instance that is in that step;
 * the per-instance control of the algorithm of ipm_step (convergence test, barrier update,
 * inertia correction, refinement or CG, fraction to the boundary, filter line search) runs on the
 * device, so a sweep of the method is one CUDA graph and every instance follows the
 * single-problem iteration up to the order of floating-point additions (the restoration phase
 * included; its steps are the refined condensed solves of ipm_step's phase for every form). */
typedef struct ipm_batch_s *ipm_batch_t;

/* Creates the batch over count model handles (HOST array of handles that must outlive the batch;
 * the same handle may not appear twice).  opt: kkt 0 (LiftedKKT), 1 (HyKKT: CG on the Schur
 * complement of K_gamma, cg_rtol and cg_maxit as in ipm_options, gamma > 0) or 2 (dual-regularized
 * form, gamma > 0); precision 0 or 64 (FP64 factor), or 32 with kkt 0 or 2: every instance
 * starts with an FP32 condensed matrix (summed in FP64, rounded once), an FP32 factorization and
 * FP32 triangular solves inside FP64 Richardson refinement on the augmented system (the
 * precision form; the rounding errors of the condensed system are those Section 4 analyses), and
 * goes to an FP64 factor at the same delta_w for the rest of its solve when an FP32
 * factorization breaks down or the refinement stalls above a backward error of 1e-10 (so each
 * accepted solve still meets 1e-10; the inertia of an FP32-factored step is decided in FP32);
 * the remaining fields as in ipm_options.  Runs one
 * ipm_symbolic per distinct pattern, allocates one
 * device pool for every instance's iterate, factor and workspace, and sets every instance to the
 * starting point of ipm_state_create.  Synchronizes.  IPM_ERR_BAD_ARG on a bad argument,
 * IPM_ERR_OOM when the pool does not fit. */
int ipm_batch_create(int count, const ipm_opf_t *opfs, const ipm_options *opt,
                     cudaStream_t stream, ipm_batch_t *out);
/* Number of distinct patterns, bytes of the instance pool, kernel launches per sweep (after the
 * first ipm_batch_run).  Pointers may be NULL. */
int ipm_batch_info(ipm_batch_t batch, int *npatterns, int64_t *device_bytes,
                   int *launches_per_sweep);
/* Puts every instance back at its starting point (as after ipm_batch_create).  Stream-ordered. */
int ipm_batch_reset(ipm_batch_t batch);
/* Runs sweeps until every instance has converged (status 1) or stopped: IPM_ERR_INERTIA,
 * IPM_ERR_RESTORATION, IPM_ERR_INFEASIBLE, IPM_ERR_NONFINITE, IPM_ERR_TIMEOUT, or
 * IPM_ERR_MAXITER after max_iter iterations (or when max_sweeps sweeps end first).  An instance
 * whose line search fails enters the feasibility restoration phase of ipm_step (unless
 * opt->no_resto), on the device like every other step; its iterations are sweeps of the same
 * graph, do not count against max_iter, and end as in ipm_step.  use_graph != 0 replays one captured CUDA
 * graph per sweep, else the sweep's kernels are launched one by one.  Reads one int back per
 * sweep.  Synchronizes. */
int ipm_batch_run(ipm_batch_t batch, int max_iter, int max_sweeps, int use_graph);
/* Per-instance results into HOST arrays [count] (any may be NULL): status, iterations, objective
 * f(x) at the last evaluated iterate, scaled KKT error there, factorizations, backtracking
 * steps.  Synchronizes. */
int ipm_batch_results(ipm_batch_t batch, int *status, int *iters, double *obj, double *kkt_err,
                      int *n_factor, int *ls_steps);
/* Autotuner of the batched launch shapes: for each candidate (cluster size 1, 2, 4 or 8 blocks for
 * the big instances; "big" = supernode count above 1.5x or 1.2x the median; 0.5x, 1x or 2x the
 * default blocks per instance of the element kernels) the sweep graph is captured, every instance
 * is reset and `sweeps` sweeps are timed with CUDA events; the fastest shape is kept and every
 * instance is put back at its starting point.  HOST outputs (any may be NULL when max_results is
 * 0): *n_results = number of candidates; for the first max_results of them cfg[4 k .. 4 k + 3] =
 * (cluster size, threshold numerator, denominator, blocks per instance) and ms_per_sweep[k];
 * *best = index of the chosen one.  Synchronizes.  Returns IPM_ERR_BAD_ARG for sweeps < 1. */
int ipm_batch_autotune(ipm_batch_t batch, int sweeps, int max_results, int *n_results, int *cfg,
                       double *ms_per_sweep, int *best);
/* HyKKT batches: CG iterations per instance since creation or the last reset into a HOST array
 * [count] (0 for the other forms).  Synchronizes. */
int ipm_batch_cg_iters(ipm_batch_t batch, int *cg_iters);
/* Feasibility restoration per instance since creation or the last reset, into HOST arrays
 * [count] (either may be NULL): phases entered and restoration iterations made.  Synchronizes. */
int ipm_batch_resto_counts(ipm_batch_t batch, int *phases, int *iters);
/* KKT solves per instance since creation or the last reset, into HOST arrays [count] (any may
 * be NULL): the factor precision the instance uses now (32 or 64), the IPM iterations whose KKT
 * solve used the FP32 factor, the iteration at which it went to FP64 (-1: it did not); the KKT
 * solves finished, how many of them ended with a normwise backward error of the augmented system
 * (computed on the device, as ipm_aug_solve does) above 1e-10 after the refinement, and the
 * largest such error.  Synchronizes. */
int ipm_batch_solve_info(ipm_batch_t batch, int *current, int *iters32, int *k64, int *solves,
                         int *above, double *eta_max);
/* Copies instance i's x [n] into a HOST buffer.  Synchronizes. */
int ipm_batch_export(ipm_batch_t batch, int i, double *x);
/* Sweeps run since creation or the last reset. */
int ipm_batch_sweeps(ipm_batch_t batch);
/* Tail of a run: in a batch of more than active_max instances, once at most active_max are
 * still running (read back after every sweep), each sweep holds four inertia rounds and eight
 * line-search trials instead of two and two (a round costs little when few instances are left,
 * and an instance that corrects its inertia or backtracks many times then needs fewer sweeps),
 * and with cluster 1, 2, 4 or 8 every remaining instance's factorization and solves run on a
 * thread-block cluster of that many blocks (the chain of the slowest instance, not the GPU's
 * throughput, then sets a sweep); cluster 0 keeps the launch shape.  The iterates are those of
 * the same method (the cluster changes only the order of floating-point sums).  active_max = 0:
 * no tail sweep.  Default (16, 8).  Applies to graph runs (use_graph != 0).  Host only. */
int ipm_batch_set_tail(ipm_batch_t batch, int active_max, int cluster);
/* Sets a launch shape (the candidates of ipm_batch_autotune): instances whose supernode count
 * exceeds big_num / big_den times the median (big_den = 0: none) factor and solve on thread-block
 * clusters of `cluster` blocks (1, 2, 4 or 8), and the element kernels take gx blocks per
 * instance (1..16; gx <= 0 keeps the current value).  *n_big (HOST, may be NULL) = instances on
 * clusters.  Keeps every instance's state. */
int ipm_batch_set_shape(ipm_batch_t batch, int cluster, int big_num, int big_den, int gx,
                        int *n_big);
/* Holds every instance right after the KKT solve (and refinement, or CG) of its iteration k:
 * such instances stop advancing, and ipm_batch_run returns once every instance is held or done.
 * k = -1 (the state after creation) holds none.  The hold lets ipm_batch_export_kkt read a solved
 * system whose values the next phase would overwrite.  Synchronizes. */
int ipm_batch_pause_at(ipm_batch_t batch, int k);
/* Releases the held instances; the next ipm_batch_run continues them from their step
 * (fraction to the boundary, line search).  Synchronizes. */
int ipm_batch_resume(ipm_batch_t batch);
/* Instance i's KKT system and refined solution while it is held (ipm_batch_pause_at), to HOST
 * buffers, in the layout of ipm_state_export_kkt (the augmented system (K_2) with the slack
 * block eliminated, Sec. 2.2; HyKKT: dy over the G rows then dz, and *m_e = the G rows).
 * Returns IPM_ERR_BAD_ARG when the instance is not held.  Synchronizes. */
int ipm_batch_export_kkt(ipm_batch_t batch, int i, double *W_val, double *sigma, double *J_val,
                         double *d_row, double *delta_w, double *a, double *b, double *dx,
                         double *dyz, int *m_e);
/* Copies every instance's x, concatenated in instance order, into a HOST buffer of sum(n)
 * doubles (one gather kernel and one device-to-host copy).  Synchronizes. */
int ipm_batch_export_all(ipm_batch_t batch, double *x_host);
/* on != 0: record CUDA events around every factorization launch (condensation + factorization
 * of the instances in that step) and the first solve launch of every sweep (event nodes inside
 * the captured graph) and accumulate their durations; ipm_batch_kernel_time reports the sums
 * (ms) and the number of sweeps since the last reset. */
int ipm_batch_set_timing(ipm_batch_t batch, int on);
int ipm_batch_kernel_time(ipm_batch_t batch, double *fact_ms, double *solve_ms, int *sweeps);
/* Algorithmic work of one condensation + factorization of each instance, into HOST arrays
 * [count] (any may be NULL): textbook factorization flops sum_j eta_j (eta_j + 3), condensation
 * flops (2 per J^T D J product), and bytes (8 (nnz(J) + m + nnz(W) + n) read, 8 per panel value
 * written). */
int ipm_batch_work(ipm_batch_t batch, double *factor_flops, double *condense_flops,
                   double *bytes);
void ipm_batch_destroy(ipm_batch_t batch);

/* ---------------------------------------------------------------- learned warm start
 * Rows for training and prediction: per instance x (n), log s (m_i), log v (m_i), log zl (n),
 * log zu (n), 0 where a bound is absent (width 3 n + 2 m_i, + m_e below; the iterate of the
 * scaled problem as the batched IPM holds it).  ipm_batch_state_rows writes every instance's row into the DEVICE
 * float matrix out (row stride ld >= width; out NULL only reports *width); all instances must
 * have the same sizes.  HyKKT and dual-regularized batches append the equality multipliers y
 * (m_e values, not logged) to the row.  Stream-ordered. */
int ipm_batch_state_rows(ipm_batch_t batch, float *out, int64_t ld, int *width);
/* Starts every instance from a predicted row (DEVICE float matrix pred, row stride ld, values
 * de-normalized as pred * stdv + mean per column when mean != NULL, else taken as they are):
 * x pushed inside its bounds (the push of the cold start), s = exp(log s), z = v = exp(log v),
 * zl, zu = exp(.) where the bound exists, y from the row's last m_e values (HyKKT and the
 * dual-regularized form), mu0 = s^T v / m_i (at least tol / 10), a fresh filter.
 * Call after ipm_batch_reset (which sets the scaling at the cold start point); an instance whose
 * row holds a non-finite value keeps its cold start.  h_used (HOST, count, may be NULL) receives
 * 1 where the prediction was used.  Synchronizes. */
int ipm_batch_warm_start(ipm_batch_t batch, const float *pred, int64_t ld, const float *mean,
                         const float *stdv, int *h_used);

/* Multilayer perceptron with BF16 weights and activations and FP32 accumulation (tensor-core
 * products), GELU after every layer but the last, mean-squared-error loss, Adam.  Layer l maps
 * dims[l] to dims[l+1] (W_l: dims[l] x dims[l+1] row-major, b_l: dims[l+1]).  All X, Y, T are
 * DEVICE float matrices, row-major, one row per sample, at most max_batch rows per call. */
typedef struct mlp_s *mlp_t;
int mlp_create(int nlayers, const int *dims, int max_batch, mlp_t *out);
/* Number of parameters: sum over layers of dims[l] dims[l+1] + dims[l+1]. */
int mlp_param_count(mlp_t net, int64_t *count);
/* Parameters from / to a HOST float array, per layer W_l (row-major) then b_l; setting them
 * also resets the Adam moments and rounds the BF16 copies.  Synchronizes. */
int mlp_set_params(mlp_t net, const float *host);
int mlp_get_params(mlp_t net, float *host);
/* Gradients of the last mlp_loss_backward, same layout as the parameters.  Synchronizes. */
int mlp_get_grads(mlp_t net, float *host);
/* Y [B x dims[L]] = net(X [B x dims[0]]) (Y may be NULL when only the loss follows). */
int mlp_forward(mlp_t net, const float *X, int B, float *Y, cudaStream_t stream);
/* After mlp_forward on the same rows: *d_loss (DEVICE float) = mean over B x dims[L] of
 * (Y - T)^2, and the gradient of that loss into the parameter gradients. */
int mlp_loss_backward(mlp_t net, const float *T, int B, float *d_loss, cudaStream_t stream);
/* One Adam step (Kingma & Ba, bias-corrected, step number t >= 1) on the FP32 master weights. */
int mlp_adam_step(mlp_t net, float lr, float beta1, float beta2, float eps, int t,
                  cudaStream_t stream);
/* out[r] = src[idx[r]] for r < rows (rows of cols floats; DEVICE pointers). */
int mlp_gather_rows(int rows, int cols, const int *idx, const float *src, float *out,
                    cudaStream_t stream);
/* Per-column mean and standard deviation (population, FP64 sums; std at least floor_std) of a
 * rows x cols DEVICE float matrix, and the column normalization out = (src - mean) / std
 * (out may alias src). */
int mlp_col_stats(int rows, int cols, const float *src, float *mean, float *stdv,
                  float floor_std, cudaStream_t stream);
int mlp_normalize(int rows, int cols, const float *src, const float *mean, const float *stdv,
                  float *out, cudaStream_t stream);
void mlp_destroy(mlp_t net);

#ifdef __cplusplus
}
#endif
#endif /* CONDIPM_H */
