// Batched interior-point solves: many AC-OPF instances, with equal or different sparsity
// patterns, advanced together by the same launches (the batched form of the method; the paper
// reuses one symbolic analysis across iterations of a pattern, Section 5, and motivates batched
// solves of many related problems in Section 1).
//
// * One symbolic analysis per distinct pattern; instances with the same pattern share it.
// * Numeric data of every instance sits in one device pool; the persistent factorization and
//   triangular-solve kernels take tasks from one ticket range per launch that lists every
//   instance's tasks instance after instance (each instance's tasks in its own topological
//   order, so a block only waits on smaller tickets and the schedule cannot deadlock).
// * The interior-point control (convergence test, barrier update, inertia correction, Richardson
//   refinement, fraction to the boundary, filter line search) runs on the device as a per-instance
//   phase machine: every kernel acts on the instances in its phase and a one-thread-per-instance
//   control kernel moves them on.  One sweep (evaluate, build, two inertia rounds, solve, three
//   refinement rounds, step, two line-search trials, accept) is captured once as a CUDA graph and
//   replayed; an instance that needs more rounds than a sweep holds continues in the next sweep
//   from the phase it is in, so every instance follows exactly the single-problem algorithm.
// LiftedKKT (Section 3.2) in FP64.
#include <algorithm>
#include <climits>
#include <cmath>
#include <cstring>
#include <map>
#include <type_traits>
#include <vector>

#include <cooperative_groups.h>

#include "ipm_core.cuh"
#include "numeric_dev.cuh"
#include "opf_dev.cuh"
#include "resto_dev.cuh"

namespace cipm {

// PH_CGI, PH_CG, PH_CGX: HyKKT's Schur-complement CG (start, iterations, primal back-solve);
// PH_PAUSE: held after the KKT solve of the iteration named by ipm_batch_pause_at (the solved
// system and its solution stay in the instance's buffers until ipm_batch_resume);
// PH_PCGI, PH_PCG, PH_PCGX (LiftedKKT batches): conjugate gradients on the condensed system after
// a refinement that stagnated above a backward error of 1e-10 (start, iterations, comparison
// with the refined solution), as in the single-problem solve
enum Phase {
  PH_EVAL = 0, PH_BUILD, PH_FACT, PH_SOLVE, PH_REFINE, PH_STEP, PH_LS, PH_ACC, PH_DONE,
  PH_CGI, PH_CG, PH_CGX, PH_PAUSE, PH_PCGI, PH_PCG, PH_PCGX
};

static constexpr int B_FACT_ROUNDS = 2, B_REFINE_ROUNDS = 3, B_LS_ROUNDS = 2, B_CG_ROUNDS = 6;
// rounds of the tail sweep (few instances left: a round then costs little, and an instance that
// backtracks or corrects its inertia many times needs fewer sweeps)
static constexpr int B_TAIL_FACT_ROUNDS = 4, B_TAIL_LS_ROUNDS = 8;
// conjugate-gradient iterations per sweep and per solve after a stagnating refinement
static constexpr int B_PCG_ROUNDS = 5, B_PCG_MAXIT = 50;
// refinement steps allowed with the FP32 factor (at a contraction rate of 1/2 per step the
// error falls by 2^-30 ~ 1e-9; a slower rate stops at the stall test first)
static constexpr int B_REFINE32 = 30;
static constexpr int B_BLOCK = 256;

// per-instance control record (device)
struct BCtl {
  int ph, status, k, nfac, ls, ftype, have_theta0, ref_it, ref_steps, nfilter;
  int total_fac, total_ls, total_ref;
  double mu, tau, sig, delta_last, theta_max, theta_min;
  double dw, next, grow;
  double alpha, az, amax, amin, gphi, theta, phi, logsum, obj, e0, eta, eta_prev, normA;
  // HyKKT CG: r.r, stopping threshold, step scalars, iterations (this IPM step, in total)
  double cg_rr, cg_stop, cg_alpha, cg_beta;
  int cg_it, cg_total, cg_maxit;
  // precision: p32 = 1 while the FP32 factor serves (cleared for good when an FP32
  // factorization breaks down or its refinement does not reach 1e-10); it32: iterations whose
  // KKT solve used it; k32: the iteration at which the instance went to FP64 (-1: never)
  int p32, it32, k32;
  // KKT solves finished, those left above a backward error of 1e-10, the largest final error
  int n_solve, n_above;
  double eta_worst;
  // directions of this iteration recomputed at a larger delta_w after a failed line search
  int n_reg, pad_reg_;
  // PCG after a stagnating refinement: runs, iterations, this run's count, whether the last
  // refinement correction is taken back, whether the refined solution is restored
  int pg_runs, pg_total, pg_it, pg_undo, pg_restore, pad_pg_;
  double pg_rz, pg_tn, pg_eta0;
  // feasibility restoration (Waechter & Biegler 2006, Sec. 3.3): resto 0 = main problem,
  // 2 = phase entered (its start is set at the next evaluation), 1 = in the phase; ret: the
  // accepted trial passed the return test.  While in the phase mu, tau, delta_last, theta_max,
  // theta_min and nfilter belong to the restoration problem and the main problem's are kept in
  // the *_m fields; k_r counts the phase's iterations.
  int resto, ret, k_r, nfilter_m, n_resto, total_resto;
  double mu_m, tau_m, delta_last_m, theta_max_m, theta_min_m;
  double zeta, theta_start, entry_theta, entry_phi;
};

// per-instance descriptor (device): pattern and model pointers, iterate and work vectors
struct BI {
  Dims D;
  It P;
  StepArgs SA;  // mu and dw are taken from the control record
  OpfData M;
  int nl, nu, m;  // finite lower / upper bounds; model rows m = me0 + mi0
  double *dscale, *gs, *hs, *Jv, *Wv, *lam, *lamw, *f, *fpart;
  double *r1, *dcond, *baug, *a, *dx, *dzc;
  double *xt, *st, *geqt, *hint, *gst, *hst, *ft;
  double *R, *filter;
  // numeric
  const int *sptr, *srow_ptr, *slot_ptr, *perm, *J_rowidx, *JT_ptr, *JT_ent;
  const int *srow, *snode, *level_sn, *lvl_ptr;  // lvl_ptr: level offsets into level_sn
  // supernodes of width B_WT < w <= B_WG of each level (level L owns g8_ptr[L] .. g8_ptr[L + 1])
  const int *g8_ptr, *g8_sn;
  // update pairs (precomputed per pattern), stored level by level: level L owns entries
  // lpair_ptr[L] .. lpair_ptr[L + 1]; each pair: the panel slots of rows i and j (i >= j >= w)
  // in column 0 of its supernode, ld << 8 | w of that panel, and the target value slot
  const int *lpair_ptr, *pair_a, *pair_b, *pair_m, *pair_tgt;
  // condensation order (per pattern): the lower panel slots of every supernode sorted by their
  // number of items (ccol: the variable of a diagonal slot, whose Sigma_x entry it takes, else
  // -1); the items of each group of
  // 32 slots are interleaved (item k of lane l at cgptr[g] + 32 k + l, padded with y = -2) so
  // that a warp's item loads are coalesced and its lanes loop over equal counts
  const int *cslot, *ccol, *cgptr;
  const int2 *citems;
  // the same items as two 16-bit indices (x, y + 2) when every index of the pattern fits, else
  // null: half the bytes of the condensation's index stream
  const ushort2 *citems16;
  int ncslot;
  const int64_t *lptr, *dptr;
  const int2 *items;
  int ns, nlevels;
  double *tJ, *Lx, *Dx;
  int *info;
  double *y, *t, *cx, *cz, *outx, *outz, *scal;
  double *cg_r, *cg_p, *cg_sp, *cg_dy, *cg_rhs1, *cg_v;  // HyKKT CG vectors
  // PCG after a stagnating refinement (LiftedKKT): condensed right-hand side t, r, z, p, K p
  // (n), d o (J v) (m), the refined solution kept for the comparison (n, m)
  double *pg_t, *pg_r, *pg_z, *pg_p, *pg_q, *pg_u, *pg_xs, *pg_zs;
  const double *dystep;  // dy of the step: cg_dy (HyKKT), dz over the G rows (form 2)
  AugArgs aug;
  // restoration phase: p, q and their duals, steps and trial values, row residuals (one per IPM
  // row), the reference point x_R and D_R^2 (n), the phase's filter (null without restoration)
  double *rp, *rq, *rzp, *rzq, *rdp, *rdq, *rdzp, *rdzq, *rpt, *rqt, *rrc, *rrp, *rrq;
  double *rxr, *rdr2, *rfilter;
};

// restoration-phase arguments of an instance (the element functions of resto_dev.cuh)
__device__ __forceinline__ RArgs rargs_b(const BI &I, const BCtl &c) {
  RArgs A;
  A.D = I.D;
  A.P = I.P;
  A.p = I.rp; A.q = I.rq; A.zp = I.rzp; A.zq = I.rzq;
  A.xr = I.rxr; A.dr2 = I.rdr2;
  A.sigma = (double *)I.SA.sigma; A.r1 = I.r1; A.r2 = (double *)I.SA.r2;
  A.Ds = (double *)I.SA.Ds;
  A.rc = I.rrc; A.rp = I.rrp; A.rq = I.rrq;
  A.mu = c.mu; A.zeta = c.zeta; A.dw = c.dw;
  A.dx = I.dx; A.jdx = I.SA.jdx;
  A.dy = (double *)I.dystep; A.dz = I.SA.dz; A.ds = I.SA.ds; A.dv = I.SA.dv;
  A.dzl = I.SA.dzl; A.dzu = I.SA.dzu;
  A.dp = I.rdp; A.dq = I.rdq; A.dzp = I.rdzp; A.dzq = I.rdzq;
  return A;
}
__device__ __forceinline__ int resto_nmax(const BI &I) {
  return max(I.D.n, max(I.D.me + I.D.mi, I.m));
}


#define B_PROLOGUE(want)                 \
  const int b = blockIdx.y;              \
  if (ctl[b].ph != (want)) return;       \
  const BI &I = bi[b];                   \
  const int gtid = blockIdx.x * blockDim.x + threadIdx.x; \
  const int gstride = gridDim.x * blockDim.x;

// ------------------------------------------------------------------ control helpers
__global__ void k_b_rreset(const BI *bi, const BCtl *ctl, int phase, int k0, int k1, double v) {
  const int b = blockIdx.x;
  if (ctl[b].ph != phase) return;
  for (int k = k0 + threadIdx.x; k < k1; k += blockDim.x) bi[b].R[k] = v;
}

// cg_maxit: HyKKT CG iteration limit (<= 0: m_e of the instance); 0 in the record = no CG
// p32: start with the FP32 factor (precision 32)
__global__ void k_b_ctl_init(const BI *bi, BCtl *ctl, int count, double mu0, int hykkt,
                             int cg_maxit, int p32) {
  int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= count) return;
  BCtl c;
  memset(&c, 0, sizeof(c));
  c.ph = PH_EVAL;
  c.mu = mu0;
  c.tau = fmax(TAU_MIN, 1.0 - mu0);
  c.sig = 1.0;
  c.eta = c.eta_prev = INFINITY;
  if (hykkt) c.cg_maxit = cg_maxit > 0 ? cg_maxit : max(bi[b].D.me0, 1);
  c.p32 = p32;
  c.k32 = -1;
  ctl[b] = c;
  for (int k = 0; k < R_COUNT; ++k) bi[b].R[k] = 0.0;
}

// ------------------------------------------------------------------ model evaluation
// mode 0: at x with J and grad f (the set-up); mode 1: J, grad f and W (with the scaled
// multipliers) at x (phase EVAL); mode 2: at the trial point, values only (phase LS)
struct EvalPtrs {
  const double *x, *y, *z;
  double sigf, *f, *grad, *g, *h, *Jv, *Wv;
};
__device__ __forceinline__ EvalPtrs eval_ptrs(const BI &I, const BCtl &c, int mode) {
  EvalPtrs E;
  if (mode == 0) {
    E = EvalPtrs{I.P.x, nullptr, nullptr, 1.0, I.f, I.P.grad, I.gs, I.hs, I.Jv, nullptr};
  } else if (mode == 1) {
    // (the restoration problem's W is the constraints' part only)
    E = EvalPtrs{I.P.x, I.lamw, I.lamw + I.D.me0, c.resto ? 0.0 : c.sig, I.f, I.P.grad, I.gs,
                 I.hs, I.Jv, I.Wv};
  } else {
    E = EvalPtrs{I.xt, nullptr, nullptr, 1.0, I.ft, nullptr, I.gst, I.hst, nullptr, nullptr};
  }
  return E;
}
__device__ __forceinline__ OpfDims opf_dims(const OpfData &M) {
  return OpfDims{M.nb, M.nbr, M.ng, M.n, M.me, M.mi, M.form};
}

__global__ void k_b_eval_init(const BI *bi, const BCtl *ctl, int phase, int mode) {
  B_PROLOGUE(phase);
  const EvalPtrs E = eval_ptrs(I, ctl[b], mode);
  const OpfData &M = I.M;
  eval_init_at(opf_dims(M), M.pd, M.qd, E.x, M.ref, E.g, E.Jv, E.Jv ? M.nnzJ : 0, E.Wv,
               E.Wv ? M.nnzW : 0, gtid, gstride);
}
__global__ void k_b_eval_branch(const BI *bi, const BCtl *ctl, int phase, int mode) {
  B_PROLOGUE(phase);
  const EvalPtrs E = eval_ptrs(I, ctl[b], mode);
  const OpfDims D = opf_dims(I.M);
  for (int e = gtid; e < 2 * D.nbr; e += gstride)
    eval_branch_at(D, I.M, E.x, E.y, E.z, E.g, E.h, E.Jv, E.Wv, e);
}
// one generator per thread (the grid covers the largest generator count): per-block cost parts
__global__ void k_b_eval_gen(const BI *bi, const BCtl *ctl, int phase, int mode) {
  __shared__ double sh[32];
  const int b = blockIdx.y;
  if (ctl[b].ph != phase) return;
  const BI &I = bi[b];
  const EvalPtrs E = eval_ptrs(I, ctl[b], mode);
  const OpfDims D = opf_dims(I.M);
  const int gi = blockIdx.x * blockDim.x + threadIdx.x;
  double fc = gi < D.ng ? eval_gen_at(D, I.M, E.x, E.sigf, E.g, E.grad, E.Jv, E.Wv, gi) : 0.0;
  block_sum_to(I.fpart + blockIdx.x, fc, sh);
}
__global__ void k_b_eval_finish(const BI *bi, const BCtl *ctl, int phase, int mode, int nparts) {
  B_PROLOGUE(phase);
  const EvalPtrs E = eval_ptrs(I, ctl[b], mode);
  eval_finish_at(opf_dims(I.M), I.M, I.fpart, nparts, E.f, E.grad, E.Jv, gtid, gstride);
}

// constraint scaling of the model outputs and the IPM rows; mode 0 also scales J
__global__ void k_b_scale_model(const BI *bi, const BCtl *ctl, int phase, int mode,
                                double relax_tau) {
  B_PROLOGUE(phase);
  const Dims &D = I.D;
  double *gs = mode == 0 ? I.gs : I.gst, *hs = mode == 0 ? I.hs : I.hst;
  double *geq = mode == 0 ? I.P.geq : I.geqt, *hin = mode == 0 ? I.P.hin : I.hint;
  const int nrow = max(D.me0, D.mi0);
  for (int k = gtid; k < nrow; k += gstride) {
    if (k < D.me0) gs[k] *= I.dscale[k];
    if (k < D.mi0) hs[k] *= I.dscale[D.me0 + k];
    ipm_rows_at(D, relax_tau, gs, hs, geq, hin, k);
  }
  if (mode == 0)
    for (int p = gtid; p < I.M.nnzJ; p += gstride) I.Jv[p] *= I.dscale[I.J_rowidx[p]];
}

// block-wide reduction of NQ values (op 0 sum, 1 max, 2 min; max / min values non-negative)
// with one atomic per value per block; every thread of the block (<= 256) must call
enum { OP_SUM = 0, OP_MAX = 1, OP_MIN = 2 };
template <int NQ>
__device__ __forceinline__ void block_reduce_atomic(double *R, const int (&slot)[NQ],
                                                    const int (&op)[NQ], double (&v)[NQ]) {
  __shared__ double sh[8][NQ];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int q = 0; q < NQ; ++q) {
    const double x = op[q] == OP_SUM ? wsum(v[q]) : op[q] == OP_MAX ? wmax(v[q]) : wmin(v[q]);
    if (lane == 0) sh[w][q] = x;
  }
  __syncthreads();
  if (threadIdx.x < NQ) {
    const int q = threadIdx.x;
    double a = sh[0][q];
    for (int k = 1; k < nw; ++k)
      a = op[q] == OP_SUM ? a + sh[k][q] : op[q] == OP_MAX ? fmax(a, sh[k][q]) : fmin(a, sh[k][q]);
    if (op[q] == OP_SUM) atomicAdd(R + slot[q], a);
    else if (op[q] == OP_MAX) amax_nonneg(R + slot[q], a);
    else amin_nonneg(R + slot[q], a);
  }
}

// ------------------------------------------------------------------ set-up
__global__ void k_b_setup_sums(const BI *bi, const BCtl *ctl) {
  B_PROLOGUE(PH_EVAL);
  double a = 0.0, q = 0.0;
  for (int i = gtid; i < I.M.nb; i += gstride) {
    a += I.M.pd[i];
    q += I.M.qd[i];
  }
  red_sum(I.R, R_PD, a);
  red_sum(I.R, R_QD, q);
}
__global__ void k_b_x0(const BI *bi, const BCtl *ctl) {
  B_PROLOGUE(PH_EVAL);
  for (int j = gtid; j < 2 * I.M.nb + 2 * I.M.ng; j += gstride)
    I.P.x[j] = x0_at(I.M.nb, I.M.ng, I.R[R_PD], I.R[R_QD], I.P.xl, I.P.xu, j);
}
// flow-variable form: each flow variable at the flow of the start voltages
__global__ void k_b_flow_start(const BI *bi, const BCtl *ctl) {
  B_PROLOGUE(PH_EVAL);
  if (!I.M.form) return;
  const OpfDims D = opf_dims(I.M);
  for (int e = gtid; e < 2 * D.nbr; e += gstride) flow_start_at(D, I.M, I.P.x, e);
}
__global__ void k_b_row_scale(const BI *bi, const BCtl *ctl) {
  B_PROLOGUE(PH_EVAL);
  for (int r = gtid; r < I.m; r += gstride) {
    double mx = 0.0;
    for (int p = I.M.J_rowptr[r]; p < I.M.J_rowptr[r + 1]; ++p) mx = fmax(mx, fabs(I.Jv[p]));
    I.dscale[r] = mx > 0.0 ? fmin(1.0, 100.0 / mx) : 1.0;
  }
  double g = 0.0;
  for (int j = gtid; j < I.D.n; j += gstride) g = fmax(g, fabs(I.P.grad[j]));
  red_max(I.R, R_MAXGRAD, g);
}
__global__ void k_b_ctl_sig(const BI *bi, BCtl *ctl, int count) {
  int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= count) return;
  ctl[b].sig = fmin(1.0, 100.0 / fmax(bi[b].R[R_MAXGRAD], 1e-300));
}
__global__ void k_b_init_duals(const BI *bi, const BCtl *ctl) {
  B_PROLOGUE(PH_EVAL);
  const int nmax = max(I.D.n, max(I.D.me, I.D.mi));
  for (int i = gtid; i < nmax; i += gstride) init_duals_at(I.D, I.P, I.P.s, i);
}

// ------------------------------------------------------------------ evaluation phase
// start of the restoration phase (instances that entered it in the line search): reference
// point, D_R^2, p and q in closed form, multipliers (resto_start_at); before k_b_lambda, since
// the constraint multipliers restart from zero
__global__ void k_b_resto_start(const BI *bi, const BCtl *ctl) {
  B_PROLOGUE(PH_EVAL);
  if (ctl[b].resto != 2) return;
  const RArgs A = rargs_b(I, ctl[b]);
  for (int i = gtid; i < resto_nmax(I); i += gstride)
    resto_start_at(A, ctl[b].mu, I.rxr, I.rdr2, i);
}
// multipliers of the model rows and their scaled copy (the weights of the constraint Hessians
// in W); they depend only on the iterate, so W is evaluated together with J at x
__global__ void k_b_lambda(const BI *bi, const BCtl *ctl) {
  B_PROLOGUE(PH_EVAL);
  const int nrow = max(I.D.me0, I.D.mi0);
  for (int k = gtid; k < nrow; k += gstride) {
    lambda_at(I.D, I.P.y, I.P.z, I.lam, k);
    if (k < I.D.me0) I.lamw[k] = I.lam[k] * I.dscale[k];
    if (k < I.D.mi0) I.lamw[I.D.me0 + k] = I.lam[I.D.me0 + k] * I.dscale[I.D.me0 + k];
  }
}
// the reduction slots of the EVAL phase: sums and maxima from 0, minima from +infinity
__global__ void k_b_rinit_eval(const BI *bi, const BCtl *ctl) {
  const int b = blockIdx.x;
  if (ctl[b].ph != PH_EVAL) return;
  for (int k = threadIdx.x; k < R_COUNT; k += blockDim.x)
    bi[b].R[k] = (k == R_SV_MIN || k == R_CL_MIN || k == R_CU_MIN) ? INFINITY : 0.0;
}
__global__ void k_b_jtu(const BI *bi, const BCtl *ctl) {
  B_PROLOGUE(PH_EVAL);
  for (int j = gtid; j < I.D.n; j += gstride) {
    double acc = 0.0;
    for (int t = I.JT_ptr[j]; t < I.JT_ptr[j + 1]; ++t) {
      int p = I.JT_ent[t];
      acc += I.Jv[p] * I.lam[I.J_rowidx[p]];
    }
    I.P.jtl[j] = acc;
  }
}
// optimality error parts (mu-independent maxima, sums, min / max of the complementarity
// products) and the merit parts at (x, s)
// Maxima and minima of non-negative values are kept on their bit patterns (integer compares,
// which order like the numbers and keep a NaN as the largest), the barrier logs in a LogSum
// (their total goes to R_LOG_S): both keep FP64 instructions for the sums.
__device__ __forceinline__ long long dbits(double v) { return __double_as_longlong(v); }
// the same parts for the restoration problem (its variables x, p, q; p, q >= 0 count among the
// lower bounds): x-gradient zeta D_R^2 (x - x_R) + J^T lambda - zl + zu, the p and q
// stationarity rows with z - v, the rows c - p + q (primal error and theta_R), products of p, q
// with their duals among the lower-bound products, the logs of s, p, q and the bound distances,
// and the restoration objective into R_RS_OBJ
__device__ void b_errors_resto(const BI &I, const BCtl &c, int gtid, int gstride) {
  const RArgs A = rargs_b(I, c);
  const Dims &D = I.D;
  const int R = D.me + D.mi;
  long long gl = 0, zv = 0, ge = 0, c0 = 0;
  const long long inf = dbits(INFINITY);
  long long svmin = inf, svmax = 0, clmin = inf, clmax = 0, cumin = inf, cumax = 0;
  double sy = 0, sz = 0, svv = 0, szl = 0, szu = 0, th = 0, ls = 0, obj = 0;
  auto cl = [&](double prod) {
    const long long q = dbits(prod);
    clmin = min(clmin, q);
    clmax = max(clmax, q);
  };
  for (int i = gtid; i < resto_nmax(I); i += gstride) {
    if (i < D.n) {
      const double x = I.P.x[i], e = x - I.rxr[i];
      gl = max(gl, dbits(fabs(c.zeta * I.rdr2[i] * e + I.P.jtl[i] - I.P.zl[i] + I.P.zu[i])));
      szl += fabs(I.P.zl[i]);
      szu += fabs(I.P.zu[i]);
      obj += 0.5 * c.zeta * I.rdr2[i] * e * e;
      if (isfinite(I.P.xl[i])) {
        cl((x - I.P.xl[i]) * I.P.zl[i]);
        ls += log(x - I.P.xl[i]);
      }
      if (isfinite(I.P.xu[i])) {
        const long long q = dbits((I.P.xu[i] - x) * I.P.zu[i]);
        cumin = min(cumin, q);
        cumax = max(cumax, q);
        ls += log(I.P.xu[i] - x);
      }
    }
    if (i < D.mi) {
      zv = max(zv, dbits(fabs(I.P.z[i] - I.P.v[i])));
      const long long q = dbits(I.P.s[i] * I.P.v[i]);
      svmin = min(svmin, q);
      svmax = max(svmax, q);
      sz += fabs(I.P.z[i]);
      svv += fabs(I.P.v[i]);
      ls += log(I.P.s[i]);
    }
    if (i < D.me) sy += fabs(I.P.y[i]);
    if (i < R) {
      const double lam = r_lam(A, i), p = I.rp[i], q = I.rq[i];
      zv = max(zv, dbits(fabs(RHO_RESTO - lam - I.rzp[i])));
      zv = max(zv, dbits(fabs(RHO_RESTO + lam - I.rzq[i])));
      const double ci = r_c(D, I.P.geq, I.P.hin, I.P.s, i), r = fabs(ci - p + q);
      c0 = max(c0, dbits(fabs(ci)));
      ge = max(ge, dbits(r));
      th += r;
      szl += fabs(I.rzp[i]) + fabs(I.rzq[i]);
      cl(p * I.rzp[i]);
      cl(q * I.rzq[i]);
      obj += RHO_RESTO * (p + q);
      ls += log(p) + log(q);
    }
  }
  // (R_RS_PRIM: the original problem's violation ||c||_inf)
  const int slot[20] = {R_MAX_GL, R_MAX_ZV, R_MAX_G, R_MAX_HS, R_SUM_Y, R_SUM_Z, R_SUM_V,
                        R_SUM_ZL, R_SUM_ZU, R_SV_MIN, R_SV_MAX, R_CL_MIN, R_CL_MAX, R_CU_MIN,
                        R_CU_MAX, R_TH_G, R_TH_H, R_LOG_S, R_RS_OBJ, R_RS_PRIM};
  const int op[20] = {OP_MAX, OP_MAX, OP_MAX, OP_MAX, OP_SUM, OP_SUM, OP_SUM, OP_SUM, OP_SUM,
                      OP_MIN, OP_MAX, OP_MIN, OP_MAX, OP_MIN, OP_MAX, OP_SUM, OP_SUM, OP_SUM,
                      OP_SUM, OP_MAX};
  auto d = [](long long x) { return __longlong_as_double(x); };
  double v[20] = {d(gl), d(zv), d(ge), 0.0, sy, sz, svv, szl, szu, d(svmin), d(svmax),
                  d(clmin), d(clmax), d(cumin), d(cumax), th, 0.0, ls, obj, d(c0)};
  block_reduce_atomic<20>(I.R, slot, op, v);
}
__global__ void k_b_errors(const BI *bi, const BCtl *ctl) {
  B_PROLOGUE(PH_EVAL);
  if (ctl[b].resto) {
    b_errors_resto(I, ctl[b], gtid, gstride);
    return;
  }
  const Dims &D = I.D;
  const double sig = ctl[b].sig;
  long long gl = 0, zv = 0, ge = 0, hs = 0;
  const long long inf = dbits(INFINITY);
  long long svmin = inf, svmax = 0, clmin = inf, clmax = 0, cumin = inf, cumax = 0;
  double sy = 0, sz = 0, svv = 0, szl = 0, szu = 0, tg = 0, th = 0;
  LogSum lg;
  const int nmax = max(D.n, max(D.me, D.mi));
  for (int i = gtid; i < nmax; i += gstride) {
    const ErrParts E = errors_at(D, I.P, sig, 0.0, i);
    gl = max(gl, dbits(E.gl));
    zv = max(zv, dbits(E.zv));
    ge = max(ge, dbits(E.ge));
    hs = max(hs, dbits(E.hs));
    sy += E.sy;
    sz += E.sz;
    svv += E.svv;
    szl += E.szl;
    szu += E.szu;
    // absent products are -1: a negative bit pattern
    const long long cs = dbits(E.csv), cl = dbits(E.ccl), cu = dbits(E.ccu);
    if (cs >= 0) { svmin = min(svmin, cs); svmax = max(svmax, cs); }
    if (cl >= 0) { clmin = min(clmin, cl); clmax = max(clmax, cl); }
    if (cu >= 0) { cumin = min(cumin, cu); cumax = max(cumax, cu); }
    if (i < D.me) tg += fabs(I.P.geq[i]);
    if (i < D.mi) {
      th += fabs(I.P.hin[i] + I.P.s[i]);
      lg.add(I.P.s[i]);
    }
    if (i < D.n) {
      if (isfinite(I.P.xl[i])) lg.add(I.P.x[i] - I.P.xl[i]);
      if (isfinite(I.P.xu[i])) lg.add(I.P.xu[i] - I.P.x[i]);
    }
  }
  const int slot[18] = {R_MAX_GL, R_MAX_ZV, R_MAX_G, R_MAX_HS, R_SUM_Y, R_SUM_Z, R_SUM_V,
                        R_SUM_ZL, R_SUM_ZU, R_SV_MIN, R_SV_MAX, R_CL_MIN, R_CL_MAX, R_CU_MIN,
                        R_CU_MAX, R_TH_G, R_TH_H, R_LOG_S};
  const int op[18] = {OP_MAX, OP_MAX, OP_MAX, OP_MAX, OP_SUM, OP_SUM, OP_SUM, OP_SUM, OP_SUM,
                      OP_MIN, OP_MAX, OP_MIN, OP_MAX, OP_MIN, OP_MAX, OP_SUM, OP_SUM, OP_SUM};
  auto d = [](long long x) { return __longlong_as_double(x); };
  double v[18] = {d(gl), d(zv), d(ge), d(hs), sy, sz, svv, szl, szu, d(svmin), d(svmax),
                  d(clmin), d(clmax), d(cumin), d(cumax), tg, th, lg.value()};
  block_reduce_atomic<18>(I.R, slot, op, v);
}

__device__ __forceinline__ double comp_mu(const double *h, double mu) {
  double c = 0.0;
  c = fmax(c, fmax(h[R_SV_MAX] - mu, mu - h[R_SV_MIN]));
  c = fmax(c, fmax(h[R_CL_MAX] - mu, mu - h[R_CL_MIN]));
  c = fmax(c, fmax(h[R_CU_MAX] - mu, mu - h[R_CU_MIN]));
  return c;
}

// convergence test, iteration limit, barrier update (repeated in the first iteration)
__global__ void k_b_ctl_eval(const BI *bi, BCtl *ctl, int count, double tol, int max_iter) {
  int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= count || ctl[b].ph != PH_EVAL) return;
  const BI &I = bi[b];
  BCtl c = ctl[b];
  const double *h = I.R;
  const bool rs = c.resto != 0;
  // the restoration problem has 2 (m_e + m_i) more lower bounds (p, q >= 0)
  const int nl = rs ? I.nl + 2 * (I.D.me + I.D.mi) : I.nl;
  c.obj = rs ? h[R_RS_OBJ] : *I.f;
  c.theta = h[R_TH_G] + h[R_TH_H];
  c.logsum = h[R_LOG_S] + h[R_LOG_XL] + h[R_LOG_XU];
  const double e0 = kkt_error(h, I.D, nl, I.nu, fmax(h[R_SV_MAX], fmax(h[R_CL_MAX], h[R_CU_MAX])));
  c.e0 = e0;
  if (c.resto == 2) c.resto = 1;
  if (!c.have_theta0) {
    c.theta_max = 1e4 * fmax(1.0, c.theta);
    c.theta_min = 1e-4 * fmax(1.0, c.theta);
    c.have_theta0 = 1;
  }
  if (e0 <= tol) {
    // a stationary point of the restoration problem before its return test passed: a local
    // minimizer of the constraint violation, unless that violation is within the tolerance (a
    // feasible point that the filter still rejects)
    c.status = !rs ? 1 : h[R_RS_PRIM] > tol ? IPM_ERR_INFEASIBLE : IPM_ERR_RESTORATION;
    c.ph = PH_DONE;
  } else if (!isfinite(e0)) {
    c.status = IPM_ERR_NONFINITE;
    c.ph = PH_DONE;
  } else if (rs ? c.k_r >= 500 : c.k >= max_iter) {
    c.status = rs ? IPM_ERR_RESTORATION : IPM_ERR_MAXITER;
    c.ph = PH_DONE;
  } else {
    bool first = true;
    const int kk = rs ? c.k_r : c.k;
    for (int rep = 0; rep < 200; ++rep) {
      const double emu = kkt_error(h, I.D, nl, I.nu, comp_mu(h, c.mu));
      if (!(emu <= KAPPA_EPS * c.mu && (first || kk == 0))) break;
      c.mu = fmax(tol / 10.0, fmin(KAPPA_MU * c.mu, pow(c.mu, THETA_MU)));
      c.tau = fmax(TAU_MIN, 1.0 - c.mu);
      c.nfilter = 0;
      first = false;
    }
    c.ph = PH_BUILD;
  }
  ctl[b] = c;
}

// ------------------------------------------------------------------ build phase
__global__ void k_b_newton_rhs(const BI *bi, const BCtl *ctl) {
  B_PROLOGUE(PH_BUILD);
  const Dims &D = I.D;
  if (ctl[b].resto) {
    const RArgs A = rargs_b(I, ctl[b]);
    for (int i = gtid; i < resto_nmax(I); i += gstride) {
      resto_rhs_at(A, i);
      if (i < D.n) I.a[i] = -I.r1[i];
    }
    return;
  }
  const int nmax = max(D.n, D.mi);
  for (int i = gtid; i < nmax; i += gstride) {
    newton_rhs_at(D, I.P, ctl[b].sig, ctl[b].mu, (double *)I.SA.sigma, I.r1, (double *)I.SA.r2,
                  (double *)I.SA.r4, (double *)I.SA.Ds, i);
    if (i < D.n) I.a[i] = -I.r1[i];
  }
}
// inertia search start: delta_w = 0, then delta_last / 3 (x8) or 1e-4 (x100)
__global__ void k_b_ctl_build(BCtl *ctl, int count) {
  int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= count || ctl[b].ph != PH_BUILD) return;
  BCtl &c = ctl[b];
  c.dw = 0.0;
  c.nfac = 0;
  c.grow = c.delta_last > 0 ? 8.0 : 100.0;
  c.next = c.delta_last > 0 ? fmax(1e-20, c.delta_last / 3.0) : 1e-4;
  c.n_reg = 0;
  c.ph = PH_FACT;
}

// ------------------------------------------------------------------ inertia rounds
__global__ void k_b_aug_rhs(const BI *bi, const BCtl *ctl, double gamma) {
  B_PROLOGUE(PH_FACT);
  const int nrow = max(I.D.me0, I.D.mi0);
  if (ctl[b].resto) {  // every row condensed, d = 1/E_r (resto_row)
    const RArgs A = rargs_b(I, ctl[b]);
    for (int k = gtid; k < nrow; k += gstride) resto_aug_at(A, I.dcond, I.baug, k);
    return;
  }
  for (int k = gtid; k < nrow; k += gstride)
    aug_rhs_at(I.D, ctl[b].dw, gamma, I.SA.r2, I.SA.r4, I.SA.Ds, I.P.geq, I.dcond, I.baug, k);
}
__global__ void k_b_scale_jv(const BI *bi, const BCtl *ctl) {
  B_PROLOGUE(PH_FACT);
  for (int p = gtid; p < I.M.nnzJ; p += gstride) I.tJ[p] = I.dcond[I.J_rowidx[p]] * I.Jv[p];
}

// ------------------------------------------------------------------ condensation
// one condensation item as (x, y): (J entry p, J entry q), (W entry, -1) or padding (-, -2)
__device__ __forceinline__ int2 citem(int2 q) { return q; }
__device__ __forceinline__ int2 citem(ushort2 q) { return make_int2(q.x, (int)q.y - 2); }

// the sum of one slot's items (list order), added to v; it: the slot's first item, the next one
// 32 entries further (items interleaved per group of 32 slots)
template <typename IT>
__device__ __forceinline__ double slot_items(const BI &I, const IT *it, int cnt, double v) {
  int k = 0;
  for (; k + 4 <= cnt; k += 4) {  // four items' loads in flight, summed in list order
    double a[4], m[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int2 q = citem(it[(k + u) * 32]);
      const bool wv = q.y < 0;
      a[u] = wv ? I.Wv[q.x] : I.tJ[q.x];
      m[u] = wv ? 1.0 : I.Jv[q.y];
      if (q.y == -2) a[u] = m[u] = 0.0;  // padding
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) v = fma(a[u], m[u], v);
  }
  for (; k < cnt; ++k) {
    const int2 q = citem(it[k * 32]);
    const bool wv = q.y < 0;
    double a = wv ? I.Wv[q.x] : I.tJ[q.x], m = wv ? 1.0 : I.Jv[q.y];
    if (q.y == -2) a = m = 0.0;
    v = fma(a, m, v);
  }
  return v;
}

// K = W + Sigma_x + delta_w I + J^T D J into the lower slots of every panel of the instances in
// the FACT phase (the diagonal block's upper triangle is never read), all slots of all instances
// in one launch (slots are independent); the W item of a slot is taken as W * 1 so that every
// lane issues the same fused multiply-add.  Also resets the factorization status.
__global__ void k_b_condense(const BI *bi, const BCtl *ctl) {
  B_PROLOGUE(PH_FACT);
  if (gtid == 0) *I.info = INT_MAX;
  const double dw = ctl[b].dw;
  const int p32 = ctl[b].p32;
  for (int t = gtid; t < I.ncslot; t += gstride) {
    const int slot = I.cslot[t], j = I.ccol[t], g = t >> 5;
    double v = j >= 0 ? I.SA.sigma[j] + dw : 0.0;
    const int off = I.cgptr[g] + (t & 31);
    const int cnt = (I.cgptr[g + 1] - I.cgptr[g]) >> 5;
    v = I.citems16 ? slot_items(I, I.citems16 + off, cnt, v) : slot_items(I, I.citems + off, cnt, v);
    if (p32)
      reinterpret_cast<float *>(I.Lx)[slot] = (float)v;  // summed in FP64, rounded once
    else
      I.Lx[slot] = v;
  }
}

// ------------------------------------------------------------------ per-instance numeric kernels
// One block per instance (a cluster of blocks for the big instances), level by level through the
// supernodal elimination tree (deepest level first for the factorization and the forward solve,
// root first for the backward solve): the supernodes of a level are independent, so a barrier
// between levels (block or cluster barrier) is the only synchronization.  In the factorization
// narrow supernodes (w <= B_WS) take one warp each and wider ones the whole block; in the solves
// every supernode takes one warp.  Contributions into other supernodes' panels (and into y) from
// one level are added atomically, since supernodes of a level may share targets.  No waits on
// blocks outside the instance's cluster.
static constexpr int B_WS = 16;
static constexpr int B_NT = 512;    // threads of the per-instance solve kernel
static constexpr int B_NT_F = 512;  // threads of the per-instance factorization kernel

// Updates of the supernodes of level L into their ancestors, every pair of the level spread over
// all threads of the cluster: entry (i, j), i >= j >= w, of L21 L21^T of supernode s is
// subtracted from the panel of the supernode owning column rows[j], at row rows[i].
template <typename T>
__device__ __forceinline__ void level_updates(const BI &I, T *Lx, int L, int tid, int nthreads) {
  const int p1 = I.lpair_ptr[L + 1];
  for (int t = I.lpair_ptr[L] + tid; t < p1; t += nthreads) {
    const int m = I.pair_m[t];
    const int w = m & 0xff, ld = m >> 8;
    const T *Pi = Lx + I.pair_a[t], *Pj = Lx + I.pair_b[t];
    T v = 0;
    int k = 0;
    for (; k + 4 <= w; k += 4) {  // four independent load pairs in flight
      T a[4], c[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        a[u] = Pi[(int64_t)(k + u) * ld];
        c[u] = Pj[(int64_t)(k + u) * ld];
      }
#pragma unroll
      for (int u = 0; u < 4; ++u) v += a[u] * c[u];
    }
    for (; k < w; ++k) v += Pi[(int64_t)k * ld] * Pj[(int64_t)k * ld];
    atomicAdd(&Lx[I.pair_tgt[t]], -v);
  }
}

// rows below the diagonal block of a narrow supernode of width W: L21 = A21 L11^{-T}, one row per
// lane held in registers (one load and one store per entry; the right-looking column loop then
// runs on registers instead of re-reading the panel)
template <int W, typename T>
__device__ __forceinline__ void rows_below(T *P, int ld, const T *D, const T *inv, int lane) {
  for (int r = W + lane; r < ld; r += 32) {
    T x[W];
#pragma unroll
    for (int k = 0; k < W; ++k) x[k] = P[r + (int64_t)k * ld];
#pragma unroll
    for (int k = 0; k < W; ++k) {
      x[k] *= inv[k];
#pragma unroll
      for (int j = k + 1; j < W; ++j) x[j] -= x[k] * D[j + k * W];
    }
#pragma unroll
    for (int k = 0; k < W; ++k) P[r + (int64_t)k * ld] = x[k];
  }
}

static constexpr int B_WT = 4;  // diagonal blocks up to this width are factored one per thread

// diagonal block of a narrow supernode (w <= B_WT) by one thread: L11 and its reciprocal pivots
// into Dd (the same arithmetic as the warp path); on GB300 an FP64 warp instruction costs the
// same with one lane active as with 32, so the pivots of a level go 32 per instruction
template <typename T>
__device__ void thread_diag_sn(const BI &I, T *Lx, T *Dx, int s) {
  const int f = I.sptr[s], w = I.sptr[s + 1] - f;
  const int ld = I.srow_ptr[s + 1] - I.srow_ptr[s];
  const T *P = Lx + I.lptr[s];
  T D[B_WT * B_WT], inv[B_WT];
#pragma unroll
  for (int k = 0; k < B_WT; ++k)
#pragma unroll
    for (int i = 0; i < B_WT; ++i) D[i + k * B_WT] = (k < w && i < w && i >= k) ? P[i + (int64_t)k * ld] : T(0);
#pragma unroll
  for (int k = 0; k < B_WT; ++k) {
    if (k < w) {
      T d = D[k + k * B_WT];
      if (!pivot_ok(d)) {
        atomicMin(I.info, f + k);
        d = 1;
      }
      const T iv = rsqrt_newton(d);
      D[k + k * B_WT] = d * iv;
      inv[k] = iv;
#pragma unroll
      for (int i = k + 1; i < B_WT; ++i)
        if (i < w) D[i + k * B_WT] *= iv;
#pragma unroll
      for (int j = k + 1; j < B_WT; ++j)
#pragma unroll
        for (int i = j; i < B_WT; ++i)
          if (i < w && j < w) D[i + j * B_WT] -= D[i + k * B_WT] * D[j + k * B_WT];
    }
  }
  T *Dd = Dx + I.dptr[s];
#pragma unroll
  for (int k = 0; k < B_WT; ++k)
#pragma unroll
    for (int i = 0; i < B_WT; ++i)
      if (k < w && i < w) Dd[i + k * w] = D[i + k * B_WT];
#pragma unroll
  for (int k = 0; k < B_WT; ++k)
    if (k < w) Dd[w * w + k] = inv[k];
}

static constexpr int B_WG = 8;  // diagonal blocks up to this width: one 8-lane group each

// diagonal block of a supernode of width B_WT < w <= B_WG by one group of 8 lanes (four
// supernodes per warp, s < 0: an idle group): lane i of the group holds row i of the block, and
// at step k every lane computes pivot k of its group (an FP64 warp instruction costs the same
// for 8 or 32 active lanes, so the four chains of pivots run in one instruction stream).  Writes
// L11 and the reciprocal pivots to Dd as thread_diag_sn does.
template <typename T>
__device__ void group_diag_sn(const BI &I, T *Lx, T *Dx, int s, int lane) {
  const int i = lane & 7, base = lane & ~7;
  int f = 0, w = 0, ld = 1;
  const T *P = nullptr;
  if (s >= 0) {
    f = I.sptr[s];
    w = I.sptr[s + 1] - f;
    ld = I.srow_ptr[s + 1] - I.srow_ptr[s];
    P = Lx + I.lptr[s];
  }
  T x[B_WG];
#pragma unroll
  for (int j = 0; j < B_WG; ++j) x[j] = (i < w && j <= i) ? P[i + (int64_t)j * ld] : T(0);
  T inv = 1;  // lane k keeps the reciprocal of pivot k
#pragma unroll
  for (int k = 0; k < B_WG; ++k) {
    T d = __shfl_sync(0xffffffffu, x[k], base + k);
    if (k < w) {
      if (!pivot_ok(d)) {
        if (i == k) atomicMin(I.info, f + k);
        d = 1;
      }
    } else {
      d = 1;
    }
    const T iv = rsqrt_newton(d);
    if (i == k) {
      x[k] = d * iv;
      inv = iv;
    } else if (i > k) {
      x[k] *= iv;
    }
    // trailing rows: x[j] -= L_ik L_jk for k < j <= i
#pragma unroll
    for (int j = k + 1; j < B_WG; ++j) {
      const T ljk = __shfl_sync(0xffffffffu, x[k], base + j);
      if (j <= i) x[j] -= x[k] * ljk;
    }
  }
  if (i < w) {
    T *Dd = Dx + I.dptr[s];
#pragma unroll
    for (int j = 0; j < B_WG; ++j)
      if (j < w) Dd[i + j * w] = j <= i ? x[j] : 0.0;
    Dd[w * w + i] = inv;
  }
}

// warp path: diagonal block, reciprocal pivots, L21 = A21 L11^{-T}, then the outer product of the
// rows below scattered into the target panels.  D: w*w doubles, inv: w doubles (this warp's).
template <typename T>
__device__ void warp_factor_sn(const BI &I, T *Lx, T *Dx, int s, T *D, T *inv) {
  const int lane = threadIdx.x & 31;
  const int f = I.sptr[s], w = I.sptr[s + 1] - f;
  const int rb = I.srow_ptr[s], ld = I.srow_ptr[s + 1] - rb;
  T *P = Lx + I.lptr[s];
  T *Dd = Dx + I.dptr[s];
  if (w <= B_WG) {  // factored by thread_diag_sn or group_diag_sn before this pass
    for (int t = lane; t < w * w; t += 32) D[t] = Dd[t];
    for (int k = lane; k < w; k += 32) inv[k] = Dd[w * w + k];
    __syncwarp();
  } else {
  for (int t = lane; t < w * w; t += 32) {
    const int k = t / w, i = t - k * w;
    D[t] = i >= k ? P[i + (int64_t)k * ld] : T(0);
  }
  __syncwarp();
  for (int k = 0; k < w; ++k) {
    if (lane == 0) {
      T d = D[k + k * w];
      if (!pivot_ok(d)) {
        atomicMin(I.info, f + k);
        d = 1;
      }
      const T iv = rsqrt_newton(d);
      D[k + k * w] = d * iv;
      inv[k] = iv;
    }
    __syncwarp();
    const T iv = inv[k];
    for (int i = k + 1 + lane; i < w; i += 32) D[i + k * w] *= iv;
    __syncwarp();
    const int nr = w - k - 1;
    for (int t = lane; t < nr * nr; t += 32) {
      const int j = k + 1 + t / nr, i = k + 1 + t % nr;
      if (i >= j) D[i + j * w] -= D[i + k * w] * D[j + k * w];
    }
    __syncwarp();
  }
  for (int t = lane; t < w * w; t += 32) Dd[t] = D[t];
  for (int k = lane; k < w; k += 32) Dd[w * w + k] = inv[k];
  __syncwarp();
  }
  // rows below: L21 = A21 L11^{-T}, lane-owned rows (the updates they cause run in the level's
  // update pass)
  switch (w) {
#define CIPM_RB_CASE(W) case W: rows_below<W>(P, ld, D, inv, lane); break;
    CIPM_RB_CASE(1) CIPM_RB_CASE(2) CIPM_RB_CASE(3) CIPM_RB_CASE(4) CIPM_RB_CASE(5)
    CIPM_RB_CASE(6) CIPM_RB_CASE(7) CIPM_RB_CASE(8)
#undef CIPM_RB_CASE
    default:  // 8 < w <= B_WS: the row in a thread-private array
      for (int r = w + lane; r < ld; r += 32) {
        T x[B_WS];
        for (int k = 0; k < w; ++k) x[k] = P[r + (int64_t)k * ld];
        for (int k = 0; k < w; ++k) {
          x[k] *= inv[k];
          for (int j = k + 1; j < w; ++j) x[j] -= x[k] * D[j + k * w];
        }
        for (int k = 0; k < w; ++k) P[r + (int64_t)k * ld] = x[k];
      }
  }
  __syncwarp();
}

// barrier of the bd threads of warp group `id` (named barrier 1 + id; bd a multiple of 32)
__device__ __forceinline__ void group_bar(int id, int bd) {
  switch (id) {  // constant barrier ids, so that the kernel reserves five barriers only
    case 0: asm volatile("bar.sync 1, %0;" ::"r"(bd) : "memory"); break;
    case 1: asm volatile("bar.sync 2, %0;" ::"r"(bd) : "memory"); break;
    case 2: asm volatile("bar.sync 3, %0;" ::"r"(bd) : "memory"); break;
    default: asm volatile("bar.sync 4, %0;" ::"r"(bd) : "memory"); break;
  }
}

// group path for a wide supernode: the bd threads (tid = 0 .. bd - 1) of warp group gid call;
// sm: w*w + 32*(w+1) doubles of this group, s_inv: w doubles of this group
template <typename T>
__device__ void block_factor_sn(const BI &I, T *Lx, T *Dx, int s, T *sm, T *s_inv, int tid,
                                int bd, int gid) {
  const int f = I.sptr[s], w = I.sptr[s + 1] - f;
  const int rb = I.srow_ptr[s], ld = I.srow_ptr[s + 1] - rb;
  T *P = Lx + I.lptr[s];
  T *sL = sm, *sR = sm + w * w;
  for (int t = tid; t < w * w; t += bd) {
    const int k = t / w, i = t - k * w;
    sL[t] = i >= k ? P[i + (int64_t)k * ld] : T(0);
  }
  group_bar(gid, bd);
  for (int k = 0; k < w; ++k) {
    if (tid == 0) {
      T d = sL[k + k * w];
      if (!pivot_ok(d)) {
        atomicMin(I.info, f + k);
        d = 1;
      }
      const T iv = rsqrt_newton(d);
      sL[k + k * w] = d * iv;
      s_inv[k] = iv;
    }
    group_bar(gid, bd);
    const T iv = s_inv[k];
    const int nr = w - k - 1;
    for (int i = k + 1 + tid; i < w; i += bd) sL[i + k * w] *= iv;
    group_bar(gid, bd);
    for (int jj = tid / 32; jj < nr; jj += bd / 32) {
      const int j = k + 1 + jj;
      const T ljk = sL[j + k * w];
      for (int i = j + (tid & 31); i < w; i += 32) sL[i + j * w] -= sL[i + k * w] * ljk;
    }
    group_bar(gid, bd);
  }
  T *Dd = Dx + I.dptr[s];
  for (int t = tid; t < w * w; t += bd) Dd[t] = sL[t];
  for (int k = tid; k < w; k += bd) Dd[w * w + k] = s_inv[k];
  // rows below in blocks of 32: each warp owns rows, lanes split the columns
  const int sw = w + 1;
  const int warp = tid >> 5, lane = tid & 31, nw = bd >> 5;
  for (int r0 = w; r0 < ld; r0 += 32) {
    const int nrow = min(32, ld - r0);
    group_bar(gid, bd);
    for (int t = tid; t < nrow * w; t += bd) {
      const int k = t / nrow, r = t - k * nrow;
      sR[r * sw + k] = P[(r0 + r) + (int64_t)k * ld];
    }
    group_bar(gid, bd);
    for (int k = 0; k < w; ++k) {
      const T iv = s_inv[k];
      for (int r = warp; r < nrow; r += nw) {
        const T xk = sR[r * sw + k] * iv;
        __syncwarp();
        for (int j = k + 1 + lane; j < w; j += 32) sR[r * sw + j] -= xk * sL[j + k * w];
        if (lane == 0) sR[r * sw + k] = xk;
        __syncwarp();
      }
    }
    group_bar(gid, bd);
    for (int t = tid; t < nrow * w; t += bd) {
      const int k = t / nrow, r = t - k * nrow;
      P[(r0 + r) + (int64_t)k * ld] = sR[r * sw + k];
    }
  }
  group_bar(gid, bd);
}

// Levels of one instance in precision T (the panels Lx and diagonal blocks Dx of a FP32 instance
// hold floats at the same slot indices); sm: the dynamic shared memory, cap_t elements of T.
template <typename T>
__device__ __forceinline__ void fact_levels(const BI &I, T *Lx, T *Dx, T *sm, int cap_t,
                                            int *s_wide, int &s_nwide, int crank, int ncl) {
  namespace cg = cooperative_groups;
  cg::cluster_group cluster = cg::this_cluster();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  const int gw = crank * nw + warp, gnw = ncl * nw;
  T *D = sm + warp * (B_WS * B_WS + B_WS), *inv = D + B_WS * B_WS;
  for (int L = 0; L < I.nlevels; ++L) {
    if (threadIdx.x == 0) s_nwide = 0;
    const int q0 = I.lvl_ptr[L], q1 = I.lvl_ptr[L + 1];
    for (int q = q0 + crank * blockDim.x + threadIdx.x; q < q1; q += ncl * blockDim.x) {
      const int s = I.level_sn[q];
      if (I.sptr[s + 1] - I.sptr[s] <= B_WT) thread_diag_sn(I, Lx, Dx, s);
    }
    {  // widths B_WT+1 .. B_WG: four supernodes per warp
      const int g0 = I.g8_ptr[L], g1 = I.g8_ptr[L + 1];
      for (int q = g0 + 4 * gw; q < g1; q += 4 * gnw) {
        const int qq = q + (lane >> 3);
        group_diag_sn(I, Lx, Dx, qq < g1 ? I.g8_sn[qq] : -1, lane);
      }
    }
    cluster.sync();  // warps of any block of the cluster read these pivots
    for (int q = q0 + gw; q < q1; q += gnw) {
      const int s = I.level_sn[q];
      if (I.sptr[s + 1] - I.sptr[s] <= B_WS) {
        warp_factor_sn(I, Lx, Dx, s, D, inv);
      } else if (lane == 0) {
        s_wide[atomicAdd(&s_nwide, 1)] = s;
      }
    }
    __syncthreads();
    if (s_nwide > 0) {
      // the wide supernodes of the level by G warp groups side by side (each with its own
      // shared-memory area), G as large as the level's count, the block's warps and the
      // dynamic shared memory allow
      int mw = 0;
      for (int k = 0; k < s_nwide; ++k) mw = max(mw, I.sptr[s_wide[k] + 1] - I.sptr[s_wide[k]]);
      const int need = mw * mw + 32 * (mw + 1) + mw;
      int G = s_nwide >= 3 ? 4 : s_nwide;
      while (G > 1 && G * need > cap_t) G >>= 1;
      const int bd = blockDim.x / G, gid = threadIdx.x / bd, gtid = threadIdx.x - gid * bd;
      T *gsm = sm + gid * need;
      for (int k = gid; k < s_nwide; k += G)
        block_factor_sn(I, Lx, Dx, s_wide[k], gsm, gsm + need - mw, gtid, bd, gid);
      __syncthreads();
    }
    cluster.sync();
    level_updates(I, Lx, L, crank * blockDim.x + threadIdx.x, ncl * blockDim.x);
    cluster.sync();
  }
}

// factorization of each instance in the FACT phase (panels condensed by k_b_condense): one
// block, or one thread-block cluster (big instances, launched with a cluster size), per
// instance.  Warps of the whole cluster share the narrow supernodes of a level; each block
// collects the wide ones its warps met and factors them with all its threads; a cluster barrier
// (release / acquire) separates the levels.  T = float factors the instances whose FP32 factor
// serves (p32 in the control record: panels and diagonal blocks hold floats at the same slot
// indices), T = double the others; a batch of precision 64 launches only the latter.
static constexpr int B_WIDE_CAP = 1024;  // wide supernodes per level and block

template <typename T>
__global__ void __launch_bounds__(B_NT_F, 3)
    k_b_fact_inst(const BI *bi, const BCtl *ctl, int smem_doubles, const int *order) {
  extern __shared__ __align__(16) unsigned char sm_raw[];
  __shared__ int s_wide[B_WIDE_CAP], s_nwide;
  namespace cg = cooperative_groups;
  cg::cluster_group cluster = cg::this_cluster();
  const int crank = (int)cluster.block_rank(), ncl = (int)cluster.num_blocks();
  const int b = order[blockIdx.x / ncl];
  // the same for every block of the cluster
  if (ctl[b].ph != PH_FACT || ctl[b].p32 != (int)(sizeof(T) == sizeof(float))) return;
  const BI &I = bi[b];
  fact_levels<T>(I, reinterpret_cast<T *>(I.Lx), reinterpret_cast<T *>(I.Dx),
                 reinterpret_cast<T *>(sm_raw), (int)(smem_doubles * sizeof(double) / sizeof(T)),
                 s_wide, s_nwide, crank, ncl);
}

// L11 and the reciprocal pivots of a supernode of width w <= B_WS copied to this warp's shared
// staging area with one load per lane (the triangular loops then read shared memory instead of
// issuing one global round trip per column); wider supernodes read them in place
template <typename T>
__device__ __forceinline__ const T *stage_diag(const T *Dd, int w, T *stage, int lane) {
  if (w > B_WS) return Dd;
  for (int t = lane; t < w * w + w; t += 32) stage[t] = Dd[t];
  __syncwarp();
  return stage;
}

// forward step of one supernode, one warp: y_own <- L11^{-1} y_own, y_below -= L21 y_own (ys:
// this warp's shared staging, w doubles, then L11 for w <= B_WS)
template <typename T>
__device__ void warp_fwd_sn(const BI &I, const T *Lx, const T *Dx, T *Y, int s, T *ys) {
  const int lane = threadIdx.x & 31;
  const int f = I.sptr[s], w = I.sptr[s + 1] - f;
  const int rb = I.srow_ptr[s], ld = I.srow_ptr[s + 1] - rb;
  const int *rows = I.srow + rb;
  const T *P = Lx + I.lptr[s];
  const T *Dd = stage_diag(Dx + I.dptr[s], w, ys + CIPM_SN_MAXW, lane), *rinv = Dd + w * w;
  for (int k = lane; k < w; k += 32) ys[k] = Y[f + k];
  __syncwarp();
  for (int k = 0; k < w; ++k) {
    if (lane == (k & 31)) ys[k] *= rinv[k];
    __syncwarp();
    const T yk = ys[k];
    for (int i = k + 1 + lane; i < w; i += 32) ys[i] -= Dd[i + k * w] * yk;
    __syncwarp();
  }
  for (int k = lane; k < w; k += 32) Y[f + k] = ys[k];
  for (int i = w + lane; i < ld; i += 32) {
    T acc = 0;
    int k = 0;
    for (; k + 4 <= w; k += 4) {  // four loads in flight
      T p[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) p[u] = P[i + (int64_t)(k + u) * ld];
#pragma unroll
      for (int u = 0; u < 4; ++u) acc += p[u] * ys[k + u];
    }
    for (; k < w; ++k) acc += P[i + (int64_t)k * ld] * ys[k];
    atomicAdd(&Y[rows[i]], -acc);
  }
  __syncwarp();
}

// backward step of one supernode, one warp: y_own <- L11^{-T} (y_own - L21^T y_below)
template <typename T>
__device__ void warp_bwd_sn(const BI &I, const T *Lx, const T *Dx, T *Y, int s, T *zs) {
  const int lane = threadIdx.x & 31;
  const int f = I.sptr[s], w = I.sptr[s + 1] - f;
  const int rb = I.srow_ptr[s], ld = I.srow_ptr[s + 1] - rb;
  const int *rows = I.srow + rb;
  const T *P = Lx + I.lptr[s];
  const T *Dd = stage_diag(Dx + I.dptr[s], w, zs + CIPM_SN_MAXW, lane), *rinv = Dd + w * w;
  if (w <= 32) {
    // zs = y_own - L21^T y_below: lane = g * W2 + k takes column k over the rows i = w + g
    // (mod G), then a shuffle tree over the G row groups (W2 = w rounded up to a power of two)
    int W2 = 1;
    while (W2 < w) W2 <<= 1;
    const int k = lane & (W2 - 1), g = lane / W2, G = 32 / W2;
    T acc = 0;
    if (k < w)
      for (int i = w + g; i < ld; i += G) acc += P[i + (int64_t)k * ld] * Y[rows[i]];
    for (int o = W2; o < 32; o <<= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (g == 0 && k < w) zs[k] = Y[f + k] - acc;
  } else {
    for (int k = 0; k < w; ++k) {
      T acc = 0;
      for (int i = w + lane; i < ld; i += 32) acc += P[i + (int64_t)k * ld] * Y[rows[i]];
      acc = warp_sum_t(acc);
      if (lane == 0) zs[k] = Y[f + k] - acc;
    }
  }
  __syncwarp();
  for (int k = w - 1; k >= 0; --k) {
    if (lane == (k & 31)) zs[k] *= rinv[k];
    __syncwarp();
    const T xk = zs[k];
    for (int j = lane; j < k; j += 32) zs[j] -= Dd[k + j * w] * xk;
    __syncwarp();
  }
  for (int k = lane; k < w; k += 32) Y[f + k] = zs[k];
  __syncwarp();
}

// forward and backward levels of one instance in precision T, then the scatter to x (FP64):
// Y is the permuted right-hand side (shared memory or the instance's y), ys this warp's staging
template <typename T>
__device__ __forceinline__ void solve_levels(const BI &I, const T *Lx, const T *Dx, T *Y, T *ys,
                                             double *x, int crank, int ncl) {
  namespace cg = cooperative_groups;
  cg::cluster_group cluster = cg::this_cluster();
  const int warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int gw = crank * nw + warp, gnw = ncl * nw;
  const int gt = crank * blockDim.x + threadIdx.x, gnt = ncl * blockDim.x;
  for (int k = gt; k < I.D.n; k += gnt) Y[k] = (T)I.t[I.perm[k]];
  cluster.sync();
  for (int L = 0; L < I.nlevels; ++L) {
    for (int q = I.lvl_ptr[L] + gw; q < I.lvl_ptr[L + 1]; q += gnw)
      warp_fwd_sn(I, Lx, Dx, Y, I.level_sn[q], ys);
    cluster.sync();
  }
  for (int L = I.nlevels - 1; L >= 0; --L) {
    for (int q = I.lvl_ptr[L] + gw; q < I.lvl_ptr[L + 1]; q += gnw)
      warp_bwd_sn(I, Lx, Dx, Y, I.level_sn[q], ys);
    cluster.sync();
  }
  for (int k = gt; k < I.D.n; k += gnt) x[I.perm[k]] = (double)Y[k];
}

// phase SOLVE: dx = K^{-1} t; phase REFINE: cx = K^{-1} t (t from k_b_jt_rhs), one cluster per
// instance: gather by the ordering, forward levels, backward levels, scatter.  With the FP32
// factor (p32) the triangular solves run in single precision (classical mixed-precision
// refinement: only the residual and the update of the refinement are FP64); T = float serves
// those instances, T = double the others.
template <typename T>
__global__ void __launch_bounds__(B_NT, 3)
    k_b_solve_inst(const BI *bi, const BCtl *ctl, int phase, int ycap, const int *order) {
  constexpr int kArea = CIPM_SN_MAXW + B_WS * B_WS + B_WS;  // per warp: ys, then L11 stage
  __shared__ double s_y[(B_NT / 32) * kArea];
  extern __shared__ __align__(16) double s_vec[];
  namespace cg = cooperative_groups;
  cg::cluster_group cluster = cg::this_cluster();
  const int crank = (int)cluster.block_rank(), ncl = (int)cluster.num_blocks();
  const int b = order[blockIdx.x / ncl];
  // the same for every block of the cluster
  if (ctl[b].ph != phase || ctl[b].p32 != (int)(sizeof(T) == sizeof(float))) return;
  const BI &I = bi[b];
  const int warp = threadIdx.x >> 5;
  double *x = phase == PH_SOLVE || phase == PH_CGI || phase == PH_CGX ? I.dx
              : phase == PH_CG ? I.cg_v : phase == PH_PCGI || phase == PH_PCG ? I.pg_z : I.cx;
  // the permuted right-hand side lives in this block's shared memory when the instance has
  // one block and n fits (ycap doubles): its loads and atomic updates then stay on the SM
  const bool in_smem = ncl == 1 && I.D.n <= ycap;
  T *Y = in_smem ? reinterpret_cast<T *>(s_vec) : reinterpret_cast<T *>(I.y);
  solve_levels<T>(I, reinterpret_cast<const T *>(I.Lx), reinterpret_cast<const T *>(I.Dx), Y,
                  reinterpret_cast<T *>(s_y) + warp * kArea, x, crank, ncl);
}

// ------------------------------------------------------------------ HyKKT CG (Eq. (10))
// CGI: t = a + J^T (d o b) = r1 + gamma G^T r2 (kept as rhs1), w = K_gamma^{-1} t (into dx);
// then r = G w - b_G, p = r, dy = 0, r.r.  CG: t = G^T p, v = K_gamma^{-1} t, Sp = G v,
// alpha = r.r / p.Sp, dy += alpha p, r -= alpha Sp, beta = r.r_new / r.r, p = r + beta p.
// CGX: t = rhs1 - G^T dy, dx = K_gamma^{-1} t, dz_H = d_H o (H dx - b_H).
__global__ void k_b_cgi_rhs(const BI *bi, const BCtl *ctl) {
  B_PROLOGUE(PH_CGI);
  for (int j = gtid; j < I.D.n; j += gstride) {
    double acc = 0.0;
    for (int t = I.JT_ptr[j]; t < I.JT_ptr[j + 1]; ++t) {
      const int p = I.JT_ent[t];
      const int r = I.J_rowidx[p];
      double v = I.Jv[p] * I.baug[r];
      v *= I.dcond[r];
      acc += v;
    }
    const double v = I.a[j] + acc;
    I.t[j] = v;
    I.cg_rhs1[j] = v;
  }
}
__device__ __forceinline__ double g_row_dot(const BI &I, int r, const double *x) {
  double acc = 0.0;
  for (int p = I.M.J_rowptr[r]; p < I.M.J_rowptr[r + 1]; ++p) acc += I.Jv[p] * x[I.M.J_colind[p]];
  return acc;
}
__global__ void k_b_cgi_start(const BI *bi, const BCtl *ctl) {
  B_PROLOGUE(PH_CGI);
  double rr = 0.0;
  for (int r = gtid; r < I.D.me0; r += gstride) {
    const double v = g_row_dot(I, r, I.dx) - I.baug[r];
    I.cg_r[r] = v;
    I.cg_p[r] = v;
    I.cg_dy[r] = 0.0;
    rr += v * v;
  }
  const int slot[1] = {R_CG_A};
  const int op[1] = {OP_SUM};
  double v1[1] = {rr};
  block_reduce_atomic<1>(I.R, slot, op, v1);
}
__global__ void k_b_ctl_cgi(const BI *bi, BCtl *ctl, int count, double rtol) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= count || ctl[b].ph != PH_CGI) return;
  BCtl &c = ctl[b];
  c.cg_rr = bi[b].R[R_CG_A];
  bi[b].R[R_CG_B] = 0.0;
  const double r0 = sqrt(c.cg_rr);
  c.cg_stop = fmax(rtol * r0, 1e-14);
  c.cg_it = 0;
  c.ph = r0 > c.cg_stop ? PH_CG : PH_CGX;
}
// t = G^T p (G = the first me0 rows of J)
__global__ void k_b_cg_u(const BI *bi, const BCtl *ctl) {
  B_PROLOGUE(PH_CG);
  for (int j = gtid; j < I.D.n; j += gstride) {
    double acc = 0.0;
    for (int t = I.JT_ptr[j]; t < I.JT_ptr[j + 1]; ++t) {
      const int p = I.JT_ent[t];
      const int r = I.J_rowidx[p];
      if (r < I.D.me0) acc += I.Jv[p] * I.cg_p[r];
    }
    I.t[j] = acc;
  }
}
__global__ void k_b_cg_sp(const BI *bi, const BCtl *ctl) {
  B_PROLOGUE(PH_CG);
  double psp = 0.0;
  for (int r = gtid; r < I.D.me0; r += gstride) {
    const double v = g_row_dot(I, r, I.cg_v);
    I.cg_sp[r] = v;
    psp += I.cg_p[r] * v;
  }
  const int slot[1] = {R_CG_B};
  const int op[1] = {OP_SUM};
  double v1[1] = {psp};
  block_reduce_atomic<1>(I.R, slot, op, v1);
}
__global__ void k_b_ctl_cg_alpha(const BI *bi, BCtl *ctl, int count) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= count || ctl[b].ph != PH_CG) return;
  BCtl &c = ctl[b];
  const double alpha = c.cg_rr / bi[b].R[R_CG_B];
  bi[b].R[R_CG_A] = 0.0;
  if (!isfinite(alpha)) {  // p.S p = 0: breakdown, as a non-finite step in hykkt_cg
    c.status = IPM_ERR_NONFINITE;
    c.ph = PH_DONE;
    return;
  }
  c.cg_alpha = alpha;
}
__global__ void k_b_cg_xr(const BI *bi, const BCtl *ctl) {
  B_PROLOGUE(PH_CG);
  const double al = ctl[b].cg_alpha;
  double rr = 0.0;
  for (int r = gtid; r < I.D.me0; r += gstride) {
    I.cg_dy[r] += al * I.cg_p[r];
    const double v = I.cg_r[r] - al * I.cg_sp[r];
    I.cg_r[r] = v;
    rr += v * v;
  }
  const int slot[1] = {R_CG_A};
  const int op[1] = {OP_SUM};
  double v1[1] = {rr};
  block_reduce_atomic<1>(I.R, slot, op, v1);
}
__global__ void k_b_ctl_cg_beta(const BI *bi, BCtl *ctl, int count) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= count || ctl[b].ph != PH_CG) return;
  BCtl &c = ctl[b];
  const double rr = bi[b].R[R_CG_A];
  bi[b].R[R_CG_B] = 0.0;
  c.cg_beta = rr / c.cg_rr;
  c.cg_rr = rr;
  ++c.cg_it;
  ++c.cg_total;
  if (!isfinite(rr)) {
    c.status = IPM_ERR_NONFINITE;
    c.ph = PH_DONE;
  } else if (sqrt(rr) <= c.cg_stop || c.cg_it >= c.cg_maxit) {
    c.ph = PH_CGX;  // at the iteration limit the step goes on inexact, as in hykkt_cg
  }
}
__global__ void k_b_cg_p(const BI *bi, const BCtl *ctl) {
  B_PROLOGUE(PH_CG);
  const double be = ctl[b].cg_beta;
  for (int r = gtid; r < I.D.me0; r += gstride) I.cg_p[r] = I.cg_r[r] + be * I.cg_p[r];
}
__global__ void k_b_cgx_rhs(const BI *bi, const BCtl *ctl) {
  B_PROLOGUE(PH_CGX);
  for (int j = gtid; j < I.D.n; j += gstride) {
    double acc = 0.0;
    for (int t = I.JT_ptr[j]; t < I.JT_ptr[j + 1]; ++t) {
      const int p = I.JT_ent[t];
      const int r = I.J_rowidx[p];
      if (r < I.D.me0) acc += I.Jv[p] * I.cg_dy[r];
    }
    I.t[j] = I.cg_rhs1[j] - acc;
  }
}
// dz over the H rows (into dzc after the G rows, as the recovery of form 2 reads it)
__global__ void k_b_cgx_dz(const BI *bi, const BCtl *ctl) {
  B_PROLOGUE(PH_CGX);
  for (int r = I.D.me0 + gtid; r < I.m; r += gstride)
    I.dzc[r] = I.dcond[r] * (g_row_dot(I, r, I.dx) - I.baug[r]);
}
__global__ void k_b_ctl_cgx(BCtl *ctl, int count, const int *pause_k) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= count || ctl[b].ph != PH_CGX) return;
  ctl[b].ph = ctl[b].k == *pause_k ? PH_PAUSE : PH_STEP;
}

// factor outcome: success -> solve; wrong inertia -> next delta_w
__global__ void k_b_ctl_fact(const BI *bi, BCtl *ctl, int count) {
  int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= count || ctl[b].ph != PH_FACT) return;
  const BI &I = bi[b];
  BCtl &c = ctl[b];
  ++c.nfac;
  ++c.total_fac;
  if (*I.info == INT_MAX) {
    if (c.dw > 0) c.delta_last = c.dw;
    if (c.cg_maxit > 0 && !c.resto) {  // HyKKT (the restoration problem: condensed solve)
      I.R[R_CG_A] = 0.0;
      c.ph = PH_CGI;
    } else {
      c.ph = PH_SOLVE;
    }
    return;
  }
  if (c.p32) {
    // the FP32 factorization broke down: that says nothing about the inertia of K (the matrix
    // rounded to FP32 and the FP32 pivots decide it), so the same delta_w is factored in FP64,
    // and the instance stays in FP64 for the rest of its solve
    c.p32 = 0;
    c.k32 = c.k;
    return;
  }
  c.dw = c.next;
  c.next *= c.grow;
  if (c.dw >= 1e40) {
    c.status = IPM_ERR_INERTIA;
    c.ph = PH_DONE;
  }
}

// ------------------------------------------------------------------ condensed solve
// phase SOLVE: dx = K^{-1}(a + J^T (d o b)), dz = d o (J dx - b);
// phase REFINE: the same for the residual (outx, outz) into (cx, cz)
__global__ void k_b_jt_rhs(const BI *bi, const BCtl *ctl, int phase) {
  B_PROLOGUE(phase);
  const double *u = phase == PH_SOLVE ? I.baug : I.outz;
  const double *base = phase == PH_SOLVE ? I.a : I.outx;
  for (int j = gtid; j < I.D.n; j += gstride) {
    double acc = 0.0;
    for (int t = I.JT_ptr[j]; t < I.JT_ptr[j + 1]; ++t) {
      int p = I.JT_ent[t];
      int r = I.J_rowidx[p];
      double v = I.Jv[p] * u[r];
      v *= I.dcond[r];
      acc += v;
    }
    I.t[j] = base[j] + acc;
  }
}

__global__ void k_b_recover_dz(const BI *bi, const BCtl *ctl, int phase) {
  B_PROLOGUE(phase);
  const double *x = phase == PH_SOLVE ? I.dx : I.cx;
  const double *rb = phase == PH_SOLVE ? I.baug : I.outz;
  double *dz = phase == PH_SOLVE ? I.dzc : I.cz;
  for (int r = gtid; r < I.m; r += gstride) {
    double acc = 0.0;
    for (int p = I.M.J_rowptr[r]; p < I.M.J_rowptr[r + 1]; ++p) acc += I.Jv[p] * x[I.M.J_colind[p]];
    dz[r] = I.dcond[r] * (acc - rb[r]);
  }
}
__global__ void k_b_ctl_solved(const BI *bi, BCtl *ctl, int count) {
  int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= count || ctl[b].ph != PH_SOLVE) return;
  BCtl &c = ctl[b];
  c.ref_it = 0;
  c.ref_steps = 0;
  c.eta = c.eta_prev = INFINITY;
  c.ph = PH_REFINE;
}

// ------------------------------------------------------------------ refinement rounds
__global__ void k_b_resid(const BI *bi, const BCtl *ctl, int phase) {
  __shared__ double sh[32];
  B_PROLOGUE(phase);
  AugArgs A = I.aug;
  A.dw = ctl[b].dw;
  double res = 0.0, solv = 0.0, rhsv = 0.0, asum = 0.0;
  for (int i = gtid; i < A.n + A.m; i += gstride) {
    double as = 0.0, r;
    if (i < A.n) {
      r = aug_resid_x_at(A, i, &as);
      A.outx[i] = r;
      solv = fmax(solv, fabs(A.sx[i]));
      rhsv = fmax(rhsv, fabs(A.ra[i]));
    } else {
      const int q = i - A.n;
      r = aug_resid_z_at(A, q, &as);
      A.outz[q] = r;
      solv = fmax(solv, fabs(A.sz[q]));
      rhsv = fmax(rhsv, fabs(A.rb[q]));
    }
    res = fmax(res, fabs(r));
    asum = fmax(asum, as);
  }
  block_max_to(&A.scal[0], res, sh);
  block_max_to(&A.scal[1], solv, sh);
  block_max_to(&A.scal[2], rhsv, sh);
  block_max_to(&A.scal[3], asum, sh);
}
// a KKT solve ends with backward error eta: counted, then the step (or the hold)
__device__ __forceinline__ void solve_done(BCtl &c, double eta, const int *pause_k) {
  c.eta = eta;
  ++c.n_solve;
  if (!(eta <= 1e-10)) ++c.n_above;
  c.eta_worst = fmax(c.eta_worst, eta);
  c.ph = !c.resto && c.k == *pause_k ? PH_PAUSE : PH_STEP;
}

// Richardson test: stop at eta <= 1e-10, after max_refine corrections, or when eta stops
// halving; otherwise one more correction.  With pcg_on (LiftedKKT), an FP64 solve left above
// 1e-10 goes on with conjugate gradients on the condensed system (PH_PCGI)
__global__ void k_b_ctl_ref(const BI *bi, BCtl *ctl, int count, int max_refine,
                            const int *pause_k, int pcg_on) {
  int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= count || ctl[b].ph != PH_REFINE) return;
  const BI &I = bi[b];
  BCtl &c = ctl[b];
  const double *sc = I.scal;
  if (c.ref_it == 0) c.normA = sc[3];
  const double den = c.normA * sc[1] + sc[2];
  const double eta = den > 0 ? sc[0] / den : 0.0;
  c.eta = eta;
  bool stop;
  if (!isfinite(eta)) {
    c.status = IPM_ERR_NONFINITE;
    c.ph = PH_DONE;
    return;
  }
  const int cap = c.p32 ? B_REFINE32 : max_refine;
  stop = eta <= 1e-10 || c.ref_it >= cap || (c.ref_it > 0 && eta > 0.5 * c.eta_prev);
  ++c.ref_it;
  if (stop) {
    if (c.p32) {
      if (!(eta <= 1e-10)) {
        // the FP32 factor does not refine this solve to 1e-10 (cond(K) u_32 not small): the
        // instance refactors at the same delta_w in FP64 and keeps FP64 from now on
        c.p32 = 0;
        c.k32 = c.k;
        c.ph = PH_FACT;
        return;
      }
      ++c.it32;
    } else if (pcg_on && !(eta <= 1e-10) && max_refine > 0) {
      // the last correction is taken back when it made the solution worse
      c.pg_undo = c.ref_it > 1 && !(eta <= c.eta_prev);
      c.pg_eta0 = c.pg_undo ? c.eta_prev : eta;
      bi[b].R[R_PG_A] = bi[b].R[R_PG_B] = bi[b].R[R_PG_C] = 0.0;
      c.ph = PH_PCGI;
      return;
    }
    solve_done(c, eta, pause_k);
    return;
  }
  c.eta_prev = eta;
  ++c.ref_steps;
  ++c.total_ref;
}
__global__ void k_b_scal_zero(const BI *bi, const BCtl *ctl, int phase) {
  const int b = blockIdx.x;
  if (ctl[b].ph != phase) return;
  if (threadIdx.x < 4) bi[b].scal[threadIdx.x] = 0.0;
}
__global__ void k_b_axpy(const BI *bi, const BCtl *ctl) {
  B_PROLOGUE(PH_REFINE);
  for (int j = gtid; j < I.D.n; j += gstride) I.dx[j] += I.cx[j];
  for (int r = gtid; r < I.m; r += gstride) I.dzc[r] += I.cz[r];
}

// ------------------------------------------------------------------ PCG after stagnation
// LiftedKKT: Richardson refinement that stalls above 1e-10 (cond(K) eps_mach near one) is
// followed, as in the single-problem solve, by conjugate gradients on the condensed system
//   K dx = t,  K = W + Sigma_x + delta_w I + J^T D J,  t = a + J^T (d o b),
// preconditioned by the same factor and started from the refined dx (at most B_PCG_MAXIT
// iterations, stop at ||r||_2 <= 1e-14 ||t||_2 or at non-positive curvature); then
// dz = d o (J dx - b), and the refined solution is restored when it had the smaller backward
// error of the augmented system.
// PCGI: take back a worsening last correction, keep the refined solution, t and ||t||^2
__global__ void k_b_pg_save(const BI *bi, const BCtl *ctl) {
  B_PROLOGUE(PH_PCGI);
  const bool undo = ctl[b].pg_undo;
  double tt = 0.0;
  for (int j = gtid; j < I.D.n; j += gstride) {
    const double x = undo ? I.dx[j] - I.cx[j] : I.dx[j];
    I.dx[j] = x;
    I.pg_xs[j] = x;
    double acc = 0.0;
    for (int t = I.JT_ptr[j]; t < I.JT_ptr[j + 1]; ++t) {
      const int p = I.JT_ent[t];
      const int r = I.J_rowidx[p];
      acc += I.Jv[p] * (I.dcond[r] * I.baug[r]);
    }
    const double v = I.a[j] + acc;
    I.pg_t[j] = v;
    tt += v * v;
  }
  for (int r = gtid; r < I.m; r += gstride) {
    const double z = undo ? I.dzc[r] - I.cz[r] : I.dzc[r];
    I.dzc[r] = z;
    I.pg_zs[r] = z;
  }
  const int slot[1] = {R_PG_C};
  const int op[1] = {OP_SUM};
  double v1[1] = {tt};
  block_reduce_atomic<1>(I.R, slot, op, v1);
}
// u = d o (J v), v = dx (PCGI) or p (PCG)
__global__ void k_b_pg_ju(const BI *bi, const BCtl *ctl, int phase) {
  B_PROLOGUE(phase);
  const double *v = phase == PH_PCGI ? I.dx : I.pg_p;
  for (int r = gtid; r < I.m; r += gstride) I.pg_u[r] = I.dcond[r] * g_row_dot(I, r, v);
}
// (W + Sigma_x + delta_w I) v + J^T u at column j
__device__ __forceinline__ double kmat_at(const BI &I, double dw, const double *v, int j) {
  double acc = (I.SA.sigma[j] + dw) * v[j];
  for (int p = I.aug.W_rowptr[j]; p < I.aug.W_rowptr[j + 1]; ++p)
    acc += I.Wv[p] * v[I.aug.W_colind[p]];
  for (int t = I.aug.WT_ptr[j]; t < I.aug.WT_ptr[j + 1]; ++t) {
    const int e = I.aug.WT_ent[t];
    const int r = I.aug.W_rowidx[e];
    if (r != j) acc += I.Wv[e] * v[r];
  }
  for (int t = I.JT_ptr[j]; t < I.JT_ptr[j + 1]; ++t) {
    const int p = I.JT_ent[t];
    acc += I.Jv[p] * I.pg_u[I.J_rowidx[p]];
  }
  return acc;
}
// PCGI: r = t - K dx (also the solve's right-hand side), r.r; PCG: q = K p, p.q
__global__ void k_b_pg_k(const BI *bi, const BCtl *ctl, int phase) {
  B_PROLOGUE(phase);
  const double dw = ctl[b].dw;
  double acc = 0.0;
  if (phase == PH_PCGI) {
    for (int j = gtid; j < I.D.n; j += gstride) {
      const double r = I.pg_t[j] - kmat_at(I, dw, I.dx, j);
      I.pg_r[j] = r;
      I.t[j] = r;
      acc += r * r;
    }
  } else {
    for (int j = gtid; j < I.D.n; j += gstride) {
      const double q = kmat_at(I, dw, I.pg_p, j);
      I.pg_q[j] = q;
      acc += I.pg_p[j] * q;
    }
  }
  const int slot[1] = {phase == PH_PCGI ? R_PG_B : R_PG_C};
  const int op[1] = {OP_SUM};
  double v1[1] = {acc};
  block_reduce_atomic<1>(I.R, slot, op, v1);
}
// after the preconditioner solve z = M^{-1} r: r.z; PCGI also p = z
__global__ void k_b_pg_rz(const BI *bi, const BCtl *ctl, int phase) {
  B_PROLOGUE(phase);
  double rz = 0.0;
  for (int j = gtid; j < I.D.n; j += gstride) {
    rz += I.pg_r[j] * I.pg_z[j];
    if (phase == PH_PCGI) I.pg_p[j] = I.pg_z[j];
  }
  const int slot[1] = {R_PG_A};
  const int op[1] = {OP_SUM};
  double v1[1] = {rz};
  block_reduce_atomic<1>(I.R, slot, op, v1);
}
__global__ void k_b_ctl_pgi(const BI *bi, BCtl *ctl, int count) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= count || ctl[b].ph != PH_PCGI) return;
  BCtl &c = ctl[b];
  double *R = bi[b].R;
  c.pg_rz = R[R_PG_A];
  c.pg_tn = sqrt(R[R_PG_C]);
  const double rn = sqrt(R[R_PG_B]);
  R[R_PG_A] = R[R_PG_B] = R[R_PG_C] = 0.0;
  c.pg_it = 0;
  ++c.pg_runs;
  c.ph = rn <= 1e-14 * c.pg_tn || !isfinite(rn) ? PH_PCGX : PH_PCG;
}
// alpha = r.z / p.K p (r.z of the previous iteration's preconditioned residual after the first)
__global__ void k_b_ctl_pg_alpha(const BI *bi, BCtl *ctl, int count) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= count || ctl[b].ph != PH_PCG) return;
  BCtl &c = ctl[b];
  double *R = bi[b].R;
  if (c.pg_it > 0) {
    c.pg_rz = R[R_PG_A];
    R[R_PG_A] = 0.0;
  }
  const double pq = R[R_PG_C];
  R[R_PG_C] = 0.0;
  if (!(pq > 0.0) || !isfinite(c.pg_rz)) {  // non-positive curvature: stop with the iterate
    c.ph = PH_PCGX;
    return;
  }
  c.cg_alpha = c.pg_rz / pq;
}
// dx += alpha p, r -= alpha q (also the solve's right-hand side), r.r
__global__ void k_b_pg_xr(const BI *bi, const BCtl *ctl) {
  B_PROLOGUE(PH_PCG);
  const double al = ctl[b].cg_alpha;
  double rr = 0.0;
  for (int j = gtid; j < I.D.n; j += gstride) {
    I.dx[j] += al * I.pg_p[j];
    const double r = I.pg_r[j] - al * I.pg_q[j];
    I.pg_r[j] = r;
    I.t[j] = r;
    rr += r * r;
  }
  const int slot[1] = {R_PG_B};
  const int op[1] = {OP_SUM};
  double v1[1] = {rr};
  block_reduce_atomic<1>(I.R, slot, op, v1);
}
__global__ void k_b_ctl_pg_check(const BI *bi, BCtl *ctl, int count) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= count || ctl[b].ph != PH_PCG) return;
  BCtl &c = ctl[b];
  double *R = bi[b].R;
  const double rn = sqrt(R[R_PG_B]);
  R[R_PG_B] = 0.0;
  ++c.pg_it;
  ++c.pg_total;
  if (!isfinite(rn) || rn <= 1e-14 * c.pg_tn || c.pg_it >= B_PCG_MAXIT) c.ph = PH_PCGX;
}
// p = z + beta p, beta = r.z (new) / r.z (old)
__global__ void k_b_pg_p(const BI *bi, const BCtl *ctl) {
  B_PROLOGUE(PH_PCG);
  const double be = I.R[R_PG_A] / ctl[b].pg_rz;
  for (int j = gtid; j < I.D.n; j += gstride) I.pg_p[j] = I.pg_z[j] + be * I.pg_p[j];
}
// PCGX: dz = d o (J dx - b), then the residual of the augmented system (k_b_resid)
__global__ void k_b_pg_dz(const BI *bi, const BCtl *ctl) {
  B_PROLOGUE(PH_PCGX);
  for (int r = gtid; r < I.m; r += gstride)
    I.dzc[r] = I.dcond[r] * (g_row_dot(I, r, I.dx) - I.baug[r]);
}
// the better of the refined and the PCG solution (smaller backward error)
__global__ void k_b_ctl_pgx(const BI *bi, BCtl *ctl, int count, const int *pause_k) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= count || ctl[b].ph != PH_PCGX) return;
  BCtl &c = ctl[b];
  const double *sc = bi[b].scal;
  const double den = c.normA * sc[1] + sc[2];
  const double eta = den > 0 ? sc[0] / den : 0.0;
  c.pg_restore = !(eta < c.pg_eta0);
  solve_done(c, c.pg_restore ? c.pg_eta0 : eta, pause_k);
}
// the refined solution back where it was the better one (after k_b_ctl_pgx; the flag is
// cleared when the step begins)
__global__ void k_b_pg_restore(const BI *bi, const BCtl *ctl) {
  const int b = blockIdx.y;
  if (!ctl[b].pg_restore) return;
  const BI &I = bi[b];
  const int gtid = blockIdx.x * blockDim.x + threadIdx.x, gstride = gridDim.x * blockDim.x;
  for (int j = gtid; j < I.D.n; j += gstride) I.dx[j] = I.pg_xs[j];
  for (int r = gtid; r < I.m; r += gstride) I.dzc[r] = I.pg_zs[r];
}

// ------------------------------------------------------------------ step
__global__ void k_b_jv(const BI *bi, const BCtl *ctl) {
  B_PROLOGUE(PH_STEP);
  for (int r = gtid; r < I.m; r += gstride) {
    double acc = 0.0;
    for (int p = I.M.J_rowptr[r]; p < I.M.J_rowptr[r + 1]; ++p) acc += I.Jv[p] * I.dx[I.M.J_colind[p]];
    ((double *)I.SA.jdx)[r] = acc;
  }
}
__global__ void k_b_recover(const BI *bi, const BCtl *ctl) {
  B_PROLOGUE(PH_STEP);
  if (ctl[b].resto) {
    const RArgs A = rargs_b(I, ctl[b]);
    for (int i = gtid; i < resto_nmax(I); i += gstride) resto_recover_at(A, i);
    return;
  }
  StepArgs A = I.SA;
  A.mu = ctl[b].mu;
  A.dw = ctl[b].dw;
  const int nmax = max(I.D.n, I.D.mi);
  for (int i = gtid; i < nmax; i += gstride) recover_at(A, i);
}
__global__ void k_b_ftb(const BI *bi, const BCtl *ctl) {
  B_PROLOGUE(PH_STEP);
  StepArgs A = I.SA;
  A.mu = ctl[b].mu;
  A.dw = ctl[b].dw;
  double ap = 1.0, az = 1.0, gx = 0.0, gs = 0.0;
  if (ctl[b].resto) {
    const RArgs R = rargs_b(I, ctl[b]);
    for (int i = gtid; i < resto_nmax(I); i += gstride) {
      double pa, za, g;
      resto_ftb_at(R, ctl[b].tau, &pa, &za, &g, i);
      ap = fmin(ap, pa);
      az = fmin(az, za);
      gx += g;
    }
  } else {
    const int nmax = max(I.D.n, I.D.mi);
    for (int i = gtid; i < nmax; i += gstride) {
      const FtbParts F = ftb_at(A, ctl[b].tau, ctl[b].sig, i);
      ap = fmin(ap, F.ap);
      az = fmin(az, F.az);
      gx += F.gx;
      gs += F.gs;
    }
  }
  const int slot[4] = {R_AMAX, R_AZ, R_GPHI_X, R_GPHI_S};
  const int op[4] = {OP_MIN, OP_MIN, OP_SUM, OP_SUM};
  double v[4] = {ap, az, gx, gs};
  block_reduce_atomic<4>(I.R, slot, op, v);
}
__global__ void k_b_ctl_ls0(const BI *bi, BCtl *ctl, int count) {
  int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= count || ctl[b].ph != PH_STEP) return;
  const double *h = bi[b].R;
  BCtl &c = ctl[b];
  c.pg_restore = 0;  // (k_b_pg_restore has run)
  c.amax = h[R_AMAX];
  c.az = h[R_AZ];
  c.gphi = h[R_GPHI_X] + h[R_GPHI_S];
  c.phi = (c.resto ? 1.0 : c.sig) * c.obj - c.mu * c.logsum;
  const double theta = c.theta, gphi = c.gphi;
  if (gphi < 0)
    c.amin = GAMMA_ALPHA * fmin(GAMMA_THETA, fmin(GAMMA_PHI * theta / -gphi,
                                                  DELTA_SW * pow(theta, S_THETA) / pow(-gphi, S_PHI)));
  else
    c.amin = GAMMA_ALPHA * GAMMA_THETA;
  c.alpha = c.amax;
  c.ls = 0;
  c.ph = PH_LS;
}

// ------------------------------------------------------------------ line search
__global__ void k_b_trial(const BI *bi, const BCtl *ctl) {
  B_PROLOGUE(PH_LS);
  const double a = ctl[b].alpha;
  if (ctl[b].resto) {
    const int R = I.D.me + I.D.mi;
    for (int i = gtid; i < resto_nmax(I); i += gstride) {
      trial_at(I.D.n, I.D.mi, a, I.P.x, I.dx, I.P.s, I.SA.ds, I.xt, I.st, i);
      if (i < R) {
        I.rpt[i] = I.rp[i] + a * I.rdp[i];
        I.rqt[i] = I.rq[i] + a * I.rdq[i];
      }
    }
    return;
  }
  const int nmax = max(I.D.n, I.D.mi);
  for (int i = gtid; i < nmax; i += gstride)
    trial_at(I.D.n, I.D.mi, a, I.P.x, I.dx, I.P.s, I.SA.ds, I.xt, I.st, i);
}
// restoration trial: theta_R, its objective and logs (resto_merit_at), and the original
// problem's theta and barrier logs at the trial point for the return test
__device__ void b_merit_trial_resto(const BI &I, const BCtl &c, int gtid, int gstride) {
  const RArgs A = rargs_b(I, c);
  const Dims &D = I.D;
  double th = 0, obj = 0, ls = 0, th0 = 0, ls0 = 0;
  for (int i = gtid; i < resto_nmax(I); i += gstride) {
    const RMerit M = resto_merit_at(A, I.xt, I.st, I.rpt, I.rqt, I.geqt, I.hint, i);
    th += M.th;
    obj += M.obj;
    ls += M.ls + M.lxl + M.lxu;
    if (i < D.me) th0 += fabs(I.geqt[i]);
    if (i < D.mi) {
      th0 += fabs(I.hint[i] + I.st[i]);
      ls0 += log(I.st[i]);
    }
    ls0 += M.lxl + M.lxu;
  }
  const int slot[5] = {R_TH_G, R_RS_OBJ, R_LOG_S, R_RS_TH0, R_RS_LOG0};
  const int op[5] = {OP_SUM, OP_SUM, OP_SUM, OP_SUM, OP_SUM};
  double v[5] = {th, obj, ls, th0, ls0};
  block_reduce_atomic<5>(I.R, slot, op, v);
}
__global__ void k_b_merit_trial(const BI *bi, const BCtl *ctl) {
  B_PROLOGUE(PH_LS);
  if (ctl[b].resto) {
    b_merit_trial_resto(I, ctl[b], gtid, gstride);
    return;
  }
  const Dims &D = I.D;
  double tg = 0, th = 0;
  LogSum lg;  // the barrier logs (total into R_LOG_S)
  const int nmax = max(D.n, max(D.me, D.mi));
  for (int i = gtid; i < nmax; i += gstride) {
    if (i < D.me) tg += fabs(I.geqt[i]);
    if (i < D.mi) {
      th += fabs(I.hint[i] + I.st[i]);
      lg.add(I.st[i]);
    }
    if (i < D.n) {
      if (isfinite(I.P.xl[i])) lg.add(I.xt[i] - I.P.xl[i]);
      if (isfinite(I.P.xu[i])) lg.add(I.P.xu[i] - I.xt[i]);
    }
  }
  const int slot[3] = {R_TH_G, R_TH_H, R_LOG_S};
  const int op[3] = {OP_SUM, OP_SUM, OP_SUM};
  double v[3] = {tg, th, lg.value()};
  block_reduce_atomic<3>(I.R, slot, op, v);
}
// filter acceptance (Ipopt: switching condition with the Armijo test on phi, else sufficient
// decrease in theta or phi against the filter); backtrack by halves down to alpha_min
// resto_on: a failed line search of the main problem enters the restoration phase
// (Waechter & Biegler 2006, Sec. 3.3) at the current point, whose filter entry the phase must
// beat; mu_R = max(mu, ||c||_inf) with ||c||_inf the primal error of this iteration's evaluation
__global__ void k_b_ctl_ls(const BI *bi, BCtl *ctl, int count, int resto_on, double tol) {
  int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= count || ctl[b].ph != PH_LS) return;
  const BI &I = bi[b];
  BCtl &c = ctl[b];
  const double *h = I.R;
  const bool rs = c.resto != 0;
  const double tht = h[R_TH_G] + h[R_TH_H];
  const double logs = h[R_LOG_S] + h[R_LOG_XL] + h[R_LOG_XU];
  const double pht = rs ? h[R_RS_OBJ] - c.mu * logs : c.sig * (*I.ft) - c.mu * logs;
  const double theta = c.theta, phi = c.phi, gphi = c.gphi, alpha = c.alpha;
  int ftype = 0;
  const bool accepted = filter_accept(theta, phi, gphi, alpha, tht, pht, rs ? I.rfilter : I.filter,
                                      c.nfilter, c.theta_min, c.theta_max, &ftype);
  if (accepted) {
    c.ftype = ftype;
    c.ph = PH_ACC;
    if (rs) {
      // return test: the original violation at most KAPPA_RESTO times the phase's start, and
      // the point acceptable to the original filter with the start's entry
      const double th0 = h[R_RS_TH0], ph0 = c.sig * (*I.ft) - c.mu_m * h[R_RS_LOG0];
      bool back = th0 <= KAPPA_RESTO * c.theta_start && th0 < c.theta_max_m &&
                  (th0 < c.entry_theta || ph0 < c.entry_phi);
      for (int q = 0; back && q < c.nfilter_m; ++q)
        if (!(th0 < I.filter[2 * q] || ph0 < I.filter[2 * q + 1])) back = false;
      c.ret = back;
    }
    return;
  }
  ++c.ls;
  ++c.total_ls;
  c.alpha = alpha * 0.5;
  if (c.alpha < c.amin) {
    // (no phase at a point already feasible within the tolerance: it cannot reduce a violation
    // at rounding level; the direction is first recomputed with the next delta_w of this
    // iteration's inertia-correction schedule, a better conditioned and more gradient-like
    // step, at most MAX_LS_REGULARIZE times: the same iterate goes back to the factorization)
    const bool feasible = fmax(h[R_MAX_G], h[R_MAX_HS]) <= tol;
    if (!rs && resto_on && feasible && c.n_reg < MAX_LS_REGULARIZE) {
      ++c.n_reg;
      c.dw = c.next;
      c.next *= c.grow;
      if (c.dw >= 1e40) {
        c.status = IPM_ERR_INERTIA;
        c.ph = PH_DONE;
        return;
      }
      c.ph = PH_FACT;
      return;
    }
    if (rs || !resto_on || feasible) {
      c.status = IPM_ERR_RESTORATION;
      c.ph = PH_DONE;
      return;
    }
    c.mu_m = c.mu;
    c.tau_m = c.tau;
    c.delta_last_m = c.delta_last;
    c.theta_max_m = c.theta_max;
    c.theta_min_m = c.theta_min;
    c.nfilter_m = c.nfilter;
    c.entry_theta = (1 - GAMMA_THETA) * theta;
    c.entry_phi = phi - GAMMA_PHI * theta;
    c.theta_start = theta;
    c.mu = fmax(c.mu, fmax(h[R_MAX_G], h[R_MAX_HS]));
    c.zeta = sqrt(c.mu);
    c.tau = fmax(TAU_MIN, 1.0 - c.mu);
    c.delta_last = 0.0;
    c.nfilter = 0;
    c.have_theta0 = 0;
    c.k_r = 0;
    c.ret = 0;
    c.resto = 2;
    ++c.n_resto;
    ++c.k;
    c.ph = PH_EVAL;
  }
}

// ------------------------------------------------------------------ accept
__global__ void k_b_accept(const BI *bi, const BCtl *ctl) {
  B_PROLOGUE(PH_ACC);
  if (ctl[b].resto) {
    const RArgs R = rargs_b(I, ctl[b]);
    const bool back = ctl[b].ret != 0;
    for (int i = gtid; i < resto_nmax(I); i += gstride) {
      resto_accept_at(R, ctl[b].alpha, ctl[b].az, I.xt, I.st, I.rpt, I.rqt, i);
      if (back) resto_finish_at(I.D, I.P, i);
    }
    return;
  }
  StepArgs A = I.SA;
  A.mu = ctl[b].mu;
  A.dw = ctl[b].dw;
  const int nmax = max(I.D.n, max(I.D.me, I.D.mi));
  for (int i = gtid; i < nmax; i += gstride)
    accept_at(A, ctl[b].alpha, ctl[b].az, I.xt, I.st, I.dystep, i);
}
// adds (theta_f, phi_f) to a filter of n entries; when full, merges it into the entry that is
// dominated the most (largest theta), which keeps a valid (conservative) filter
__device__ void filter_add(double *F, int &n, int cap, double theta_f, double phi_f) {
  if (n < cap) {
    F[2 * n] = theta_f;
    F[2 * n + 1] = phi_f;
    ++n;
  } else {
    int q = 0;
    for (int k = 1; k < n; ++k)
      if (F[2 * k] > F[2 * q]) q = k;
    F[2 * q] = fmin(F[2 * q], theta_f);
    F[2 * q + 1] = fmin(F[2 * q + 1], phi_f);
  }
}
__global__ void k_b_ctl_acc(const BI *bi, BCtl *ctl, int count, int fmax_entries) {
  int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= count || ctl[b].ph != PH_ACC) return;
  BCtl &c = ctl[b];
  const bool rs = c.resto != 0;
  if (!c.ftype)
    filter_add(rs ? bi[b].rfilter : bi[b].filter, c.nfilter, fmax_entries,
               (1 - GAMMA_THETA) * c.theta, c.phi - GAMMA_PHI * c.theta);
  if (rs) {
    ++c.k_r;
    ++c.total_resto;
    if (c.ret) {
      // back to the main problem, whose filter takes the phase's starting entry
      c.mu = c.mu_m;
      c.tau = c.tau_m;
      c.delta_last = c.delta_last_m;
      c.theta_max = c.theta_max_m;
      c.theta_min = c.theta_min_m;
      c.nfilter = c.nfilter_m;
      c.have_theta0 = 1;
      filter_add(bi[b].filter, c.nfilter, fmax_entries, c.entry_theta, c.entry_phi);
      c.resto = 0;
      c.ret = 0;
    }
  } else {
    ++c.k;
  }
  c.ph = PH_EVAL;
}

__global__ void k_b_count(const BCtl *ctl, int count, int *active) {
  int b = blockIdx.x * blockDim.x + threadIdx.x;
  int a = b < count && ctl[b].ph != PH_DONE && ctl[b].ph != PH_PAUSE;
  a = __syncthreads_count(a);
  if (threadIdx.x == 0 && a) atomicAdd(active, a);
}
__global__ void k_b_resume(BCtl *ctl, int count) {
  int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b < count && ctl[b].ph == PH_PAUSE) ctl[b].ph = PH_STEP;
}
__global__ void k_b_finish_unfinished(BCtl *ctl, int count) {
  int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b < count && ctl[b].ph != PH_DONE && ctl[b].ph != PH_PAUSE) {
    ctl[b].status = IPM_ERR_MAXITER;
    ctl[b].ph = PH_DONE;
  }
}

// ------------------------------------------------------------------ learned warm start
// Row of an instance for training and prediction: x (n), log s (mi), log v (mi), log zl (n),
// log zu (n) (0 where the bound is absent), then y (me: the equality multipliers of HyKKT and
// the dual-regularized form; none for LiftedKKT); the iterate as the IPM holds it (scaled).
__global__ void k_b_state_rows(const BI *bi, float *out, int64_t ld) {
  const int b = blockIdx.y;
  const BI &I = bi[b];
  const int n = I.D.n, mi = I.D.mi;
  float *o = out + (int64_t)b * ld;
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x) {
    o[j] = (float)I.P.x[j];
    o[n + 2 * mi + j] = isfinite(I.P.xl[j]) ? (float)log(I.P.zl[j]) : 0.f;
    o[2 * n + 2 * mi + j] = isfinite(I.P.xu[j]) ? (float)log(I.P.zu[j]) : 0.f;
  }
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < mi; i += gridDim.x * blockDim.x) {
    o[n + i] = (float)log(I.P.s[i]);
    o[n + mi + i] = (float)log(I.P.v[i]);
  }
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < I.D.me; i += gridDim.x * blockDim.x)
    o[3 * n + 2 * mi + i] = (float)I.P.y[i];
}

__device__ __forceinline__ float denorm(const float *pred, const float *mean, const float *stdv,
                                        int j) {
  return mean ? pred[j] * stdv[j] + mean[j] : pred[j];
}

// pass 1: count non-finite predicted values and sum s v (into R_QD, R_PD)
__global__ void k_b_warm_check(const BI *bi, const float *pred, int64_t ld, const float *mean,
                               const float *stdv) {
  const int b = blockIdx.y;
  const BI &I = bi[b];
  const int n = I.D.n, mi = I.D.mi, w = 3 * n + 2 * mi + I.D.me;
  const float *p = pred + (int64_t)b * ld;
  double bad = 0.0, sv = 0.0;
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < w; j += gridDim.x * blockDim.x) {
    const float v = denorm(p, mean, stdv, j);
    if (!isfinite(v)) bad += 1.0;
    if (j >= n && j < n + mi) sv += exp((double)v + (double)denorm(p, mean, stdv, j + mi));
  }
  red_sum(I.R, R_QD, bad);
  red_sum(I.R, R_PD, sv);
}

// pass 2: the iterate of every instance whose prediction is finite: x pushed inside its bounds,
// s = exp(log s), z = v = exp(log v), zl, zu = exp(.) where the bound exists
__global__ void k_b_warm_apply(const BI *bi, const float *pred, int64_t ld, const float *mean,
                               const float *stdv) {
  const int b = blockIdx.y;
  const BI &I = bi[b];
  if (I.R[R_QD] != 0.0) return;
  const int n = I.D.n, mi = I.D.mi;
  const float *p = pred + (int64_t)b * ld;
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x) {
    const double xl = I.P.xl[j], xu = I.P.xu[j];
    const bool hl = isfinite(xl), hu = isfinite(xu);
    double pl = hl ? KAPPA1 * fmax(1.0, fabs(xl)) : 0.0, pu = hu ? KAPPA1 * fmax(1.0, fabs(xu)) : 0.0;
    if (hl && hu) {
      pl = fmin(pl, KAPPA1 * (xu - xl));
      pu = fmin(pu, KAPPA1 * (xu - xl));
    }
    double v = denorm(p, mean, stdv, j);
    if (hl) v = fmax(v, xl + pl);
    if (hu) v = fmin(v, xu - pu);
    I.P.x[j] = v;
    I.P.zl[j] = hl ? exp((double)denorm(p, mean, stdv, n + 2 * mi + j)) : 0.0;
    I.P.zu[j] = hu ? exp((double)denorm(p, mean, stdv, 2 * n + 2 * mi + j)) : 0.0;
  }
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < mi; i += gridDim.x * blockDim.x) {
    I.P.s[i] = exp((double)denorm(p, mean, stdv, n + i));
    const double v = exp((double)denorm(p, mean, stdv, n + mi + i));
    I.P.v[i] = v;
    I.P.z[i] = v;
  }
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < I.D.me; i += gridDim.x * blockDim.x)
    I.P.y[i] = (double)denorm(p, mean, stdv, 3 * n + 2 * mi + i);
}

// pass 3: barrier parameter mu0 = s^T v / m_i of the predicted point, fresh filter
__global__ void k_b_warm_ctl(const BI *bi, BCtl *ctl, int count, double tol, int *used) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= count) return;
  const BI &I = bi[b];
  const int ok = I.R[R_QD] == 0.0;
  used[b] = ok;
  if (!ok) return;
  BCtl &c = ctl[b];
  c.mu = fmax(I.R[R_PD] / (double)max(I.D.mi, 1), tol / 10.0);
  c.tau = fmax(TAU_MIN, 1.0 - c.mu);
  c.nfilter = 0;
  c.have_theta0 = 0;
  c.delta_last = 0.0;
}

}  // namespace cipm

using namespace cipm;

// ------------------------------------------------------------------ host side
struct ipm_batch_s {
  int count = 0;
  ipm_options opt;
  cudaStream_t stream = 0;
  std::vector<ipm_opf_t> opf;
  std::vector<ipm_sym_t> syms;  // one per distinct pattern
  std::vector<int> pat;         // instance -> pattern
  double *dpool = nullptr;
  int *ipool = nullptr;
  size_t dpool_len = 0, ipool_len = 0;
  BI *d_bi = nullptr;
  BCtl *d_ctl = nullptr;
  std::vector<void *> bufs;  // per-pattern level offsets
  int *d_tickets = nullptr;  // scratch counters: active count at [8], pause iteration at [12]
  int *d_order = nullptr;  // small instances by decreasing supernode count, then the big ones
  // tail of a run (batches of more than tail_active instances): once at most tail_active are
  // still running, the sweeps hold more inertia rounds and line-search trials (a round then
  // costs little) and, with tail_cl > 0, run every instance on clusters of tail_cl blocks;
  // d_order_all lists every instance by decreasing supernode count
  int tail_active = 16, tail_cl = 8;
  int fact_rounds = B_FACT_ROUNDS, ls_rounds = B_LS_ROUNDS;  // of the sweep being captured
  int *d_order_all = nullptr;
  cudaGraph_t graph_tail = nullptr;
  cudaGraphExec_t exec_tail = nullptr;
  int n_small = 0, n_big = 0;
  // launch shapes (ipm_batch_autotune): cluster size of the big instances, "big" = supernode
  // count above big_num / big_den times the median (big_den = 0: none), blocks per instance of
  // the element kernels
  int cl_big = 4, big_num = 6, big_den = 5;
  cudaStream_t side = nullptr;  // second branch of the sweep: the big instances
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  int *h_active = nullptr;                       // pinned
  int gx = 1, gx_gen = 1, max_ns = 1, fmax_entries = 0;
  size_t fact_smem = 0;
  int gx_cond = 1;  // blocks per instance of the condensation
  size_t solve_smem = 0;  // dynamic shared memory of the solve launches: the right-hand side
  int solve_ycap = 0;     // doubles of it
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  int launches_per_sweep = 0;
  int sweeps = 0;
  int max_iter = 3000;  // iteration limit of the captured sweep
  // kernel timing (ipm_batch_set_timing): events around both factorization launches and the
  // first solve of every sweep, recorded inside the sweep (graph event nodes when captured)
  bool timing = false;
  cudaEvent_t ev[6] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
  double t_fact_ms = 0.0, t_solve_ms = 0.0;
  int t_n = 0;
  double *x_stage = nullptr;  // all instances' x, contiguous (ipm_batch_export_all)
  std::vector<int64_t> x_off;
  int64_t x_total = 0;
};

namespace {

struct Bump {
  size_t n = 0;
  size_t take(size_t k) {
    size_t o = n;
    n += (std::max<size_t>(k, 1) + 31) & ~size_t(31);
    return o;
  }
};

int pattern_of(const OpfData &M, std::vector<int> &out) {
  const int m = M.me + M.mi;
  out.resize(4 + (m + 1) + M.nnzJ + (M.n + 1) + M.nnzW);
  int *o = out.data();
  o[0] = M.n;
  o[1] = M.me;
  o[2] = M.mi;
  o[3] = M.nnzJ;
  o += 4;
  CK(cudaMemcpy(o, M.J_rowptr, sizeof(int) * (m + 1), cudaMemcpyDeviceToHost));
  o += m + 1;
  CK(cudaMemcpy(o, M.J_colind, sizeof(int) * M.nnzJ, cudaMemcpyDeviceToHost));
  o += M.nnzJ;
  CK(cudaMemcpy(o, M.W_rowptr, sizeof(int) * (M.n + 1), cudaMemcpyDeviceToHost));
  o += M.n + 1;
  CK(cudaMemcpy(o, M.W_colind, sizeof(int) * M.nnzW, cudaMemcpyDeviceToHost));
  return IPM_OK;
}

int b_smem_limits() {
  static bool done = false;
  if (done) return IPM_OK;
  CK(cudaFuncSetAttribute(k_b_fact_inst<double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                          64 * 1024));
  CK(cudaFuncSetAttribute(k_b_fact_inst<float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                          64 * 1024));
  CK(cudaFuncSetAttribute(k_b_solve_inst<double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                          64 * 1024));
  CK(cudaFuncSetAttribute(k_b_solve_inst<float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                          64 * 1024));
  done = true;
  return IPM_OK;
}


// every kernel of one sweep, in order; returns the number of launches
int enqueue_sweep(ipm_batch_t B, cudaStream_t s) {
  const int C = B->count;
  const dim3 g2(B->gx, C), blk(B_BLOCK);
  const int gc = grid_for(C, 128);
  const double tol = B->opt.tol, relax = B->opt.tau;
  BI *bi = B->d_bi;
  BCtl *ctl = B->d_ctl;
  int n = 0;
  auto L = [&](int k) { n += k; };
  auto rreset = [&](int phase, int k0, int k1, double v) {
    k_b_rreset<<<C, 32, 0, s>>>(bi, ctl, phase, k0, k1, v);
    L(1);
  };
  auto eval = [&](int phase, int mode) {
    k_b_eval_init<<<g2, blk, 0, s>>>(bi, ctl, phase, mode);
    k_b_eval_branch<<<g2, blk, 0, s>>>(bi, ctl, phase, mode);
    k_b_eval_gen<<<dim3(B->gx_gen, C), blk, 0, s>>>(bi, ctl, phase, mode);
    k_b_eval_finish<<<g2, blk, 0, s>>>(bi, ctl, phase, mode, B->gx_gen);
    L(4);
  };
  auto rec = [&](int k) -> int {
    if (B->timing) CK(cudaEventRecordWithFlags(B->ev[k], s, cudaEventRecordExternal));
    return IPM_OK;
  };
  // one launch for the one-block instances on s and, in a concurrent branch, one cluster launch
  // for the big ones (order: small instances first, then big)
  auto split = [&](auto kernel, int nt, size_t smem, auto... args) -> int {
    if (B->n_big) {
      CK(cudaEventRecord(B->ev_fork, s));
      CK(cudaStreamWaitEvent(B->side, B->ev_fork, 0));
      cudaLaunchConfig_t cfg = {};
      cudaLaunchAttribute at[1];
      at[0].id = cudaLaunchAttributeClusterDimension;
      at[0].val.clusterDim.x = B->cl_big;
      at[0].val.clusterDim.y = 1;
      at[0].val.clusterDim.z = 1;
      cfg.gridDim = dim3(B->n_big * B->cl_big);
      cfg.blockDim = dim3(nt);
      cfg.dynamicSmemBytes = smem;
      cfg.stream = B->side;
      cfg.attrs = at;
      cfg.numAttrs = 1;
      CK(cudaLaunchKernelEx(&cfg, kernel, bi, ctl, args..., (const int *)(B->d_order + B->n_small)));
      L(1);
    }
    if (B->n_small) {
      kernel<<<B->n_small, nt, smem, s>>>(bi, ctl, args..., (const int *)B->d_order);
      L(1);
    }
    CKL();
    if (B->n_big) {
      CK(cudaEventRecord(B->ev_join, B->side));
      CK(cudaStreamWaitEvent(s, B->ev_join, 0));
    }
    return IPM_OK;
  };
  auto solve = [&](int phase) -> int {
    k_b_jt_rhs<<<g2, blk, 0, s>>>(bi, ctl, phase);
    if (phase == PH_SOLVE) CKR(rec(2));
    if (B->opt.precision == 32)  // the instances whose FP32 factor serves
      CKR(split(k_b_solve_inst<float>, B_NT, B->solve_smem, phase, B->solve_ycap));
    CKR(split(k_b_solve_inst<double>, B_NT, B->solve_smem, phase, B->solve_ycap));
    if (phase == PH_SOLVE) CKR(rec(3));
    k_b_recover_dz<<<g2, blk, 0, s>>>(bi, ctl, phase);
    L(2);
    return IPM_OK;
  };
  const bool resto_on = !B->opt.no_resto;
  // evaluate f, grad f, g, h, J and W at x, optimality error, convergence, barrier update
  if (resto_on) {
    k_b_resto_start<<<g2, blk, 0, s>>>(bi, ctl);
    L(1);
  }
  k_b_lambda<<<g2, blk, 0, s>>>(bi, ctl);
  L(1);
  eval(PH_EVAL, 1);
  k_b_scale_model<<<g2, blk, 0, s>>>(bi, ctl, PH_EVAL, 0, relax);
  k_b_jtu<<<g2, blk, 0, s>>>(bi, ctl);
  k_b_rinit_eval<<<C, 32, 0, s>>>(bi, ctl);
  L(3);
  k_b_errors<<<g2, blk, 0, s>>>(bi, ctl);
  k_b_ctl_eval<<<gc, 128, 0, s>>>(bi, ctl, C, tol, B->max_iter);
  L(2);
  // Newton right-hand sides
  k_b_newton_rhs<<<g2, blk, 0, s>>>(bi, ctl);
  k_b_ctl_build<<<gc, 128, 0, s>>>(ctl, C);
  L(2);
  // inertia rounds: condense + factor with the current delta_w
  // (timing: the first round between events 0 and 1, the others between 4 and 5)
  for (int r = 0; r < B->fact_rounds; ++r) {
    k_b_aug_rhs<<<g2, blk, 0, s>>>(bi, ctl, B->opt.gamma);
    k_b_scale_jv<<<g2, blk, 0, s>>>(bi, ctl);
    if (r <= 1) CKR(rec(r == 0 ? 0 : 4));
    k_b_condense<<<dim3(B->gx_cond, C), blk, 0, s>>>(bi, ctl);
    L(1);
    if (B->opt.precision == 32)
      CKR(split(k_b_fact_inst<float>, B_NT_F, B->fact_smem, (int)(B->fact_smem / sizeof(double))));
    CKR(split(k_b_fact_inst<double>, B_NT_F, B->fact_smem, (int)(B->fact_smem / sizeof(double))));
    if (r == 0 || r == B->fact_rounds - 1) CKR(rec(r == 0 ? 1 : 5));
    k_b_ctl_fact<<<gc, 128, 0, s>>>(bi, ctl, C);
    L(3);
  }
  if (B->opt.kkt == 1) {
    // HyKKT: CG on the Schur complement of K_gamma (Eq. (10)), one K_gamma solve per iteration;
    // an instance whose CG needs more than B_CG_ROUNDS iterations goes on in the next sweep
    k_b_cgi_rhs<<<g2, blk, 0, s>>>(bi, ctl);
    L(1);
    CKR(rec(2));
    CKR(split(k_b_solve_inst<double>, B_NT, B->solve_smem, (int)PH_CGI, B->solve_ycap));
    CKR(rec(3));
    k_b_cgi_start<<<g2, blk, 0, s>>>(bi, ctl);
    k_b_ctl_cgi<<<gc, 128, 0, s>>>(bi, ctl, C, B->opt.cg_rtol);
    L(2);
    for (int r = 0; r < B_CG_ROUNDS; ++r) {
      k_b_cg_u<<<g2, blk, 0, s>>>(bi, ctl);
      L(1);
      CKR(split(k_b_solve_inst<double>, B_NT, B->solve_smem, (int)PH_CG, B->solve_ycap));
      k_b_cg_sp<<<g2, blk, 0, s>>>(bi, ctl);
      k_b_ctl_cg_alpha<<<gc, 128, 0, s>>>(bi, ctl, C);
      k_b_cg_xr<<<g2, blk, 0, s>>>(bi, ctl);
      k_b_ctl_cg_beta<<<gc, 128, 0, s>>>(bi, ctl, C);
      k_b_cg_p<<<g2, blk, 0, s>>>(bi, ctl);
      L(5);
    }
    k_b_cgx_rhs<<<g2, blk, 0, s>>>(bi, ctl);
    L(1);
    CKR(split(k_b_solve_inst<double>, B_NT, B->solve_smem, (int)PH_CGX, B->solve_ycap));
    k_b_cgx_dz<<<g2, blk, 0, s>>>(bi, ctl);
    k_b_ctl_cgx<<<gc, 128, 0, s>>>(ctl, C, B->d_tickets + 12);
    L(2);
  }
  if (B->opt.kkt != 1 || resto_on) {
    // condensed solve, then Richardson refinement on the augmented system (HyKKT: the
    // restoration problem's steps, whose rows are all condensed)
    CKR(solve(PH_SOLVE));
    k_b_ctl_solved<<<gc, 128, 0, s>>>(bi, ctl, C);
    L(1);
    for (int r = 0; r < B_REFINE_ROUNDS; ++r) {
      k_b_scal_zero<<<C, 32, 0, s>>>(bi, ctl, (int)PH_REFINE);
      k_b_resid<<<g2, blk, 0, s>>>(bi, ctl, (int)PH_REFINE);
      k_b_ctl_ref<<<gc, 128, 0, s>>>(bi, ctl, C, B->opt.max_refine, B->d_tickets + 12,
                                     (int)(B->opt.kkt == 0));
      L(3);
      CKR(solve(PH_REFINE));
      k_b_axpy<<<g2, blk, 0, s>>>(bi, ctl);
      L(1);
    }
    if (B->opt.kkt == 0) {
      // LiftedKKT: conjugate gradients after a refinement that stagnated above 1e-10
      auto psolve = [&](int phase) -> int {
        if (B->opt.precision == 32)
          CKR(split(k_b_solve_inst<float>, B_NT, B->solve_smem, phase, B->solve_ycap));
        CKR(split(k_b_solve_inst<double>, B_NT, B->solve_smem, phase, B->solve_ycap));
        return IPM_OK;
      };
      k_b_pg_save<<<g2, blk, 0, s>>>(bi, ctl);
      k_b_pg_ju<<<g2, blk, 0, s>>>(bi, ctl, (int)PH_PCGI);
      k_b_pg_k<<<g2, blk, 0, s>>>(bi, ctl, (int)PH_PCGI);
      L(3);
      CKR(psolve(PH_PCGI));
      k_b_pg_rz<<<g2, blk, 0, s>>>(bi, ctl, (int)PH_PCGI);
      k_b_ctl_pgi<<<gc, 128, 0, s>>>(bi, ctl, C);
      L(2);
      for (int r = 0; r < B_PCG_ROUNDS; ++r) {
        k_b_pg_ju<<<g2, blk, 0, s>>>(bi, ctl, (int)PH_PCG);
        k_b_pg_k<<<g2, blk, 0, s>>>(bi, ctl, (int)PH_PCG);
        k_b_ctl_pg_alpha<<<gc, 128, 0, s>>>(bi, ctl, C);
        k_b_pg_xr<<<g2, blk, 0, s>>>(bi, ctl);
        k_b_ctl_pg_check<<<gc, 128, 0, s>>>(bi, ctl, C);
        L(5);
        CKR(psolve(PH_PCG));
        k_b_pg_rz<<<g2, blk, 0, s>>>(bi, ctl, (int)PH_PCG);
        k_b_pg_p<<<g2, blk, 0, s>>>(bi, ctl);
        L(2);
      }
      k_b_pg_dz<<<g2, blk, 0, s>>>(bi, ctl);
      k_b_scal_zero<<<C, 32, 0, s>>>(bi, ctl, (int)PH_PCGX);
      k_b_resid<<<g2, blk, 0, s>>>(bi, ctl, (int)PH_PCGX);
      k_b_ctl_pgx<<<gc, 128, 0, s>>>(bi, ctl, C, B->d_tickets + 12);
      k_b_pg_restore<<<g2, blk, 0, s>>>(bi, ctl);
      L(5);
    }
  }
  // step recovery, fraction to the boundary, line-search set-up
  k_b_jv<<<g2, blk, 0, s>>>(bi, ctl);
  k_b_recover<<<g2, blk, 0, s>>>(bi, ctl);
  L(2);
  rreset(PH_STEP, R_AMAX, R_AZ + 1, 1.0);
  rreset(PH_STEP, R_GPHI_X, R_GPHI_S + 1, 0.0);
  k_b_ftb<<<g2, blk, 0, s>>>(bi, ctl);
  k_b_ctl_ls0<<<gc, 128, 0, s>>>(bi, ctl, C);
  L(2);
  // line-search trials
  for (int r = 0; r < B->ls_rounds; ++r) {
    k_b_trial<<<g2, blk, 0, s>>>(bi, ctl);
    L(1);
    eval(PH_LS, 2);
    k_b_scale_model<<<g2, blk, 0, s>>>(bi, ctl, PH_LS, 2, relax);
    L(1);
    rreset(PH_LS, R_TH_G, R_LOG_XU + 1, 0.0);
    if (resto_on) rreset(PH_LS, R_RS_OBJ, R_COUNT, 0.0);
    k_b_merit_trial<<<g2, blk, 0, s>>>(bi, ctl);
    k_b_ctl_ls<<<gc, 128, 0, s>>>(bi, ctl, C, (int)resto_on, tol);
    L(2);
  }
  k_b_accept<<<g2, blk, 0, s>>>(bi, ctl);
  k_b_ctl_acc<<<gc, 128, 0, s>>>(bi, ctl, C, B->fmax_entries);
  L(2);
  CK(cudaMemsetAsync(B->d_tickets + 8, 0, sizeof(int), s));
  k_b_count<<<gc, 128, 0, s>>>(ctl, C, B->d_tickets + 8);
  L(1);
  CK(cudaMemcpyAsync(B->h_active, B->d_tickets + 8, sizeof(int), cudaMemcpyDeviceToHost, s));
  CKL();
  B->launches_per_sweep = n;
  return IPM_OK;
}

// Instances whose supernode count exceeds big_num / big_den times the median are "big": their
// factorization and solves run on a cluster of cl_big blocks in a second branch of the sweep,
// concurrently with the one-block instances, so that they do not set the length of every sweep.
// Writes the launch order (one-block instances by decreasing supernode count, then the big ones).
int set_order(ipm_batch_t B) {
  const int count = B->count;
  std::vector<int> order(count);
  for (int i = 0; i < count; ++i) order[i] = i;
  std::stable_sort(order.begin(), order.end(), [&](int a, int b2) {
    return B->syms[B->pat[a]]->nsuper > B->syms[B->pat[b2]]->nsuper;
  });
  const int64_t med = B->syms[B->pat[order[count / 2]]]->nsuper;
  int nbig = 0;
  if (B->big_den > 0 && B->cl_big > 1)
    while (nbig < count &&
           (int64_t)B->syms[B->pat[order[nbig]]]->nsuper * B->big_den > B->big_num * med)
      ++nbig;
  std::vector<int> ord2(order.begin() + nbig, order.end());
  ord2.insert(ord2.end(), order.begin(), order.begin() + nbig);
  B->n_big = nbig;
  B->n_small = count - nbig;
  CK(cudaMemcpy(B->d_order, ord2.data(), sizeof(int) * count, cudaMemcpyHostToDevice));
  CK(cudaMemcpy(B->d_order_all, order.data(), sizeof(int) * count, cudaMemcpyHostToDevice));
  return IPM_OK;
}

void drop_graph(ipm_batch_t B) {
  if (B->exec) {
    cudaGraphExecDestroy(B->exec);
    cudaGraphDestroy(B->graph);
    B->exec = nullptr;
    B->graph = nullptr;
  }
  if (B->exec_tail) {
    cudaGraphExecDestroy(B->exec_tail);
    cudaGraphDestroy(B->graph_tail);
    B->exec_tail = nullptr;
    B->graph_tail = nullptr;
  }
}

int enqueue_sweep(ipm_batch_t B, cudaStream_t s);

// captures one sweep into *graph / *exec; tail = true: the tail's rounds (and, with tail_cl > 0,
// every instance on clusters of tail_cl blocks)
int capture_sweep(ipm_batch_t B, bool tail, cudaGraph_t *graph, cudaGraphExec_t *exec) {
  const int n_small = B->n_small, n_big = B->n_big, cl_big = B->cl_big;
  int *order = B->d_order;
  if (tail && B->tail_cl > 0) {
    B->n_small = 0;
    B->n_big = B->count;
    B->cl_big = B->tail_cl;
    B->d_order = B->d_order_all;
  }
  if (tail) {
    B->fact_rounds = B_TAIL_FACT_ROUNDS;
    B->ls_rounds = B_TAIL_LS_ROUNDS;
  }
  // sweeps are captured on a private stream: legacy default streams cannot be captured
  cudaStream_t cs;
  int rc = IPM_OK;
  if (cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) != cudaSuccess) rc = IPM_ERR_CUDA;
  if (rc == IPM_OK) {
    if (cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal) != cudaSuccess) rc = IPM_ERR_CUDA;
    const int launches = B->launches_per_sweep;
    if (rc == IPM_OK) rc = enqueue_sweep(B, cs);
    if (tail) B->launches_per_sweep = launches;  // the count of the main graph is reported
    cudaGraph_t g = nullptr;
    if (cudaStreamEndCapture(cs, &g) != cudaSuccess && rc == IPM_OK) rc = IPM_ERR_CUDA;
    cudaStreamDestroy(cs);
    if (rc == IPM_OK && cudaGraphInstantiate(exec, g, 0) != cudaSuccess) rc = IPM_ERR_CUDA;
    if (rc != IPM_OK) {
      if (g) cudaGraphDestroy(g);
      set_error_msg("ipm_batch_run: capturing the sweep failed");
    } else {
      *graph = g;
    }
  }
  B->n_small = n_small;
  B->n_big = n_big;
  B->cl_big = cl_big;
  B->d_order = order;
  B->fact_rounds = B_FACT_ROUNDS;
  B->ls_rounds = B_LS_ROUNDS;
  return rc;
}

// The host-side set-up of this file (shapes, orders, pause point) copies into device memory
// with the synchronous copy calls, which run on the legacy default stream and may return before
// the data lands: work on the batch's stream waits for them first.
int after_host_copies(ipm_batch_t B) {
  if (B->stream != cudaStreamLegacy && B->stream != nullptr)
    CK(cudaStreamSynchronize(cudaStreamLegacy));
  return IPM_OK;
}

// starting point, scaling and multipliers of every instance (Ipopt: see ipm_state_create)
int init_instances(ipm_batch_t B) {
  const int C = B->count;
  cudaStream_t s = B->stream;
  const dim3 g2(B->gx, C), blk(B_BLOCK);
  BI *bi = B->d_bi;
  BCtl *ctl = B->d_ctl;
  const double mu0 = B->opt.mu0;
  k_b_ctl_init<<<grid_for(C, 128), 128, 0, s>>>(bi, ctl, C, mu0, B->opt.kkt == 1,
                                                B->opt.cg_maxit, B->opt.precision == 32);
  k_b_setup_sums<<<g2, blk, 0, s>>>(bi, ctl);
  k_b_x0<<<g2, blk, 0, s>>>(bi, ctl);
  k_b_flow_start<<<g2, blk, 0, s>>>(bi, ctl);
  auto eval0 = [&]() {
    k_b_eval_init<<<g2, blk, 0, s>>>(bi, ctl, PH_EVAL, 0);
    k_b_eval_branch<<<g2, blk, 0, s>>>(bi, ctl, PH_EVAL, 0);
    k_b_eval_gen<<<dim3(B->gx_gen, C), blk, 0, s>>>(bi, ctl, PH_EVAL, 0);
    k_b_eval_finish<<<g2, blk, 0, s>>>(bi, ctl, PH_EVAL, 0, B->gx_gen);
  };
  eval0();
  k_b_row_scale<<<g2, blk, 0, s>>>(bi, ctl);
  k_b_ctl_sig<<<grid_for(C, 128), 128, 0, s>>>(bi, ctl, C);
  eval0();
  k_b_scale_model<<<g2, blk, 0, s>>>(bi, ctl, PH_EVAL, 0, B->opt.tau);
  k_b_init_duals<<<g2, blk, 0, s>>>(bi, ctl);
  CKL();
  count_launches(16);
  return IPM_OK;
}

}  // namespace

extern "C" int ipm_batch_create(int count, const ipm_opf_t *opfs, const ipm_options *opt,
                                cudaStream_t stream, ipm_batch_t *out) {
  NvtxRange nvtx_range("ipm_batch_create");
  if (count <= 0 || !opfs || !opt || !out || opt->kkt < 0 || opt->kkt > 2 ||
      !(opt->tol > 0) || (opt->kkt != 0 && !(opt->gamma > 0))) {
    set_error_msg("ipm_batch_create: bad argument (count > 0, kkt = 0 (LiftedKKT), 1 (HyKKT, "
                  "gamma > 0) or 2 (dual-regularized, gamma > 0), tol > 0)");
    return IPM_ERR_BAD_ARG;
  }
  if (opt->precision != 0 && opt->precision != 64 && opt->precision != 32) {
    set_error_msg("ipm_batch_create: precision 0 or 64 (FP64 factor) or 32 (FP32 factor with "
                  "FP64 refinement)");
    return IPM_ERR_BAD_ARG;
  }
  if (opt->precision == 32 && opt->kkt == 1) {
    set_error_msg("ipm_batch_create: the FP32 factor serves the refined condensed solve (kkt 0 "
                  "or 2); HyKKT's Schur-complement CG needs exact K_gamma solves");
    return IPM_ERR_BAD_ARG;
  }
  for (int i = 0; i < count; ++i)
    if (!opfs[i]) {
      set_error_msg("ipm_batch_create: null model handle");
      return IPM_ERR_BAD_ARG;
    }
  *out = nullptr;
  CKR(b_smem_limits());
  // creation runs on the set-up stream; the sweeps on the caller's
  const cudaStream_t caller = stream;
  stream = setup_stream(stream);
  ipm_batch_t B = new ipm_batch_s();
  auto fail = [&](int rc) {
    ipm_batch_destroy(B);
    return rc;
  };
  B->count = count;
  B->opt = *opt;
  if (!(B->opt.tau > 0)) B->opt.tau = B->opt.tol;
  if (!(B->opt.mu0 > 0)) B->opt.mu0 = 0.1;
  if (B->opt.max_refine < 0) B->opt.max_refine = 10;
  if (!(B->opt.cg_rtol > 0)) B->opt.cg_rtol = 1e-10;
  B->stream = stream;
  B->opf.assign(opfs, opfs + count);
  // ---- one symbolic analysis per distinct pattern
  {
    std::map<std::vector<int>, int> seen;
    std::vector<int> key;
    B->pat.resize(count);
    for (int i = 0; i < count; ++i) {
      int rc = pattern_of(opfs[i]->M, key);
      if (rc != IPM_OK) return fail(rc);
      auto it = seen.find(key);
      if (it != seen.end()) {
        B->pat[i] = it->second;
        continue;
      }
      const OpfData &M = opfs[i]->M;
      ipm_sym_t S = nullptr;
      const bool dflt = B->opt.sn_relax_w <= 0;
      rc = ipm_symbolic_relaxed(M.n, M.me + M.mi, M.J_rowptr, M.J_colind, M.nnzJ, M.W_rowptr,
                                M.W_colind, M.nnzW, dflt ? 8 : B->opt.sn_relax_w,
                                dflt ? 5 : B->opt.sn_relax_den, stream, &S);
      if (rc != IPM_OK) return fail(rc);
      B->pat[i] = (int)B->syms.size();
      B->syms.push_back(S);
      seen.emplace(key, B->pat[i]);
    }
  }
  // ---- sizes and pool layout
  struct Off {
    size_t x, s, y, z, v, zl, zu, grad, jtl, geq, hin, dscale, gs, hs, Jv, Wv, lam, lamw, f, fpart;
    size_t sigma, r1, r2, r4, Ds, dcond, baug, a, dx, dzc, jdx, dz, ds, dv, dzl, dzu;
    size_t xt, st, geqt, hint, gst, hst, ft, R, filter, tJ, Lx, Dx, y_s, t, cx, cz, outx, outz,
        scal;
    size_t cg_r, cg_p, cg_sp, cg_dy, cg_rhs1, cg_v;
    size_t pg_t, pg_r, pg_z, pg_p, pg_q, pg_u, pg_xs, pg_zs;
    size_t rp, rq, rzp, rzq, rdp, rdq, rdzp, rdzq, rpt, rqt, rrc, rrp, rrq, rxr, rdr2, rfilter;
    size_t info;
  };
  std::vector<Off> off(count);
  Bump dp, ip;
  int max_elems = 1, max_ng = 1;
  B->fmax_entries = 512;
  for (int i = 0; i < count; ++i) max_ng = std::max(max_ng, opfs[i]->M.ng);
  B->gx_gen = grid_for(max_ng, B_BLOCK);
  for (int i = 0; i < count; ++i) {
    const OpfData &M = opfs[i]->M;
    ipm_sym_t S = B->syms[B->pat[i]];
    const bool lifted = B->opt.kkt == 0;
    const size_t n = M.n, me0 = M.me, mi0 = M.mi, m = me0 + mi0;
    const size_t mi = lifted ? 2 * me0 + mi0 : mi0, me = lifted ? 0 : me0;
    Off &o = off[i];
    o.x = dp.take(n); o.s = dp.take(mi); o.y = dp.take(me); o.z = dp.take(mi); o.v = dp.take(mi);
    o.zl = dp.take(n); o.zu = dp.take(n); o.grad = dp.take(n); o.jtl = dp.take(n);
    o.geq = dp.take(me); o.hin = dp.take(mi); o.dscale = dp.take(m); o.gs = dp.take(me0);
    o.hs = dp.take(mi0); o.Jv = dp.take(M.nnzJ); o.Wv = dp.take(M.nnzW); o.lam = dp.take(m);
    o.lamw = dp.take(m); o.f = dp.take(2); o.fpart = dp.take(B->gx_gen);
    o.sigma = dp.take(n); o.r1 = dp.take(n); o.r2 = dp.take(mi); o.r4 = dp.take(mi);
    o.Ds = dp.take(mi); o.dcond = dp.take(m); o.baug = dp.take(m); o.a = dp.take(n);
    o.dx = dp.take(n); o.dzc = dp.take(m); o.jdx = dp.take(m); o.dz = dp.take(mi);
    o.ds = dp.take(mi); o.dv = dp.take(mi); o.dzl = dp.take(n); o.dzu = dp.take(n);
    o.xt = dp.take(n); o.st = dp.take(mi); o.geqt = dp.take(me); o.hint = dp.take(mi);
    o.gst = dp.take(me0); o.hst = dp.take(mi0); o.ft = dp.take(2); o.R = dp.take(R_COUNT);
    o.filter = dp.take(2 * (size_t)B->fmax_entries); o.tJ = dp.take(M.nnzJ);
    o.Lx = dp.take(S->panel_len); o.Dx = dp.take(S->diag_len); o.y_s = dp.take(n);
    o.t = dp.take(n); o.cx = dp.take(n); o.cz = dp.take(m); o.outx = dp.take(n);
    o.outz = dp.take(m); o.scal = dp.take(8);
    const size_t ncg = B->opt.kkt == 1 ? n : 0, mcg = B->opt.kkt == 1 ? me0 : 0;
    o.cg_r = dp.take(mcg); o.cg_p = dp.take(mcg); o.cg_sp = dp.take(mcg); o.cg_dy = dp.take(mcg);
    o.cg_rhs1 = dp.take(ncg); o.cg_v = dp.take(ncg);
    const size_t npg = lifted ? n : 0, mpg = lifted ? m : 0;  // PCG after stagnation
    o.pg_t = dp.take(npg); o.pg_r = dp.take(npg); o.pg_z = dp.take(npg); o.pg_p = dp.take(npg);
    o.pg_q = dp.take(npg); o.pg_u = dp.take(mpg); o.pg_xs = dp.take(npg); o.pg_zs = dp.take(mpg);
    // restoration phase: per IPM row, x_R and D_R^2, the phase's filter
    const size_t nr = B->opt.no_resto ? 0 : me + mi, nx = B->opt.no_resto ? 0 : n;
    o.rp = dp.take(nr); o.rq = dp.take(nr); o.rzp = dp.take(nr); o.rzq = dp.take(nr);
    o.rdp = dp.take(nr); o.rdq = dp.take(nr); o.rdzp = dp.take(nr); o.rdzq = dp.take(nr);
    o.rpt = dp.take(nr); o.rqt = dp.take(nr); o.rrc = dp.take(nr); o.rrp = dp.take(nr);
    o.rrq = dp.take(nr); o.rxr = dp.take(nx); o.rdr2 = dp.take(nx);
    o.rfilter = dp.take(B->opt.no_resto ? 0 : 2 * (size_t)B->fmax_entries);
    o.info = ip.take(1);
    max_elems = std::max({max_elems, M.n, (int)mi, (int)m, M.nnzJ, M.nnzW, 2 * M.nbr});
    B->max_ns = std::max(B->max_ns, S->nsuper);
  }
  {
    int64_t max_slots = 1;
    for (int i = 0; i < count; ++i) {
      ipm_sym_t S = B->syms[B->pat[i]];
      max_slots = std::max<int64_t>(max_slots, S->panel_len);
    }
    B->gx_cond = std::max(1, std::min(64, (int)((max_slots + B_BLOCK * 4 - 1) / (B_BLOCK * 4))));
  }
  B->dpool_len = dp.n;
  B->ipool_len = ip.n;
  // up to 32 elements per thread and at most 16 blocks per instance: phase-masked launches stay
  // cheap (a masked block only checks its instance's phase) while each instance keeps 4,096 threads
  B->gx = std::max(1, std::min(grid_for(max_elems, B_BLOCK * 32), 16));
  if (cudaMalloc(&B->dpool, sizeof(double) * B->dpool_len) != cudaSuccess ||
      cudaMalloc(&B->ipool, sizeof(int) * B->ipool_len) != cudaSuccess) {
    set_error_msg("ipm_batch_create: out of device memory for the instance pool");
    return fail(IPM_ERR_OOM);
  }
  if (cudaMemset(B->dpool, poison_allocations() ? 0xFF : 0, sizeof(double) * B->dpool_len) !=
          cudaSuccess ||
      cudaMemset(B->ipool, 0, sizeof(int) * B->ipool_len) != cudaSuccess)
    return fail(IPM_ERR_CUDA);
  // ---- descriptors, task-argument blocks and ticket ranges
  std::vector<BI> hbi(count);
  // wide supernodes of one level must fit the per-block list of the factorization kernel
  for (ipm_sym_t S : B->syms) {
    std::vector<int> sp(S->nsuper + 1), ls(S->nsuper);
    if (cudaMemcpy(sp.data(), S->sptr, sizeof(int) * (S->nsuper + 1), cudaMemcpyDeviceToHost) != cudaSuccess ||
        cudaMemcpy(ls.data(), S->level_sn, sizeof(int) * S->nsuper, cudaMemcpyDeviceToHost) != cudaSuccess)
      return fail(IPM_ERR_CUDA);
    for (int L = 0; L < S->nlevels; ++L) {
      int wide = 0;
      for (int q = S->h_level_ptr[L]; q < S->h_level_ptr[L + 1]; ++q)
        wide += sp[ls[q] + 1] - sp[ls[q]] > B_WS;
      if (wide > B_WIDE_CAP) {
        set_error_msg("ipm_batch_create: a level holds more wide supernodes than the batched "
                      "factorization takes (" + std::to_string(B_WIDE_CAP) + ")");
        return fail(IPM_ERR_BAD_ARG);
      }
    }
  }
  // update pairs of every pattern: for each supernode, the pairs (i, j) of its rows below the
  // diagonal block and the slot of the target panel that entry (i, j) of L21 L21^T updates
  std::vector<int *> pptr(B->syms.size()), pa(B->syms.size()), pb(B->syms.size()),
      pm(B->syms.size()), ptgt(B->syms.size()), g8p(B->syms.size()), g8s(B->syms.size());
  std::vector<int *> cslot(B->syms.size()), ccol(B->syms.size()), cgp(B->syms.size());
  std::vector<int2 *> citm(B->syms.size());
  std::vector<ushort2 *> citm16(B->syms.size(), nullptr);
  std::vector<int> ncslot(B->syms.size());
  for (size_t q = 0; q < B->syms.size(); ++q) {
    ipm_sym_t S = B->syms[q];
    const int ns = S->nsuper;
    std::vector<int> sp(ns + 1), rp(ns + 1), sn(S->n);
    std::vector<int64_t> lp(ns + 1);
    if (cudaMemcpy(sp.data(), S->sptr, sizeof(int) * (ns + 1), cudaMemcpyDeviceToHost) != cudaSuccess ||
        cudaMemcpy(rp.data(), S->srow_ptr, sizeof(int) * (ns + 1), cudaMemcpyDeviceToHost) != cudaSuccess ||
        cudaMemcpy(sn.data(), S->snode, sizeof(int) * S->n, cudaMemcpyDeviceToHost) != cudaSuccess ||
        cudaMemcpy(lp.data(), S->lptr, sizeof(int64_t) * (ns + 1), cudaMemcpyDeviceToHost) != cudaSuccess)
      return fail(IPM_ERR_CUDA);
    std::vector<int> rows(rp[ns]);
    if (rp[ns] && cudaMemcpy(rows.data(), S->srow, sizeof(int) * rp[ns], cudaMemcpyDeviceToHost) != cudaSuccess)
      return fail(IPM_ERR_CUDA);
    if (S->panel_len >= INT_MAX) return fail(IPM_ERR_BAD_ARG);
    std::vector<int> lsn(ns);
    if (ns && cudaMemcpy(lsn.data(), S->level_sn, sizeof(int) * ns, cudaMemcpyDeviceToHost) != cudaSuccess)
      return fail(IPM_ERR_CUDA);
    std::vector<int> hp(S->nlevels + 1, 0), ha, hb, hm, htg, hg8p(S->nlevels + 1, 0), hg8s;
    for (int L = 0; L < S->nlevels; ++L) {
      for (int qq = S->h_level_ptr[L]; qq < S->h_level_ptr[L + 1]; ++qq) {
        const int sn_ = lsn[qq];
        const int w = sp[sn_ + 1] - sp[sn_], rb = rp[sn_], ld = rp[sn_ + 1] - rb;
        if (ld >= (1 << 23) || w > 255) return fail(IPM_ERR_BAD_ARG);
        if (w > B_WT && w <= B_WG) hg8s.push_back(sn_);
        for (int j = w; j < ld; ++j) {
          const int col = rows[rb + j], ts = sn[col];
          const int tb = rp[ts], tld = rp[ts + 1] - tb;
          const int *tr = rows.data() + tb;
          for (int i = j; i < ld; ++i) {
            const int r = (int)(std::lower_bound(tr, tr + tld, rows[rb + i]) - tr);
            ha.push_back((int)(lp[sn_] + i));
            hb.push_back((int)(lp[sn_] + j));
            hm.push_back(ld << 8 | w);
            htg.push_back((int)(lp[ts] + (int64_t)(col - sp[ts]) * tld + r));
          }
        }
      }
      hp[L + 1] = (int)ha.size();
      hg8p[L + 1] = (int)hg8s.size();
    }
    auto upi = [&](int **dst, const std::vector<int> &v) -> int {
      if (cudaMalloc((void **)dst, sizeof(int) * std::max<size_t>(v.size(), 1)) != cudaSuccess)
        return IPM_ERR_OOM;
      B->bufs.push_back(*dst);
      if (!v.empty() && cudaMemcpy(*dst, v.data(), sizeof(int) * v.size(), cudaMemcpyHostToDevice) != cudaSuccess)
        return IPM_ERR_CUDA;
      return IPM_OK;
    };
    // condensation order: lower slots by descending item count (then by slot)
    std::vector<int> sptr_items(S->panel_len + 1);
    std::vector<int2> items(std::max<int64_t>(S->nitems, 1));
    if (cudaMemcpy(sptr_items.data(), S->slot_ptr, sizeof(int) * (S->panel_len + 1),
                   cudaMemcpyDeviceToHost) != cudaSuccess ||
        (S->nitems && cudaMemcpy(items.data(), S->items, sizeof(int2) * S->nitems,
                                 cudaMemcpyDeviceToHost) != cudaSuccess))
      return fail(IPM_ERR_CUDA);
    std::vector<int> hperm(S->n);
    if (cudaMemcpy(hperm.data(), S->perm, sizeof(int) * S->n, cudaMemcpyDeviceToHost) != cudaSuccess)
      return fail(IPM_ERR_CUDA);
    std::vector<std::pair<int, int>> order;  // (-count, slot)
    std::vector<int> diagcol(S->panel_len, -1);
    for (int sn_ = 0; sn_ < ns; ++sn_) {
      const int w = sp[sn_ + 1] - sp[sn_], ld = rp[sn_ + 1] - rp[sn_];
      for (int c = 0; c < w; ++c)
        for (int r = c; r < ld; ++r) {
          const int slot = (int)(lp[sn_] + (int64_t)c * ld + r);
          order.push_back({-(sptr_items[slot + 1] - sptr_items[slot]), slot});
          if (r == c) diagcol[slot] = hperm[sp[sn_] + c];
        }
    }
    std::sort(order.begin(), order.end());
    std::vector<int> hcs(order.size()), hcc(order.size());
    for (size_t t = 0; t < order.size(); ++t) {
      hcs[t] = order[t].second;
      hcc[t] = diagcol[order[t].second];
    }
    ncslot[q] = (int)order.size();
    const size_t ngrp = (order.size() + 31) / 32;
    std::vector<int> hgp(ngrp + 1, 0);
    std::vector<int2> hci;
    for (size_t g = 0; g < ngrp; ++g) {
      const int cnt = -order[g * 32].first;  // the largest count of the group (sorted)
      if ((int64_t)hci.size() + 32 * (int64_t)cnt >= INT_MAX) return fail(IPM_ERR_BAD_ARG);
      for (int k = 0; k < cnt; ++k)
        for (int l = 0; l < 32; ++l) {
          const size_t t = g * 32 + l;
          int2 v = make_int2(0, -2);
          if (t < order.size()) {
            const int slot = order[t].second;
            if (k < sptr_items[slot + 1] - sptr_items[slot]) v = items[sptr_items[slot] + k];
          }
          hci.push_back(v);
        }
      hgp[g + 1] = (int)hci.size();
    }
    int r1 = upi(&pptr[q], hp);
    if (r1 == IPM_OK) r1 = upi(&pa[q], ha);
    if (r1 == IPM_OK) r1 = upi(&pb[q], hb);
    if (r1 == IPM_OK) r1 = upi(&pm[q], hm);
    if (r1 == IPM_OK) r1 = upi(&ptgt[q], htg);
    if (r1 == IPM_OK) r1 = upi(&g8p[q], hg8p);
    if (r1 == IPM_OK) r1 = upi(&g8s[q], hg8s);
    if (r1 == IPM_OK) r1 = upi(&cslot[q], hcs);
    if (r1 == IPM_OK) r1 = upi(&ccol[q], hcc);
    if (r1 == IPM_OK) r1 = upi(&cgp[q], hgp);
    if (r1 != IPM_OK) return fail(r1);
    // 16-bit items (x, y + 2) when every J and W entry index of the pattern fits
    int max_x = 0, max_y = 0;
    for (const int2 &v : hci) {
      max_x = std::max(max_x, v.x);
      max_y = std::max(max_y, v.y);
    }
    if (max_x <= 0xFFFF && max_y + 2 <= 0xFFFF) {
      std::vector<ushort2> h16(hci.size());
      for (size_t t = 0; t < hci.size(); ++t)
        h16[t] = make_ushort2((unsigned short)hci[t].x, (unsigned short)(hci[t].y + 2));
      if (cudaMalloc((void **)&citm16[q], sizeof(ushort2) * std::max<size_t>(h16.size(), 1)) !=
          cudaSuccess)
        return fail(IPM_ERR_OOM);
      B->bufs.push_back(citm16[q]);
      if (!h16.empty() && cudaMemcpy(citm16[q], h16.data(), sizeof(ushort2) * h16.size(),
                                     cudaMemcpyHostToDevice) != cudaSuccess)
        return fail(IPM_ERR_CUDA);
    } else {
      if (cudaMalloc((void **)&citm[q], sizeof(int2) * std::max<size_t>(hci.size(), 1)) !=
          cudaSuccess)
        return fail(IPM_ERR_OOM);
      B->bufs.push_back(citm[q]);
      if (!hci.empty() && cudaMemcpy(citm[q], hci.data(), sizeof(int2) * hci.size(),
                                     cudaMemcpyHostToDevice) != cudaSuccess)
        return fail(IPM_ERR_CUDA);
    }
  }
  // level offsets of each pattern's supernode schedule, on the device
  std::vector<int *> lvl(B->syms.size(), nullptr);
  for (size_t q = 0; q < B->syms.size(); ++q) {
    const std::vector<int> &h = B->syms[q]->h_level_ptr;
    if (cudaMalloc((void **)&lvl[q], sizeof(int) * h.size()) != cudaSuccess) return fail(IPM_ERR_OOM);
    B->bufs.push_back(lvl[q]);
    if (cudaMemcpy(lvl[q], h.data(), sizeof(int) * h.size(), cudaMemcpyHostToDevice) != cudaSuccess)
      return fail(IPM_ERR_CUDA);
  }
  for (int i = 0; i < count; ++i) {
    const OpfData &M = opfs[i]->M;
    ipm_sym_t S = B->syms[B->pat[i]];
    const Off &o = off[i];
    double *d = B->dpool;
    BI &I = hbi[i];
    memset(&I, 0, sizeof(I));
    // LiftedKKT: equalities relaxed into slack rows; HyKKT and form 2 (delta_c = 1/gamma): equalities
    // kept (y)
    I.D = B->opt.kkt == 0 ? Dims{M.n, M.me, M.mi, 0, 2 * M.me + M.mi, 1}
                          : Dims{M.n, M.me, M.mi, M.me, M.mi, 0};
    I.P.x = d + o.x; I.P.s = d + o.s; I.P.y = d + o.y; I.P.z = d + o.z; I.P.v = d + o.v;
    I.P.zl = d + o.zl; I.P.zu = d + o.zu; I.P.xl = M.xl; I.P.xu = M.xu;
    I.P.grad = d + o.grad; I.P.jtl = d + o.jtl; I.P.geq = d + o.geq; I.P.hin = d + o.hin;
    I.SA.D = I.D;
    I.SA.P = I.P;
    I.SA.r2 = d + o.r2; I.SA.r4 = d + o.r4; I.SA.Ds = d + o.Ds; I.SA.jdx = d + o.jdx;
    I.SA.dx = d + o.dx; I.SA.sigma = d + o.sigma;
    I.SA.dzH = B->opt.kkt == 0 ? nullptr : d + o.dzc + M.me;  // dz over the H rows
    I.SA.dz = d + o.dz; I.SA.ds = d + o.ds; I.SA.dv = d + o.dv; I.SA.dzl = d + o.dzl;
    I.SA.dzu = d + o.dzu;
    I.M = M;
    I.m = M.me + M.mi;
    I.dscale = d + o.dscale; I.gs = d + o.gs; I.hs = d + o.hs; I.Jv = d + o.Jv; I.Wv = d + o.Wv;
    I.lam = d + o.lam; I.lamw = d + o.lamw; I.f = d + o.f; I.fpart = d + o.fpart;
    I.r1 = d + o.r1; I.dcond = d + o.dcond; I.baug = d + o.baug; I.a = d + o.a; I.dx = d + o.dx;
    I.dzc = d + o.dzc; I.xt = d + o.xt; I.st = d + o.st; I.geqt = d + o.geqt; I.hint = d + o.hint;
    I.gst = d + o.gst; I.hst = d + o.hst; I.ft = d + o.ft; I.R = d + o.R; I.filter = d + o.filter;
    I.sptr = S->sptr; I.srow_ptr = S->srow_ptr; I.slot_ptr = S->slot_ptr; I.perm = S->perm;
    I.J_rowidx = S->J_rowidx; I.JT_ptr = S->JT_ptr; I.JT_ent = S->JT_ent; I.lptr = S->lptr;
    I.items = S->items; I.ns = S->nsuper;
    I.tJ = d + o.tJ; I.Lx = d + o.Lx; I.Dx = d + o.Dx;
    I.info = B->ipool + o.info;
    I.srow = S->srow; I.snode = S->snode; I.level_sn = S->level_sn; I.dptr = S->dptr;
    I.nlevels = S->nlevels;
    I.lvl_ptr = lvl[B->pat[i]];
    I.lpair_ptr = pptr[B->pat[i]];
    I.pair_a = pa[B->pat[i]];
    I.pair_b = pb[B->pat[i]];
    I.pair_m = pm[B->pat[i]];
    I.pair_tgt = ptgt[B->pat[i]];
    I.g8_ptr = g8p[B->pat[i]];
    I.g8_sn = g8s[B->pat[i]];
    I.cslot = cslot[B->pat[i]];
    I.ccol = ccol[B->pat[i]];
    I.cgptr = cgp[B->pat[i]];
    I.citems = citm[B->pat[i]];
    I.citems16 = citm16[B->pat[i]];
    I.ncslot = ncslot[B->pat[i]];
    I.y = d + o.y_s; I.t = d + o.t; I.cx = d + o.cx; I.cz = d + o.cz; I.outx = d + o.outx;
    I.outz = d + o.outz; I.scal = d + o.scal;
    I.cg_r = d + o.cg_r; I.cg_p = d + o.cg_p; I.cg_sp = d + o.cg_sp; I.cg_dy = d + o.cg_dy;
    I.cg_rhs1 = d + o.cg_rhs1; I.cg_v = d + o.cg_v;
    I.pg_t = d + o.pg_t; I.pg_r = d + o.pg_r; I.pg_z = d + o.pg_z; I.pg_p = d + o.pg_p;
    I.pg_q = d + o.pg_q; I.pg_u = d + o.pg_u; I.pg_xs = d + o.pg_xs; I.pg_zs = d + o.pg_zs;
    I.dystep = B->opt.kkt == 1 ? I.cg_dy : I.dzc;
    if (!B->opt.no_resto) {
      I.rp = d + o.rp; I.rq = d + o.rq; I.rzp = d + o.rzp; I.rzq = d + o.rzq; I.rdp = d + o.rdp;
      I.rdq = d + o.rdq; I.rdzp = d + o.rdzp; I.rdzq = d + o.rdzq; I.rpt = d + o.rpt;
      I.rqt = d + o.rqt; I.rrc = d + o.rrc; I.rrp = d + o.rrp; I.rrq = d + o.rrq;
      I.rxr = d + o.rxr; I.rdr2 = d + o.rdr2; I.rfilter = d + o.rfilter;
    }
    AugArgs &A = I.aug;
    A.n = M.n; A.m = I.m; A.m_e = 0;
    A.J_rowptr = S->J_rowptr; A.J_colind = S->J_colind; A.J_rowidx = S->J_rowidx;
    A.JT_ptr = S->JT_ptr; A.JT_ent = S->JT_ent;
    A.W_rowptr = S->W_rowptr; A.W_colind = S->W_colind; A.W_rowidx = S->W_rowidx;
    A.WT_ptr = S->WT_ptr; A.WT_ent = S->WT_ent;
    A.Wv = I.Wv; A.sigma = I.SA.sigma; A.Jv = I.Jv; A.d = I.dcond; A.dw = 0.0;
    A.sx = I.dx; A.sz = I.dzc; A.ra = I.a; A.rb = I.baug; A.outx = I.outx; A.outz = I.outz;
    A.scal = I.scal; A.want_norm_a = 1;
  }
  int rc = IPM_OK;
  auto up = [&](auto **dst, const auto &v) {
    using T = std::remove_reference_t<decltype(v[0])>;
    if (rc != IPM_OK) return;
    if (cudaMalloc((void **)dst, sizeof(T) * v.size()) != cudaSuccess) {
      rc = IPM_ERR_OOM;
      return;
    }
    if (cudaMemcpy(*dst, v.data(), sizeof(T) * v.size(), cudaMemcpyHostToDevice) != cudaSuccess)
      rc = IPM_ERR_CUDA;
  };
  up(&B->d_bi, hbi);
  if (rc == IPM_OK && cudaMalloc(&B->d_order, sizeof(int) * count) != cudaSuccess) rc = IPM_ERR_OOM;
  if (rc == IPM_OK && cudaMalloc(&B->d_order_all, sizeof(int) * count) != cudaSuccess)
    rc = IPM_ERR_OOM;
  if (rc == IPM_OK) rc = set_order(B);
  if (rc == IPM_OK && cudaMalloc(&B->d_ctl, sizeof(BCtl) * count) != cudaSuccess) rc = IPM_ERR_OOM;
  if (rc == IPM_OK && cudaMalloc(&B->d_tickets, sizeof(int) * 16) != cudaSuccess) rc = IPM_ERR_OOM;
  if (rc == IPM_OK && cudaMemset(B->d_tickets, 0, sizeof(int) * 16) != cudaSuccess) rc = IPM_ERR_CUDA;
  if (rc == IPM_OK) {
    const int no_pause = -1;
    if (cudaMemcpy(B->d_tickets + 12, &no_pause, sizeof(int), cudaMemcpyHostToDevice) != cudaSuccess)
      rc = IPM_ERR_CUDA;
  }
  if (rc == IPM_OK && cudaMallocHost((void **)&B->h_active, sizeof(int)) != cudaSuccess) rc = IPM_ERR_OOM;
  if (rc == IPM_OK && (cudaStreamCreateWithFlags(&B->side, cudaStreamNonBlocking) != cudaSuccess ||
                       cudaEventCreateWithFlags(&B->ev_fork, cudaEventDisableTiming) != cudaSuccess ||
                       cudaEventCreateWithFlags(&B->ev_join, cudaEventDisableTiming) != cudaSuccess))
    rc = IPM_ERR_CUDA;
  if (rc != IPM_OK) return fail(rc);
  int max_w = 1;
  for (ipm_sym_t S : B->syms) max_w = std::max(max_w, S->max_w);
  // the warps' staging of the narrow supernodes, one wide supernode of the widest pattern, or up
  // to four wide supernodes of 24 columns side by side (k_b_fact_inst)
  const size_t need24 = 24 * 24 + 32 * 25 + 24;
  B->fact_smem = sizeof(double) *
                 std::max({(size_t)max_w * max_w + (size_t)32 * (max_w + 1) + max_w,
                           (size_t)(B_NT_F / 32) * (B_WS * B_WS + B_WS), 4 * need24});
  // the solves keep the right-hand side in shared memory for instances with n <= 3,800 (with
  // the 43 KB of per-warp staging, three blocks of the solve kernel per SM still fit); larger
  // instances use global memory
  {
    int max_n = 0;
    for (int i = 0; i < count; ++i)
      if (opfs[i]->M.n <= 3800) max_n = std::max(max_n, opfs[i]->M.n);
    B->solve_ycap = max_n;
    B->solve_smem = sizeof(double) * (size_t)B->solve_ycap;
  }
  rc = init_instances(B);
  if (rc == IPM_OK && cudaStreamSynchronize(stream) != cudaSuccess) rc = IPM_ERR_CUDA;
  if (rc != IPM_OK) return fail(rc);
  B->stream = caller;
  *out = B;
  return IPM_OK;
}

extern "C" int ipm_batch_info(ipm_batch_t B, int *npatterns, int64_t *device_bytes,
                              int *launches_per_sweep) {
  if (!B) return IPM_ERR_BAD_ARG;
  if (npatterns) *npatterns = (int)B->syms.size();
  if (device_bytes)
    *device_bytes = (int64_t)(sizeof(double) * B->dpool_len + sizeof(int) * B->ipool_len);
  if (launches_per_sweep) *launches_per_sweep = B->launches_per_sweep;
  return IPM_OK;
}

extern "C" int ipm_batch_reset(ipm_batch_t B) {
  if (!B) return IPM_ERR_BAD_ARG;
  CKR(after_host_copies(B));
  CKR(init_instances(B));
  B->sweeps = 0;
  B->t_fact_ms = B->t_solve_ms = 0.0;
  B->t_n = 0;
  return IPM_OK;
}

extern "C" int ipm_batch_run(ipm_batch_t B, int max_iter, int max_sweeps, int use_graph) {
  NvtxRange nvtx_range("ipm_batch_run");
  if (!B || max_iter < 0 || max_sweeps < 1) return IPM_ERR_BAD_ARG;
  cudaStream_t s = B->stream;
  CKR(after_host_copies(B));
  if (B->max_iter != max_iter) drop_graph(B);
  B->max_iter = max_iter;
  if (use_graph && !B->exec) CKR(capture_sweep(B, false, &B->graph, &B->exec));
  // (a batch no larger than the tail threshold keeps its launch shape throughout)
  const bool has_tail = use_graph && B->tail_active > 0 && B->count > B->tail_active;
  if (has_tail && !B->exec_tail) CKR(capture_sweep(B, true, &B->graph_tail, &B->exec_tail));
  int rc = IPM_OK;
  *B->h_active = B->count;
  for (int sw = 0; sw < max_sweeps; ++sw) {
    if (use_graph) {
      const bool tail = has_tail && *B->h_active <= B->tail_active;
      CK(cudaGraphLaunch(tail ? B->exec_tail : B->exec, s));
    } else {
      CKR(enqueue_sweep(B, s));
    }
    count_launches(B->launches_per_sweep);
    ++B->sweeps;
    CK(cudaStreamSynchronize(s));
    if (B->timing) {
      float a = 0.f, a2 = 0.f, c = 0.f;
      CK(cudaEventElapsedTime(&a, B->ev[0], B->ev[1]));
      CK(cudaEventElapsedTime(&a2, B->ev[4], B->ev[5]));
      CK(cudaEventElapsedTime(&c, B->ev[2], B->ev[3]));
      B->t_fact_ms += a + a2;
      B->t_solve_ms += c;
      ++B->t_n;
    }
    if (*B->h_active == 0) break;
  }
  k_b_finish_unfinished<<<grid_for(B->count, 128), 128, 0, s>>>(B->d_ctl, B->count);
  count_launches(1);
  CKL();
  CK(cudaStreamSynchronize(s));
  return rc;
}

extern "C" int ipm_batch_autotune(ipm_batch_t B, int sweeps, int max_results, int *n_results,
                                  int *cfg, double *ms_per_sweep, int *best) {
  NvtxRange nvtx_range("ipm_batch_autotune");
  if (!B || sweeps < 1 || max_results < 0 || (max_results > 0 && (!cfg || !ms_per_sweep)))
    return IPM_ERR_BAD_ARG;
  struct Shape { int cl, num, den, gx; };
  std::vector<Shape> cand;
  const int gx0 = B->gx;
  for (int gx : {std::max(1, gx0 / 2), gx0, std::min(16, 2 * gx0)}) {
    if (!cand.empty() && cand.back().gx == gx) continue;
    cand.push_back({1, 0, 0, gx});  // no clusters
    for (int cl : {2, 4, 8})
      for (int th : {0, 1}) cand.push_back({cl, th ? 3 : 6, th ? 2 : 5, gx});  // 1.5x, 1.2x
  }
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  const bool timing = B->timing;
  B->timing = false;
  int rc = IPM_OK, ibest = -1;
  double tbest = INFINITY;
  std::vector<double> times(cand.size(), INFINITY);
  auto apply = [&](const Shape &c) -> int {
    B->cl_big = c.cl;
    B->big_num = c.num;
    B->big_den = c.den;
    B->gx = c.gx;
    drop_graph(B);
    return set_order(B);
  };
  for (size_t k = 0; k < cand.size() && rc == IPM_OK; ++k) {
    rc = apply(cand[k]);
    // first run captures the sweep graph; the second, from the starting point, is timed
    if (rc == IPM_OK) rc = ipm_batch_reset(B);
    if (rc == IPM_OK) rc = ipm_batch_run(B, B->max_iter, 1, 1);
    if (rc == IPM_OK) rc = ipm_batch_reset(B);
    if (rc != IPM_OK) break;
    if (cudaEventRecord(e0, B->stream) != cudaSuccess) { rc = IPM_ERR_CUDA; break; }
    rc = ipm_batch_run(B, B->max_iter, sweeps, 1);
    if (rc != IPM_OK) break;
    if (cudaEventRecord(e1, B->stream) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess) {
      rc = IPM_ERR_CUDA;
      break;
    }
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    const int done = std::max(1, B->sweeps);
    times[k] = ms / done;
    if (times[k] < tbest) {
      tbest = times[k];
      ibest = (int)k;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  B->timing = timing;
  if (rc == IPM_OK && ibest >= 0) rc = apply(cand[ibest]);
  if (rc == IPM_OK) rc = ipm_batch_reset(B);
  if (rc != IPM_OK) return rc;
  const int n = std::min((int)cand.size(), max_results);
  for (int k = 0; k < n; ++k) {
    cfg[4 * k] = cand[k].cl;
    cfg[4 * k + 1] = cand[k].num;
    cfg[4 * k + 2] = cand[k].den;
    cfg[4 * k + 3] = cand[k].gx;
    ms_per_sweep[k] = times[k];
  }
  if (n_results) *n_results = (int)cand.size();
  if (best) *best = ibest;
  return IPM_OK;
}

extern "C" int ipm_batch_results(ipm_batch_t B, int *status, int *iters, double *obj,
                                 double *kkt_err, int *n_factor, int *ls_steps) {
  if (!B) return IPM_ERR_BAD_ARG;
  std::vector<BCtl> h(B->count);
  CK(cudaMemcpy(h.data(), B->d_ctl, sizeof(BCtl) * B->count, cudaMemcpyDeviceToHost));
  for (int i = 0; i < B->count; ++i) {
    if (status) status[i] = h[i].status;
    if (iters) iters[i] = h[i].k;
    if (obj) obj[i] = h[i].obj;
    if (kkt_err) kkt_err[i] = h[i].e0;
    if (n_factor) n_factor[i] = h[i].total_fac;
    if (ls_steps) ls_steps[i] = h[i].total_ls;
  }
  return IPM_OK;
}

extern "C" int ipm_batch_cg_iters(ipm_batch_t B, int *cg_iters) {
  if (!B || !cg_iters) return IPM_ERR_BAD_ARG;
  std::vector<BCtl> h(B->count);
  CK(cudaMemcpy(h.data(), B->d_ctl, sizeof(BCtl) * B->count, cudaMemcpyDeviceToHost));
  for (int i = 0; i < B->count; ++i) cg_iters[i] = h[i].cg_total;
  return IPM_OK;
}

extern "C" int ipm_batch_solve_info(ipm_batch_t B, int *current, int *iters32, int *k64,
                                    int *solves, int *above, double *eta_max) {
  if (!B) return IPM_ERR_BAD_ARG;
  std::vector<BCtl> h(B->count);
  CK(cudaMemcpy(h.data(), B->d_ctl, sizeof(BCtl) * B->count, cudaMemcpyDeviceToHost));
  for (int i = 0; i < B->count; ++i) {
    if (current) current[i] = h[i].p32 ? 32 : 64;
    if (iters32) iters32[i] = h[i].it32;
    if (k64) k64[i] = h[i].k32;
    if (solves) solves[i] = h[i].n_solve;
    if (above) above[i] = h[i].n_above;
    if (eta_max) eta_max[i] = h[i].eta_worst;
  }
  return IPM_OK;
}

extern "C" int ipm_batch_resto_counts(ipm_batch_t B, int *phases, int *iters) {
  if (!B) return IPM_ERR_BAD_ARG;
  std::vector<BCtl> h(B->count);
  CK(cudaMemcpy(h.data(), B->d_ctl, sizeof(BCtl) * B->count, cudaMemcpyDeviceToHost));
  for (int i = 0; i < B->count; ++i) {
    if (phases) phases[i] = h[i].n_resto;
    if (iters) iters[i] = h[i].total_resto;
  }
  return IPM_OK;
}

extern "C" int ipm_batch_export(ipm_batch_t B, int i, double *x) {
  if (!B || i < 0 || i >= B->count || !x) return IPM_ERR_BAD_ARG;
  BI h;
  CK(cudaMemcpy(&h, B->d_bi + i, sizeof(BI), cudaMemcpyDeviceToHost));
  CK(cudaMemcpy(x, h.P.x, sizeof(double) * h.D.n, cudaMemcpyDeviceToHost));
  return IPM_OK;
}

extern "C" int ipm_batch_sweeps(ipm_batch_t B) { return B ? B->sweeps : 0; }

extern "C" void ipm_batch_destroy(ipm_batch_t B) {
  if (!B) return;
  drop_graph(B);
  for (ipm_sym_t S : B->syms) ipm_symbolic_destroy(S);
  void *ps[] = {B->dpool, B->ipool, B->d_bi, B->d_ctl, B->d_tickets, B->d_order,
                B->d_order_all};
  for (void *p : ps)
    if (p) cudaFree(p);
  if (B->h_active) cudaFreeHost(B->h_active);
  for (void *p : B->bufs) cudaFree(p);
  for (cudaEvent_t e : B->ev)
    if (e) cudaEventDestroy(e);
  if (B->x_stage) cudaFree(B->x_stage);
  if (B->side) cudaStreamDestroy(B->side);
  if (B->ev_fork) cudaEventDestroy(B->ev_fork);
  if (B->ev_join) cudaEventDestroy(B->ev_join);
  delete B;
}

extern "C" int ipm_batch_work(ipm_batch_t B, double *factor_flops, double *condense_flops,
                              double *bytes) {
  if (!B) return IPM_ERR_BAD_ARG;
  for (int i = 0; i < B->count; ++i) {
    ipm_sym_t S = B->syms[B->pat[i]];
    const OpfData &M = B->opf[i]->M;
    if (factor_flops) factor_flops[i] = S->flops;
    if (condense_flops) condense_flops[i] = 2.0 * (double)S->nitems;
    if (bytes)
      bytes[i] = 8.0 * ((double)M.nnzJ + M.me + M.mi + M.nnzW + M.n) + 8.0 * (double)S->panel_len;
  }
  return IPM_OK;
}

extern "C" int ipm_batch_set_timing(ipm_batch_t B, int on) {
  if (!B) return IPM_ERR_BAD_ARG;
  if ((on != 0) == B->timing) return IPM_OK;
  if (on && !B->ev[0])
    for (cudaEvent_t &e : B->ev) CK(cudaEventCreate(&e));
  B->timing = on != 0;
  if (B->exec) {  // the captured sweep changes: capture again at the next run
    cudaGraphExecDestroy(B->exec);
    cudaGraphDestroy(B->graph);
    B->exec = nullptr;
    B->graph = nullptr;
  }
  return IPM_OK;
}

extern "C" int ipm_batch_kernel_time(ipm_batch_t B, double *fact_ms, double *solve_ms,
                                     int *sweeps) {
  if (!B) return IPM_ERR_BAD_ARG;
  if (fact_ms) *fact_ms = B->t_fact_ms;
  if (solve_ms) *solve_ms = B->t_solve_ms;
  if (sweeps) *sweeps = B->t_n;
  return IPM_OK;
}

__global__ void k_b_gather_x(const BI *bi, const int64_t *off, double *out) {
  const int b = blockIdx.y;
  const BI &I = bi[b];
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < I.D.n; j += gridDim.x * blockDim.x)
    out[off[b] + j] = I.P.x[j];
}

extern "C" int ipm_batch_export_all(ipm_batch_t B, double *x_host) {
  if (!B || !x_host) return IPM_ERR_BAD_ARG;
  if (!B->x_stage) {
    std::vector<BI> h(B->count);
    CK(cudaMemcpy(h.data(), B->d_bi, sizeof(BI) * B->count, cudaMemcpyDeviceToHost));
    B->x_off.assign(B->count + 1, 0);
    for (int i = 0; i < B->count; ++i) B->x_off[i + 1] = B->x_off[i] + h[i].D.n;
    B->x_total = B->x_off[B->count];
    CK(cudaMalloc(&B->x_stage, sizeof(double) * (B->x_total + B->count + 1)));
    // the offsets live after the staged values
    CK(cudaMemcpy(B->x_stage + B->x_total, B->x_off.data(), sizeof(int64_t) * (B->count + 1),
                  cudaMemcpyHostToDevice));
  }
  CKR(after_host_copies(B));
  k_b_gather_x<<<dim3(B->gx, B->count), B_BLOCK, 0, B->stream>>>(
      B->d_bi, (const int64_t *)(B->x_stage + B->x_total), B->x_stage);
  count_launches(1);
  CKL();
  CK(cudaMemcpyAsync(x_host, B->x_stage, sizeof(double) * B->x_total, cudaMemcpyDeviceToHost,
                     B->stream));
  CK(cudaStreamSynchronize(B->stream));
  return IPM_OK;
}

extern "C" int ipm_batch_state_rows(ipm_batch_t B, float *out, int64_t ld, int *width) {
  if (!B) return IPM_ERR_BAD_ARG;
  std::vector<BI> h(B->count);
  CK(cudaMemcpy(h.data(), B->d_bi, sizeof(BI) * B->count, cudaMemcpyDeviceToHost));
  const int w = 3 * h[0].D.n + 2 * h[0].D.mi + h[0].D.me;
  for (const BI &I : h)
    if (3 * I.D.n + 2 * I.D.mi + I.D.me != w) {
      set_error_msg("ipm_batch_state_rows: instances of different sizes");
      return IPM_ERR_BAD_ARG;
    }
  if (width) *width = w;
  if (!out) return IPM_OK;
  if (ld < w) return IPM_ERR_BAD_ARG;
  k_b_state_rows<<<dim3(B->gx, B->count), B_BLOCK, 0, B->stream>>>(B->d_bi, out, ld);
  count_launches(1);
  CKL();
  return IPM_OK;
}

extern "C" int ipm_batch_warm_start(ipm_batch_t B, const float *pred, int64_t ld,
                                    const float *mean, const float *stdv, int *h_used) {
  int w = 0;
  if (!B || !pred || (mean && !stdv)) return IPM_ERR_BAD_ARG;
  CKR(ipm_batch_state_rows(B, nullptr, 0, &w));
  if (ld < w) return IPM_ERR_BAD_ARG;
  cudaStream_t s = B->stream;
  const dim3 g2(B->gx, B->count), blk(B_BLOCK);
  k_b_rreset<<<B->count, 32, 0, s>>>(B->d_bi, B->d_ctl, PH_EVAL, R_PD, R_QD + 1, 0.0);
  k_b_warm_check<<<g2, blk, 0, s>>>(B->d_bi, pred, ld, mean, stdv);
  k_b_warm_apply<<<g2, blk, 0, s>>>(B->d_bi, pred, ld, mean, stdv);
  int *used = nullptr;
  CK(cudaMalloc(&used, sizeof(int) * B->count));
  k_b_warm_ctl<<<grid_for(B->count, 128), 128, 0, s>>>(B->d_bi, B->d_ctl, B->count, B->opt.tol,
                                                       used);
  count_launches(4);
  CKL();
  std::vector<int> hu(B->count);
  cudaError_t e = cudaMemcpyAsync(hu.data(), used, sizeof(int) * B->count, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  cudaFree(used);
  CK(e);
  if (h_used) std::copy(hu.begin(), hu.end(), h_used);
  return IPM_OK;
}

// the batched kernels keep their own copy of the spin limit
int batch_set_spin_limit(long long polls) {
  CK(cudaMemcpyToSymbol(g_spin_limit, &polls, sizeof(polls)));
  return IPM_OK;
}

extern "C" int ipm_batch_pause_at(ipm_batch_t B, int k) {
  if (!B || k < -1) return IPM_ERR_BAD_ARG;
  CK(cudaMemcpy(B->d_tickets + 12, &k, sizeof(int), cudaMemcpyHostToDevice));
  return IPM_OK;
}

extern "C" int ipm_batch_resume(ipm_batch_t B) {
  if (!B) return IPM_ERR_BAD_ARG;
  CKR(after_host_copies(B));
  k_b_resume<<<grid_for(B->count, 128), 128, 0, B->stream>>>(B->d_ctl, B->count);
  count_launches(1);
  CKL();
  CK(cudaStreamSynchronize(B->stream));
  return IPM_OK;
}

extern "C" int ipm_batch_export_kkt(ipm_batch_t B, int i, double *W_val, double *sigma,
                                    double *J_val, double *d_row, double *delta_w, double *a,
                                    double *b, double *dx, double *dyz, int *m_e) {
  if (!B || i < 0 || i >= B->count) return IPM_ERR_BAD_ARG;
  CK(cudaStreamSynchronize(B->stream));
  BI I;
  BCtl c;
  CK(cudaMemcpy(&I, B->d_bi + i, sizeof(BI), cudaMemcpyDeviceToHost));
  CK(cudaMemcpy(&c, B->d_ctl + i, sizeof(BCtl), cudaMemcpyDeviceToHost));
  if (c.ph != PH_PAUSE) {
    set_error_msg("ipm_batch_export_kkt: instance " + std::to_string(i) +
                  " is not held after a KKT solve (ipm_batch_pause_at)");
    return IPM_ERR_BAD_ARG;
  }
  const int n = I.D.n, me0 = I.D.me0, m = I.m;
  auto get = [&](double *dst, const double *src, int64_t count) -> int {
    if (dst && count > 0)
      CK(cudaMemcpy(dst, src, sizeof(double) * count, cudaMemcpyDeviceToHost));
    return IPM_OK;
  };
  CKR(get(W_val, I.Wv, I.M.nnzW));
  CKR(get(sigma, I.SA.sigma, n));
  CKR(get(J_val, I.Jv, I.M.nnzJ));
  CKR(get(d_row, I.dcond, m));
  CKR(get(a, I.a, n));
  CKR(get(b, I.baug, m));
  CKR(get(dx, I.dx, n));
  const bool hykkt = B->opt.kkt == 1;
  if (hykkt) {
    CKR(get(dyz, I.cg_dy, me0));
    CKR(get(dyz ? dyz + me0 : nullptr, I.dzc + me0, m - me0));
  } else {
    CKR(get(dyz, I.dzc, m));
  }
  if (delta_w) *delta_w = c.dw;
  if (m_e) *m_e = hykkt ? me0 : 0;
  return IPM_OK;
}

extern "C" int ipm_batch_set_tail(ipm_batch_t B, int active_max, int cluster) {
  if (!B || active_max < 0 ||
      (cluster != 0 && cluster != 1 && cluster != 2 && cluster != 4 && cluster != 8))
    return IPM_ERR_BAD_ARG;
  B->tail_active = active_max;
  B->tail_cl = cluster;
  drop_graph(B);
  return IPM_OK;
}

extern "C" int ipm_batch_set_shape(ipm_batch_t B, int cluster, int big_num, int big_den, int gx,
                                   int *n_big) {
  if (!B || (cluster != 1 && cluster != 2 && cluster != 4 && cluster != 8) || big_num < 0 ||
      big_den < 0 || gx > 16)
    return IPM_ERR_BAD_ARG;
  B->cl_big = cluster;
  B->big_num = big_num;
  B->big_den = big_den;
  if (gx > 0) B->gx = gx;
  drop_graph(B);
  CKR(set_order(B));
  if (n_big) *n_big = B->n_big;
  return IPM_OK;
}
