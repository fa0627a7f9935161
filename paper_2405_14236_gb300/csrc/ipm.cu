// One primal-dual interior-point iteration on the GPU (ipm_step).
//
// Problem (2) of the paper with slacks h(x) + s = 0, s >= 0 and Ipopt-style variable bounds
// (bound multipliers zl, zu eliminated into Sigma_x on the diagonal of K).  The Newton step
// (K_2) is solved in condensed form, either
//   LiftedKKT (Section 3.2): equalities relaxed to -tau <= g <= tau, i.e. rows g - tau <= 0 and
//     -g - tau <= 0 in front of h <= 0; each pair of relaxed rows shares the pattern of its G
//     row, so K_tau = W + Sigma_x + delta_w I + G^T (D1 + D2) G + H^T D_H H is condensed from
//     J = [G; H] and the step is refined on the augmented system (ipm_aug_solve), or
//   HyKKT (Section 3.1): K_gamma = K + gamma G^T G and CG on the Schur complement (hykkt_cg).
// The line search, barrier update, inertia correction and safeguards are those of Ipopt
// (Waechter & Biegler 2006, cited in Section 2.2), with its published constants.  Decisions
// that need a few scalars (convergence, inertia, filter acceptance) read them back to the host.
#include <algorithm>
#include <cmath>
#include <vector>

#include "internal.cuh"
#include "ipm_core.cuh"
#include "opf.cuh"
#include "resto_dev.cuh"

namespace cipm {

// ------------------------------------------------------------------ set-up kernels
__global__ void k_setup_sums(int nb, const double *pd, const double *qd, double *R) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  double a = i < nb ? pd[i] : 0.0, b = i < nb ? qd[i] : 0.0;
  red_sum(R, R_PD, a);
  red_sum(R, R_QD, b);
}

__global__ void k_x0(int nb, int ng, const double *R, const double *xl, const double *xu,
                     double *x) {
  int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j < 2 * nb + 2 * ng) x[j] = x0_at(nb, ng, R[R_PD], R[R_QD], xl, xu, j);
}
__global__ void k_push(int n, const double *xl, const double *xu, double *x) {
  int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j < n) x[j] = push_at(x[j], xl, xu, j);
}

// row scale d_r = min(1, 100 / max_j |J_rj|) (Ipopt gradient-based scaling)
__device__ __forceinline__ double row_scale_at(const int *rowptr, const double *Jv, int r) {
  double mx = 0.0;
  for (int p = rowptr[r]; p < rowptr[r + 1]; ++p) mx = fmax(mx, fabs(Jv[p]));
  return mx > 0.0 ? fmin(1.0, 100.0 / mx) : 1.0;
}
__global__ void k_row_scale(int m, const int *rowptr, const double *Jv, double *d) {
  int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r < m) d[r] = row_scale_at(rowptr, Jv, r);
}

__global__ void k_max_abs(int n, const double *v, double *R, int k) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  red_max(R, k, i < n ? fabs(v[i]) : 0.0);
}

// scale the model outputs: g~ = d_e g, h~ = d_i h, J~ rows by d
__global__ void k_scale_rows(int m, const int *rowptr, const double *d, double *Jv) {
  int r = blockIdx.x * blockDim.y + threadIdx.y;
  if (r >= m) return;
  const double dr = d[r];
  for (int p = rowptr[r] + threadIdx.x; p < rowptr[r + 1]; p += blockDim.x) Jv[p] *= dr;
}
__global__ void k_scale_vec(int n, const double *d, double *v) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) v[i] *= d[i];
}

__global__ void k_ipm_rows(Dims D, double tau, const double *gs, const double *hs, double *geq,
                           double *hin) {
  ipm_rows_at(D, tau, gs, hs, geq, hin, blockIdx.x * blockDim.x + threadIdx.x);
}

__global__ void k_lambda(Dims D, const double *y, const double *z, double *lam) {
  lambda_at(D, y, z, lam, blockIdx.x * blockDim.x + threadIdx.x);
}

__global__ void k_mul(int n, const double *a, const double *b, double *out) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = a[i] * b[i];
}

// out_j = sum_p J~_pj u_row(p) (J^T u)
__device__ __forceinline__ double jtu_at(const int *JT_ptr, const int *JT_ent, const int *rowidx,
                                         const double *Jv, const double *u, int j) {
  double acc = 0.0;
  for (int t = JT_ptr[j]; t < JT_ptr[j + 1]; ++t) {
    int p = JT_ent[t];
    acc += Jv[p] * u[rowidx[p]];
  }
  return acc;
}
__global__ void k_jtu(int n, const int *JT_ptr, const int *JT_ent, const int *rowidx,
                      const double *Jv, const double *u, double *out) {
  int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j < n) out[j] = jtu_at(JT_ptr, JT_ent, rowidx, Jv, u, j);
}
// out_r = (J~ v)_r
__device__ __forceinline__ double jv_at(const int *rowptr, const int *colind, const double *Jv,
                                        const double *v, int r) {
  double acc = 0.0;
  for (int p = rowptr[r]; p < rowptr[r + 1]; ++p) acc += Jv[p] * v[colind[p]];
  return acc;
}
__global__ void k_jv(int m, const int *rowptr, const int *colind, const double *Jv,
                     const double *v, double *out) {
  int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r < m) out[r] = jv_at(rowptr, colind, Jv, v, r);
}

__global__ void k_errors(Dims D, It P, double sig, double mu, double *R) {
  const ErrParts E = errors_at(D, P, sig, mu, blockIdx.x * blockDim.x + threadIdx.x);
  red_max(R, R_MAX_GL, E.gl);
  red_max(R, R_MAX_ZV, E.zv);
  red_max(R, R_MAX_G, E.ge);
  red_max(R, R_MAX_HS, E.hs);
  red_max(R, R_MAX_SV, E.sv);
  red_max(R, R_MAX_XL, E.xl);
  red_max(R, R_MAX_XU, E.xu);
  red_sum(R, R_SUM_Y, E.sy);
  red_sum(R, R_SUM_Z, E.sz);
  red_sum(R, R_SUM_V, E.svv);
  red_sum(R, R_SUM_ZL, E.szl);
  red_sum(R, R_SUM_ZU, E.szu);
}

__global__ void k_merit(Dims D, const double *x, const double *s, const double *xl,
                        const double *xu, const double *geq, const double *hin, double *R) {
  const MeritParts M = merit_at(D, x, s, xl, xu, geq, hin, blockIdx.x * blockDim.x + threadIdx.x);
  red_sum(R, R_TH_G, M.tg);
  red_sum(R, R_TH_H, M.th);
  red_sum(R, R_LOG_S, M.ls);
  red_sum(R, R_LOG_XL, M.lxl);
  red_sum(R, R_LOG_XU, M.lxu);
}

__global__ void k_newton_rhs(Dims D, It P, double sig, double mu, double *sigma, double *r1,
                             double *r2, double *r4, double *Ds) {
  newton_rhs_at(D, P, sig, mu, sigma, r1, r2, r4, Ds, blockIdx.x * blockDim.x + threadIdx.x);
}

__global__ void k_aug_rhs(Dims D, double dw, double gamma, const double *r2, const double *r4,
                          const double *Ds, const double *geq, double *d, double *b) {
  aug_rhs_at(D, dw, gamma, r2, r4, Ds, geq, d, b, blockIdx.x * blockDim.x + threadIdx.x);
}

__global__ void k_neg(int n, const double *a, double *out) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = -a[i];
}

__global__ void k_recover(StepArgs A) { recover_at(A, blockIdx.x * blockDim.x + threadIdx.x); }

__global__ void k_ftb(StepArgs A, double tau, double sig, double *R) {
  const FtbParts F = ftb_at(A, tau, sig, blockIdx.x * blockDim.x + threadIdx.x);
  red_min(R, R_AMAX, F.ap);
  red_min(R, R_AZ, F.az);
  red_sum(R, R_GPHI_X, F.gx);
  red_sum(R, R_GPHI_S, F.gs);
}

__global__ void k_trial(int n, int mi, double a, const double *x, const double *dx,
                        const double *s, const double *ds, double *xt, double *st) {
  trial_at(n, mi, a, x, dx, s, ds, xt, st, blockIdx.x * blockDim.x + threadIdx.x);
}

__global__ void k_accept(StepArgs A, double alpha, double az, const double *xt, const double *st,
                         const double *dy) {
  accept_at(A, alpha, az, xt, st, dy, blockIdx.x * blockDim.x + threadIdx.x);
}

// ||K|| bound for the automatic gamma: per column j the row sum of |W + Sigma_x| plus
// sum over H rows r of |Ds_r| |J_rj| sum_t |J_rt| (delta_w = 0), max-reduced into R[k_out];
// and max over G rows of sum |G_rj| into R[g_out]
__global__ void k_gamma_norms(Dims D, const int *W_rowptr, const int *W_colind,
                              const int *W_rowidx, const int *WT_ptr, const int *WT_ent,
                              const double *Wv, const double *sigma, const int *JT_ptr,
                              const int *JT_ent, const int *J_rowidx, const int *J_rowptr,
                              const double *Jv, const double *Ds, double *R, int k_out,
                              int g_out) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  double acc = 0.0, gr = 0.0;
  if (j < D.n) {
    double diag = sigma[j];
    for (int q = W_rowptr[j]; q < W_rowptr[j + 1]; ++q) {
      if (W_colind[q] == j) diag += Wv[q];
      else acc += fabs(Wv[q]);
    }
    for (int u = WT_ptr[j]; u < WT_ptr[j + 1]; ++u) {
      const int e = WT_ent[u];
      if (W_rowidx[e] != j) acc += fabs(Wv[e]);
    }
    acc += fabs(diag);
    for (int u = JT_ptr[j]; u < JT_ptr[j + 1]; ++u) {
      const int q = JT_ent[u];
      const int r = J_rowidx[q];
      if (r < D.me0) continue;
      double rs = 0.0;
      for (int t = J_rowptr[r]; t < J_rowptr[r + 1]; ++t) rs += fabs(Jv[t]);
      acc += fabs(Ds[r - D.me0]) * fabs(Jv[q]) * rs;
    }
  }
  if (j < D.me0)
    for (int t = J_rowptr[j]; t < J_rowptr[j + 1]; ++t) gr += fabs(Jv[t]);
  red_max(R, k_out, acc);
  red_max(R, g_out, gr);
}

__global__ void k_init_duals(Dims D, It P, double *s) {
  init_duals_at(D, P, s, blockIdx.x * blockDim.x + threadIdx.x);
}

// ------------------------------------------------------------------ restoration phase kernels
__global__ void k_rows_absmax(Dims D, const double *geq, const double *hin, const double *s,
                              double *R) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  red_max(R, R_RS_PRIM, i < D.me + D.mi ? fabs(r_c(D, geq, hin, s, i)) : 0.0);
}
__global__ void k_resto_start(RArgs A, double mu_r, double *xr, double *dr2) {
  resto_start_at(A, mu_r, xr, dr2, blockIdx.x * blockDim.x + threadIdx.x);
}
__global__ void k_resto_rhs(RArgs A) { resto_rhs_at(A, blockIdx.x * blockDim.x + threadIdx.x); }
__global__ void k_resto_aug(RArgs A, double *d, double *b) {
  resto_aug_at(A, d, b, blockIdx.x * blockDim.x + threadIdx.x);
}
__global__ void k_resto_recover(RArgs A) {
  resto_recover_at(A, blockIdx.x * blockDim.x + threadIdx.x);
}
__global__ void k_resto_ftb(RArgs A, double tau, double *R) {
  double ap, az, g;
  resto_ftb_at(A, tau, &ap, &az, &g, blockIdx.x * blockDim.x + threadIdx.x);
  red_min(R, R_AMAX, ap);
  red_min(R, R_AZ, az);
  red_sum(R, R_GPHI_X, g);
}
__global__ void k_resto_trial(RArgs A, double a, double *xt, double *st, double *pt,
                              double *qt) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < A.D.n) xt[i] = A.P.x[i] + a * A.dx[i];
  if (i < A.D.mi) st[i] = A.P.s[i] + a * A.ds[i];
  if (i < A.D.me + A.D.mi) {
    pt[i] = A.p[i] + a * A.dp[i];
    qt[i] = A.q[i] + a * A.dq[i];
  }
}
__global__ void k_resto_merit(RArgs A, const double *xt, const double *st, const double *pt,
                              const double *qt, const double *geqt, const double *hint,
                              double *R) {
  const RMerit M = resto_merit_at(A, xt, st, pt, qt, geqt, hint,
                                  blockIdx.x * blockDim.x + threadIdx.x);
  red_sum(R, R_TH_G, M.th);
  red_sum(R, R_RS_OBJ, M.obj);
  red_sum(R, R_LOG_S, M.ls);
  red_sum(R, R_LOG_XL, M.lxl);
  red_sum(R, R_LOG_XU, M.lxu);
}
__global__ void k_resto_errors(RArgs A, double mu, double *R) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const RErr E = resto_errors_at(A, mu, i);
  // the original problem's violation ||c||_inf
  red_max(R, R_MAX_G, i < A.D.me + A.D.mi ? fabs(r_c(A.D, A.P.geq, A.P.hin, A.P.s, i)) : 0.0);
  red_max(R, R_RS_DUAL, E.dual);
  red_max(R, R_RS_PRIM, E.prim);
  red_max(R, R_RS_COMP, E.comp);
  red_sum(R, R_RS_SUMD, E.sumd);
  red_sum(R, R_RS_SUMC, E.sumc);
}
__global__ void k_resto_accept(RArgs A, double alpha, double az, const double *xt,
                               const double *st, const double *pt, const double *qt) {
  resto_accept_at(A, alpha, az, xt, st, pt, qt, blockIdx.x * blockDim.x + threadIdx.x);
}
__global__ void k_resto_finish(Dims D, It P) {
  resto_finish_at(D, P, blockIdx.x * blockDim.x + threadIdx.x);
}

}  // namespace cipm

using namespace cipm;

struct ipm_state_s {
  ipm_opf_t opf = nullptr;
  ipm_options opt;
  cudaStream_t stream = 0;
  Dims D;
  ipm_sym_t sym = nullptr;
  ipm_num_t num = nullptr;    // the factor in use
  ipm_num_t num32 = nullptr;  // FP32 factor while it serves (precision 32), else null
  std::vector<double *> bufs;
  It P;
  double *dscale, *gs, *hs, *Jv, *Wv, *lam, *lamw, *f;
  double *sigma, *r1, *r2, *r4, *Ds, *dcond, *baug, *a, *dx, *dy, *dzH, *dzc, *jdx;
  double *dz, *ds, *dv, *dzl, *dzu, *xt, *st, *geqt, *hint, *gst, *hst, *ft;
  double *R = nullptr, *hR = nullptr, *eta = nullptr;
  int *info = nullptr, *steps = nullptr;
  int nnzJ = 0, nnzW = 0, nb = 0, ng = 0;
  // host-side algorithm state
  double sig = 1.0, mu = 0.1, tau = 0.99, delta_last = 0.0;
  double theta_max = 0, theta_min = 0;
  bool have_theta0 = false;
  std::vector<double> filter;  // interleaved (theta, phi) entries
  int k = 0;
  int status = 0;  // 0 running, 1 converged, <0/IPM_ERR_* failure
  int nl = 0, nu = 0;
  bool have_kkt = false;  // a KKT solve has completed (ipm_state_export_kkt)
  bool kkt_resto = false;  // ... and it was a step of the restoration problem (all rows condensed)
  double last_dw = 0.0;
  // restoration phase: per IPM row p, q, their duals, steps and trial values; reference point
  double *rp = nullptr, *rq = nullptr, *rzp = nullptr, *rzq = nullptr, *rdp = nullptr,
         *rdq = nullptr, *rdzp = nullptr, *rdzq = nullptr, *rpt = nullptr, *rqt = nullptr;
  double *rxr = nullptr, *rdr2 = nullptr, *rrc = nullptr, *rrp = nullptr, *rrq = nullptr;
  bool in_resto = false, have_theta0_r = false;
  double prim_inf = INFINITY;  // ||c||_inf of the last main evaluation
  double rs_cinf = INFINITY;   // the same at the last restoration evaluation
  double mu_r = 0, zeta_r = 0, tau_r = 0, theta_start = 0, theta_max_r = 0, theta_min_r = 0;
  double delta_last_r = 0, entry_theta = 0, entry_phi = 0;
  std::vector<double> filter_r;
  int k_r = 0;
};

static int grid1(int64_t n) { return grid_for(n > 0 ? n : 1, 256); }

static int st_alloc(ipm_state_t S, double **p, int64_t n) {
  CKR(dev_alloc(p, n > 0 ? n : 1));
  S->bufs.push_back(*p);
  return IPM_OK;
}

static int reduce_reset(ipm_state_t S, std::initializer_list<int> which, double init) {
  for (int k : which) {
    // +inf for min-reductions, 0 otherwise (bit patterns of non-negative doubles)
    CK(cudaMemcpyAsync(S->R + k, &init, sizeof(double), cudaMemcpyHostToDevice, S->stream));
  }
  return IPM_OK;
}

static int read_R(ipm_state_t S) {
  CK(cudaMemcpyAsync(S->hR, S->R, sizeof(double) * R_COUNT, cudaMemcpyDeviceToHost, S->stream));
  CK(cudaStreamSynchronize(S->stream));
  return IPM_OK;
}

// model evaluation at x (constraints scaled, IPM rows built); with_jac: also J~, grad, J~^T lambda
static int eval_point(ipm_state_t S, const double *x, double *gs, double *hs, double *geq,
                      double *hin, double *f, bool with_jac) {
  const OpfData &M = S->opf->M;
  cudaStream_t s = S->stream;
  CKR(opf_eval(M, x, nullptr, nullptr, 1.0, f, with_jac ? S->P.grad : nullptr, gs, hs,
               with_jac ? S->Jv : nullptr, nullptr, s));
  k_scale_vec<<<grid1(S->D.me0), 256, 0, s>>>(S->D.me0, S->dscale, gs);
  k_scale_vec<<<grid1(S->D.mi0), 256, 0, s>>>(S->D.mi0, S->dscale + S->D.me0, hs);
  k_ipm_rows<<<grid1(std::max(S->D.me0, S->D.mi0)), 256, 0, s>>>(S->D, S->opt.tau, gs, hs, geq,
                                                                 hin);
  CKL();
  if (with_jac) {
    const int m = S->D.me0 + S->D.mi0;
    dim3 blk(32, 8);
    k_scale_rows<<<grid_for(m, 8), blk, 0, s>>>(m, M.J_rowptr, S->dscale, S->Jv);
    CKL();
  }
  return IPM_OK;
}

static int jt_lambda(ipm_state_t S) {
  cudaStream_t s = S->stream;
  const int m = S->D.me0 + S->D.mi0;
  k_lambda<<<grid1(std::max(S->D.me0, S->D.mi0)), 256, 0, s>>>(S->D, S->P.y, S->P.z, S->lam);
  CKL();
  k_jtu<<<grid1(S->D.n), 256, 0, s>>>(S->D.n, S->sym->JT_ptr, S->sym->JT_ent, S->sym->J_rowidx,
                                      S->Jv, S->lam, S->P.jtl);
  CKL();
  (void)m;
  return IPM_OK;
}

static int errors(ipm_state_t S, double mu, double *out) {
  CKR(reduce_reset(S, {R_MAX_GL, R_MAX_ZV, R_MAX_G, R_MAX_HS, R_MAX_SV, R_MAX_XL, R_MAX_XU,
                       R_SUM_Y, R_SUM_Z, R_SUM_V, R_SUM_ZL, R_SUM_ZU}, 0.0));
  int nmax = std::max({S->D.n, S->D.me, S->D.mi});
  k_errors<<<grid1(nmax), 256, 0, S->stream>>>(S->D, S->P, S->sig, mu, S->R);
  CKL();
  CKR(read_R(S));
  const double *h = S->hR;
  *out = kkt_error(h, S->D, S->nl, S->nu, std::max({h[R_MAX_SV], h[R_MAX_XL], h[R_MAX_XU]}));
  S->prim_inf = std::max(h[R_MAX_G], h[R_MAX_HS]);
  return IPM_OK;
}

// theta, phi at (x, s) with rows (geq, hin) and objective value *f (device)
static int merit(ipm_state_t S, const double *x, const double *sv, const double *geq,
                 const double *hin, const double *f, double mu, double *theta, double *phi) {
  CKR(reduce_reset(S, {R_TH_G, R_TH_H, R_LOG_S, R_LOG_XL, R_LOG_XU}, 0.0));
  int nmax = std::max({S->D.n, S->D.me, S->D.mi});
  k_merit<<<grid1(nmax), 256, 0, S->stream>>>(S->D, x, sv, S->P.xl, S->P.xu, geq, hin, S->R);
  CKL();
  double fv = 0.0;
  CK(cudaMemcpyAsync(&fv, f, sizeof(double), cudaMemcpyDeviceToHost, S->stream));
  CKR(read_R(S));
  const double *h = S->hR;
  *theta = h[R_TH_G] + h[R_TH_H];
  *phi = S->sig * fv - mu * (h[R_LOG_S] + h[R_LOG_XL] + h[R_LOG_XU]);
  return IPM_OK;
}

static int state_create(ipm_opf_t opf, const ipm_options *opt, const double *x0_host,
                        cudaStream_t stream, ipm_state_t *out);

extern "C" int ipm_state_create(ipm_opf_t opf, const ipm_options *opt, cudaStream_t stream,
                                ipm_state_t *out) {
  return state_create(opf, opt, nullptr, stream, out);
}

extern "C" int ipm_state_create_at(ipm_opf_t opf, const ipm_options *opt, const double *x0,
                                   cudaStream_t stream, ipm_state_t *out) {
  if (!x0) return IPM_ERR_BAD_ARG;
  return state_create(opf, opt, x0, stream, out);
}

static int state_create(ipm_opf_t opf, const ipm_options *opt, const double *x0_host,
                        cudaStream_t stream, ipm_state_t *out) {
  if (!opf || !opt || !out || opt->kkt < 0 || opt->kkt > 2 || !(opt->tol > 0)) {
    set_error_msg("ipm_state_create: bad argument");
    return IPM_ERR_BAD_ARG;
  }
  *out = nullptr;
  // creation runs on the set-up stream; the iterations on the caller's
  const cudaStream_t caller = stream;
  stream = setup_stream(stream);
  ipm_state_t S = new ipm_state_s();
  S->opf = opf;
  S->opt = *opt;
  if (!(S->opt.tau > 0)) S->opt.tau = S->opt.tol;
  if (!(S->opt.mu0 > 0)) S->opt.mu0 = 0.1;
  if (!(S->opt.cg_rtol > 0)) S->opt.cg_rtol = 1e-10;
  if (S->opt.max_refine < 0) S->opt.max_refine = 10;
  S->stream = stream;
  const OpfData &M = opf->M;
  Dims &D = S->D;
  D.n = M.n;
  D.me0 = M.me;
  D.mi0 = M.mi;
  D.lifted = opt->kkt == 0;  // HyKKT (1) and the dual-regularized form (2) keep the equalities
  D.me = D.lifted ? 0 : M.me;
  D.mi = D.lifted ? 2 * M.me + M.mi : M.mi;
  S->nb = M.nb;
  S->ng = M.ng;
  S->nnzJ = M.nnzJ;
  S->nnzW = M.nnzW;
  const int n = D.n, m = M.me + M.mi;
  int rc = IPM_OK;
  auto A = [&](double **p, int64_t k) {
    if (rc == IPM_OK) rc = st_alloc(S, p, k);
  };
  A(&S->P.x, n); A(&S->P.s, D.mi); A(&S->P.y, D.me); A(&S->P.z, D.mi); A(&S->P.v, D.mi);
  A(&S->P.zl, n); A(&S->P.zu, n); A(&S->P.grad, n); A(&S->P.jtl, n);
  A(&S->P.geq, D.me); A(&S->P.hin, D.mi);
  A(&S->dscale, m); A(&S->gs, M.me); A(&S->hs, M.mi); A(&S->Jv, M.nnzJ); A(&S->Wv, M.nnzW);
  A(&S->lam, m); A(&S->lamw, m); A(&S->f, 2);
  A(&S->sigma, n); A(&S->r1, n); A(&S->r2, D.mi); A(&S->r4, D.mi); A(&S->Ds, D.mi);
  A(&S->dcond, m); A(&S->baug, m); A(&S->a, n); A(&S->dx, n); A(&S->dy, M.me); A(&S->dzH, M.mi);
  A(&S->dzc, m); A(&S->jdx, m);
  A(&S->dz, D.mi); A(&S->ds, D.mi); A(&S->dv, D.mi); A(&S->dzl, n); A(&S->dzu, n);
  A(&S->xt, n); A(&S->st, D.mi); A(&S->geqt, D.me); A(&S->hint, D.mi); A(&S->gst, M.me);
  A(&S->hst, M.mi); A(&S->ft, 2); A(&S->R, R_COUNT); A(&S->eta, 1);
  const int64_t nr = (int64_t)D.me + D.mi;
  A(&S->rp, nr); A(&S->rq, nr); A(&S->rzp, nr); A(&S->rzq, nr); A(&S->rdp, nr); A(&S->rdq, nr);
  A(&S->rdzp, nr); A(&S->rdzq, nr); A(&S->rpt, nr); A(&S->rqt, nr); A(&S->rrc, nr);
  A(&S->rrp, nr); A(&S->rrq, nr); A(&S->rxr, n); A(&S->rdr2, n);
  S->P.xl = M.xl;
  S->P.xu = M.xu;
  if (rc == IPM_OK) rc = dev_alloc(&S->info, 2);
  if (rc == IPM_OK) rc = dev_alloc(&S->steps, 2);
  if (rc == IPM_OK && cudaMallocHost((void **)&S->hR, sizeof(double) * R_COUNT) != cudaSuccess)
    rc = IPM_ERR_OOM;
  if (rc == IPM_OK) {
    // bounds present
    std::vector<double> hxl(n), hxu(n);
    if (cudaMemcpy(hxl.data(), M.xl, sizeof(double) * n, cudaMemcpyDeviceToHost) != cudaSuccess ||
        cudaMemcpy(hxu.data(), M.xu, sizeof(double) * n, cudaMemcpyDeviceToHost) != cudaSuccess)
      rc = IPM_ERR_CUDA;
    for (int j = 0; j < n; ++j) {
      S->nl += std::isfinite(hxl[j]);
      S->nu += std::isfinite(hxu[j]);
    }
  }
  if (rc == IPM_OK) {
    const bool dflt = S->opt.sn_relax_w <= 0;
    rc = ipm_symbolic_relaxed(n, m, M.J_rowptr, M.J_colind, M.nnzJ, M.W_rowptr, M.W_colind,
                              M.nnzW, dflt ? 8 : S->opt.sn_relax_w, dflt ? 5 : S->opt.sn_relax_den,
                              stream, &S->sym);
  }
  if (rc == IPM_OK) rc = ipm_num_create(S->sym, 64, &S->num);
  if (rc == IPM_OK && S->opt.precision == 32) rc = ipm_num_create(S->sym, 32, &S->num32);
  if (rc == IPM_OK) {
    // starting point, objective scaling and row scaling at x0 (Ipopt gradient-based scaling)
    cudaStream_t s = stream;
    if (cudaMemsetAsync(S->R, 0, sizeof(double) * R_COUNT, s) != cudaSuccess) rc = IPM_ERR_CUDA;
    if (x0_host) {
      // the caller's point, pushed inside the bounds
      if (cudaMemcpyAsync(S->P.x, x0_host, sizeof(double) * n, cudaMemcpyHostToDevice, s) !=
          cudaSuccess)
        rc = IPM_ERR_CUDA;
      k_push<<<grid1(n), 256, 0, s>>>(n, M.xl, M.xu, S->P.x);
    } else {
      k_setup_sums<<<grid1(M.nb), 256, 0, s>>>(M.nb, M.pd, M.qd, S->R);
      k_x0<<<grid1(n), 256, 0, s>>>(M.nb, M.ng, S->R, M.xl, M.xu, S->P.x);
      rc = opf_flow_start(M, S->P.x, s);
    }
    if (rc == IPM_OK)
      rc = opf_eval(M, S->P.x, nullptr, nullptr, 1.0, S->f, S->P.grad, S->gs, S->hs, S->Jv,
                    nullptr, s);
  }
  if (rc == IPM_OK) {
    cudaStream_t s = stream;
    k_row_scale<<<grid1(m), 256, 0, s>>>(m, M.J_rowptr, S->Jv, S->dscale);
    k_max_abs<<<grid1(n), 256, 0, s>>>(n, S->P.grad, S->R, R_MAXGRAD);
    if (read_R(S) != IPM_OK) rc = IPM_ERR_CUDA;
  }
  if (rc == IPM_OK) {
    S->sig = std::min(1.0, 100.0 / std::max(S->hR[R_MAXGRAD], 1e-300));
    rc = eval_point(S, S->P.x, S->gs, S->hs, S->P.geq, S->P.hin, S->f, true);
  }
  if (rc == IPM_OK) {
    k_init_duals<<<grid1(std::max({D.n, D.me, D.mi})), 256, 0, stream>>>(D, S->P, S->P.s);
    if (cudaStreamSynchronize(stream) != cudaSuccess) rc = IPM_ERR_CUDA;
  }
  S->mu = S->opt.mu0;
  S->tau = std::max(TAU_MIN, 1.0 - S->mu);
  if (rc != IPM_OK) {
    ipm_state_destroy(S);
    return rc;
  }
  S->stream = caller;
  *out = S;
  return IPM_OK;
}

extern "C" void ipm_state_destroy(ipm_state_t S) {
  if (!S) return;
  for (double *p : S->bufs) cudaFree(p);
  if (S->info) cudaFree(S->info);
  if (S->steps) cudaFree(S->steps);
  if (S->hR) cudaFreeHost(S->hR);
  if (S->num) ipm_num_destroy(S->num);
  if (S->num32) ipm_num_destroy(S->num32);
  if (S->sym) ipm_symbolic_destroy(S->sym);
  delete S;
}

// ------------------------------------------------------------------ restoration phase (host)
static RArgs rargs(ipm_state_t S, double dw) {
  RArgs A;
  A.D = S->D;
  A.P = S->P;
  A.p = S->rp; A.q = S->rq; A.zp = S->rzp; A.zq = S->rzq;
  A.xr = S->rxr; A.dr2 = S->rdr2;
  A.sigma = S->sigma; A.r1 = S->r1; A.r2 = S->r2; A.Ds = S->Ds;
  A.rc = S->rrc; A.rp = S->rrp; A.rq = S->rrq;
  A.mu = S->mu_r; A.zeta = S->zeta_r; A.dw = dw;
  A.dx = S->dx; A.jdx = S->jdx;
  A.dy = S->dy; A.dz = S->dz; A.ds = S->ds; A.dv = S->dv; A.dzl = S->dzl; A.dzu = S->dzu;
  A.dp = S->rdp; A.dq = S->rdq; A.dzp = S->rdzp; A.dzq = S->rdzq;
  return A;
}

static int nmax_r(ipm_state_t S) {
  return std::max({S->D.n, S->D.me + S->D.mi, S->D.me0 + S->D.mi0});
}

// theta_R, phi_R at (xt, st, pt, qt) with the model rows geqt / hint of xt
static int resto_merit(ipm_state_t S, const double *xt, const double *st, const double *pt,
                       const double *qt, const double *geqt, const double *hint, double mu,
                       double *theta, double *phi) {
  CKR(reduce_reset(S, {R_TH_G, R_RS_OBJ, R_LOG_S, R_LOG_XL, R_LOG_XU}, 0.0));
  k_resto_merit<<<grid1(nmax_r(S)), 256, 0, S->stream>>>(rargs(S, 0.0), xt, st, pt, qt, geqt,
                                                          hint, S->R);
  CKL();
  CKR(read_R(S));
  const double *h = S->hR;
  *theta = h[R_TH_G];
  *phi = h[R_RS_OBJ] - mu * (h[R_LOG_S] + h[R_LOG_XL] + h[R_LOG_XU]);
  return IPM_OK;
}

// scaled optimality error of the restoration problem (Ipopt's E_mu with its s_d, s_c; the bounds
// p, q >= 0 count among the bounds)
static int resto_errors(ipm_state_t S, double mu, double *out) {
  CKR(reduce_reset(S, {R_RS_DUAL, R_RS_PRIM, R_RS_COMP, R_RS_SUMD, R_RS_SUMC, R_MAX_G}, 0.0));
  k_resto_errors<<<grid1(nmax_r(S)), 256, 0, S->stream>>>(rargs(S, 0.0), mu, S->R);
  CKL();
  CKR(read_R(S));
  const double *h = S->hR;
  S->rs_cinf = h[R_MAX_G];
  const int R = S->D.me + S->D.mi, nb = S->nl + S->nu + 2 * R;
  const double sd = std::max(S_MAX, h[R_RS_SUMD] / std::max(S->D.me + 2 * S->D.mi + nb, 1)) / S_MAX;
  const double sc = std::max(S_MAX, h[R_RS_SUMC] / std::max(S->D.mi + nb, 1)) / S_MAX;
  *out = std::max({h[R_RS_DUAL] / sd, h[R_RS_PRIM], h[R_RS_COMP] / sc});
  return IPM_OK;
}

// enter the restoration phase at the current iterate (the line search failed); theta, phi of
// the main problem there, whose filter entry the phase must beat
static int resto_begin(ipm_state_t S, double theta, double phi) {
  cudaStream_t s = S->stream;
  CKR(reduce_reset(S, {R_RS_PRIM}, 0.0));
  k_rows_absmax<<<grid1(S->D.me + S->D.mi), 256, 0, s>>>(S->D, S->P.geq, S->P.hin, S->P.s, S->R);
  CKL();
  CKR(read_R(S));
  S->mu_r = std::max(S->mu, S->hR[R_RS_PRIM]);
  S->zeta_r = std::sqrt(S->mu_r);
  S->tau_r = std::max(TAU_MIN, 1.0 - S->mu_r);
  k_resto_start<<<grid1(nmax_r(S)), 256, 0, s>>>(rargs(S, 0.0), S->mu_r, S->rxr, S->rdr2);
  CKL();
  S->entry_theta = (1 - GAMMA_THETA) * theta;
  S->entry_phi = phi - GAMMA_PHI * theta;
  S->theta_start = theta;
  S->filter_r.clear();
  S->have_theta0_r = false;
  S->delta_last_r = 0.0;
  S->k_r = 0;
  S->in_resto = true;
  CK(cudaStreamSynchronize(s));
  return IPM_OK;
}

// one iteration of the filter IPM on the restoration problem, then the return test
static int resto_step(ipm_state_t S, ipm_iter_info *info) {
  cudaStream_t s = S->stream;
  const Dims &D = S->D;
  const OpfData &M = S->opf->M;
  const int n = D.n, m = D.me0 + D.mi0, nr = nmax_r(S);
  info->resto = 1;
  if (S->k_r >= 500) return IPM_ERR_RESTORATION;
  CKR(eval_point(S, S->P.x, S->gs, S->hs, S->P.geq, S->P.hin, S->f, true));
  CKR(jt_lambda(S));
  double e0, theta, phi;
  CKR(resto_errors(S, 0.0, &e0));
  if (!S->have_theta0_r) {
    CKR(resto_merit(S, S->P.x, S->P.s, S->rp, S->rq, S->P.geq, S->P.hin, S->mu_r, &theta, &phi));
    S->theta_max_r = 1e4 * std::max(1.0, theta);
    S->theta_min_r = 1e-4 * std::max(1.0, theta);
    S->have_theta0_r = true;
  }
  info->kkt_err = e0;
  // a stationary point of the restoration problem reached before the return test passed: a
  // local minimizer of the constraint violation, unless that violation is within the tolerance
  // (a feasible point that the filter still rejects)
  if (e0 <= S->opt.tol) return S->rs_cinf > S->opt.tol ? IPM_ERR_INFEASIBLE : IPM_ERR_RESTORATION;
  bool first = true;
  while (true) {
    double emu;
    CKR(resto_errors(S, S->mu_r, &emu));
    if (!(emu <= KAPPA_EPS * S->mu_r && (first || S->k_r == 0))) break;
    S->mu_r = std::max(S->opt.tol / 10.0, std::min(KAPPA_MU * S->mu_r, std::pow(S->mu_r, THETA_MU)));
    S->tau_r = std::max(TAU_MIN, 1.0 - S->mu_r);
    S->filter_r.clear();
    first = false;
  }
  info->mu = S->mu_r;
  // Hessian of the constraints' Lagrangian only (the restoration objective is quadratic in x
  // with its Hessian zeta D_R^2 on the diagonal, added to sigma)
  k_mul<<<grid1(m), 256, 0, s>>>(m, S->lam, S->dscale, S->lamw);
  CKL();
  CKR(opf_eval(M, S->P.x, S->lamw, S->lamw + D.me0, 0.0, S->ft, nullptr, S->gst, S->hst, nullptr,
               S->Wv, s));
  k_resto_rhs<<<grid1(nr), 256, 0, s>>>(rargs(S, 0.0));
  k_neg<<<grid1(n), 256, 0, s>>>(n, S->r1, S->a);
  CKL();
  // inertia correction as in the main iterations
  double dw = 0.0;
  bool ok = false;
  int nfac = 0;
  const double grow = S->delta_last_r > 0 ? 8.0 : 100.0;
  double next = S->delta_last_r > 0 ? std::max(1e-20, S->delta_last_r / 3.0) : 1e-4;
  for (int attempt = 0; attempt < 200; ++attempt) {
    dw = attempt == 0 ? 0.0 : next;
    if (attempt > 0) next *= grow;
    if (dw >= 1e40) break;
    k_resto_aug<<<grid1(m), 256, 0, s>>>(rargs(S, dw), S->dcond, S->baug);
    CKL();
    CKR(ipm_condense(S->sym, S->num, S->Wv, S->sigma, S->Jv, S->dcond, dw, s));
    CKR(ipm_factor(S->sym, S->num, S->info, s));
    int hinfo = 0;
    CK(cudaMemcpyAsync(&hinfo, S->info, sizeof(int), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    ++nfac;
    if (hinfo == -2) return IPM_ERR_TIMEOUT;
    if (hinfo != -1) continue;
    const int st = ipm_aug_solve(S->sym, S->num, S->Wv, S->sigma, S->Jv, S->dcond, dw, S->a,
                                 S->baug, S->dx, S->dzc, S->opt.max_refine, 1e-10, S->eta,
                                 S->steps, s);
    if (st < 0 || st == IPM_ERR_TIMEOUT || st == IPM_ERR_NONFINITE) return st;
    if (st == IPM_ERR_NOT_PD) continue;
    ok = true;
    break;
  }
  if (!ok) return IPM_ERR_INERTIA;
  S->have_kkt = true;
  S->kkt_resto = true;
  S->last_dw = dw;
  if (dw > 0) S->delta_last_r = dw;
  info->delta_w = dw;
  info->n_factor = nfac;
  CK(cudaMemcpyAsync(&info->eta, S->eta, sizeof(double), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  k_jv<<<grid1(m), 256, 0, s>>>(m, M.J_rowptr, M.J_colind, S->Jv, S->dx, S->jdx);
  k_resto_recover<<<grid1(nr), 256, 0, s>>>(rargs(S, dw));
  CKL();
  // fraction to the boundary, d phi_R, theta_R and phi_R at the iterate
  CKR(reduce_reset(S, {R_AMAX, R_AZ}, 1.0));
  CKR(reduce_reset(S, {R_GPHI_X}, 0.0));
  k_resto_ftb<<<grid1(nr), 256, 0, s>>>(rargs(S, dw), S->tau_r, S->R);
  CKL();
  CKR(read_R(S));
  const double amax = S->hR[R_AMAX], az = S->hR[R_AZ], gphi = S->hR[R_GPHI_X];
  CKR(resto_merit(S, S->P.x, S->P.s, S->rp, S->rq, S->P.geq, S->P.hin, S->mu_r, &theta, &phi));
  double amin;
  if (gphi < 0)
    amin = GAMMA_ALPHA * std::min({GAMMA_THETA, GAMMA_PHI * theta / -gphi,
                                   DELTA_SW * std::pow(theta, S_THETA) / std::pow(-gphi, S_PHI)});
  else
    amin = GAMMA_ALPHA * GAMMA_THETA;
  double alpha = amax;
  bool accepted = false;
  int ft = 0, ls = 0;
  while (true) {
    k_resto_trial<<<grid1(nr), 256, 0, s>>>(rargs(S, dw), alpha, S->xt, S->st, S->rpt, S->rqt);
    CKL();
    CKR(eval_point(S, S->xt, S->gst, S->hst, S->geqt, S->hint, S->ft, false));
    double tht, pht;
    CKR(resto_merit(S, S->xt, S->st, S->rpt, S->rqt, S->geqt, S->hint, S->mu_r, &tht, &pht));
    accepted = filter_accept(theta, phi, gphi, alpha, tht, pht, S->filter_r.data(),
                             (int)(S->filter_r.size() / 2), S->theta_min_r, S->theta_max_r, &ft);
    if (accepted) break;
    ++ls;
    alpha *= 0.5;
    if (alpha < amin) break;
  }
  info->ls_steps = ls;
  info->alpha = alpha;
  info->theta = theta;
  if (!accepted) return IPM_ERR_RESTORATION;
  if (!ft) {
    S->filter_r.push_back((1 - GAMMA_THETA) * theta);
    S->filter_r.push_back(phi - GAMMA_PHI * theta);
  }
  RArgs A = rargs(S, dw);
  k_resto_accept<<<grid1(nr), 256, 0, s>>>(A, alpha, az, S->xt, S->st, S->rpt, S->rqt);
  CKL();
  S->k_r++;
  // return test: the original violation reduced to KAPPA_RESTO times the phase's start and the
  // point acceptable to the original filter (with the start's entry)
  CKR(eval_point(S, S->P.x, S->gs, S->hs, S->P.geq, S->P.hin, S->f, false));
  double th0, ph0;
  CKR(merit(S, S->P.x, S->P.s, S->P.geq, S->P.hin, S->f, S->mu, &th0, &ph0));
  bool back = th0 <= KAPPA_RESTO * S->theta_start && th0 < S->theta_max &&
              (th0 < S->entry_theta || ph0 < S->entry_phi);
  for (size_t q = 0; back && q + 1 < S->filter.size(); q += 2)
    if (!(th0 < S->filter[q] || ph0 < S->filter[q + 1])) back = false;
  if (back) {
    k_resto_finish<<<grid1(nr), 256, 0, s>>>(D, S->P);
    CKL();
    S->filter.push_back(S->entry_theta);
    S->filter.push_back(S->entry_phi);
    S->in_resto = false;
  }
  CK(cudaStreamSynchronize(s));
  return IPM_OK;
}

static int step_impl(ipm_state_t S, ipm_iter_info *info) {
  cudaStream_t s = S->stream;
  const Dims &D = S->D;
  const OpfData &M = S->opf->M;
  const int n = D.n, m = D.me0 + D.mi0;
  const int nmax = std::max({D.n, D.me, D.mi, m});
  *info = ipm_iter_info{};
  info->k = S->k;
  // ---- evaluate at the current iterate
  CKR(eval_point(S, S->P.x, S->gs, S->hs, S->P.geq, S->P.hin, S->f, true));
  CKR(jt_lambda(S));
  double e0;
  CKR(errors(S, 0.0, &e0));
  double theta, phi;
  if (!S->have_theta0) {
    CKR(merit(S, S->P.x, S->P.s, S->P.geq, S->P.hin, S->f, S->mu, &theta, &phi));
    S->theta_max = 1e4 * std::max(1.0, theta);
    S->theta_min = 1e-4 * std::max(1.0, theta);
    S->have_theta0 = true;
  }
  double fval = 0.0;
  CK(cudaMemcpyAsync(&fval, S->f, sizeof(double), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  info->kkt_err = e0;
  info->obj = fval;
  info->mu = S->mu;
  if (e0 <= S->opt.tol) {
    S->status = 1;
    info->status = 1;
    return IPM_OK;
  }
  // ---- barrier update (repeated only in the first iteration)
  bool first = true;
  while (true) {
    double emu;
    CKR(errors(S, S->mu, &emu));
    if (!(emu <= KAPPA_EPS * S->mu && (first || S->k == 0))) break;
    S->mu = std::max(S->opt.tol / 10.0, std::min(KAPPA_MU * S->mu, std::pow(S->mu, THETA_MU)));
    S->tau = std::max(TAU_MIN, 1.0 - S->mu);
    S->filter.clear();
    first = false;
  }
  const double mu = S->mu;
  info->mu = mu;
  // ---- Hessian with scaled multipliers, Newton right-hand sides
  k_mul<<<grid1(m), 256, 0, s>>>(m, S->lam, S->dscale, S->lamw);
  CKL();
  CKR(opf_eval(M, S->P.x, S->lamw, S->lamw + D.me0, S->sig, S->ft, nullptr, S->gst, S->hst,
               nullptr, S->Wv, s));
  k_newton_rhs<<<grid1(nmax), 256, 0, s>>>(D, S->P, S->sig, mu, S->sigma, S->r1, S->r2, S->r4,
                                           S->Ds);
  k_neg<<<grid1(n), 256, 0, s>>>(n, S->r1, S->a);
  CKL();
  // ---- inertia correction: delta_w = 0, then delta_last/3 (x8) or 1e-4 (x100).  A failed
  // factorization, or (FP32 factor) a solve whose FP64 refinement meets negative curvature or
  // does not converge, counts as wrong inertia.
  // gamma: the option, or (<= 0) ||K|| / ||G||^2 of this iteration (Golub & Greif, Sec. 3.1)
  double gamma = S->opt.gamma;
  if (!D.lifted && !(gamma > 0)) {
    CKR(reduce_reset(S, {R_PD, R_QD}, 0.0));
    k_gamma_norms<<<grid1(n), 256, 0, s>>>(D, M.W_rowptr, M.W_colind, S->sym->W_rowidx,
                                           S->sym->WT_ptr, S->sym->WT_ent, S->Wv, S->sigma,
                                           S->sym->JT_ptr, S->sym->JT_ent, S->sym->J_rowidx,
                                           M.J_rowptr, S->Jv, S->Ds, S->R, R_PD, R_QD);
    CKL();
    CKR(read_R(S));
    const double gn = S->hR[R_QD];
    gamma = gn > 0 ? S->hR[R_PD] / (gn * gn) : 1.0;
  }
  info->gamma = gamma;
  double dw = 0.0;
  int nfac = 0;
  bool ok = false;
  double grow = S->delta_last > 0 ? 8.0 : 100.0;
  double next = S->delta_last > 0 ? std::max(1e-20, S->delta_last / 3.0) : 1e-4;
  StepArgs SA;
  SA.D = D;
  SA.P = S->P;
  SA.mu = mu;
  SA.r2 = S->r2;
  SA.r4 = S->r4;
  SA.Ds = S->Ds;
  SA.jdx = S->jdx;
  SA.dx = S->dx;
  SA.sigma = S->sigma;
  SA.dzH = S->dzH;
  SA.dz = S->dz;
  SA.ds = S->ds;
  SA.dv = S->dv;
  SA.dzl = S->dzl;
  SA.dzu = S->dzu;
  // a line search that fails at a point feasible within the tolerance sends the iteration back
  // here with the schedule continued from its next candidate (resume), at most
  // MAX_LS_REGULARIZE times
  int n_reg = 0;
  bool resume = false;
retry_solve:
  ok = false;
  for (int attempt = resume ? 1 : 0; attempt < 200; ++attempt) {
    dw = attempt == 0 ? 0.0 : next;
    if (attempt > 0) next *= grow;
    if (dw >= 1e40) break;
    ipm_num_t num = S->num32 ? S->num32 : S->num;
    k_aug_rhs<<<grid1(std::max(D.me0, D.mi0)), 256, 0, s>>>(D, dw, gamma, S->r2, S->r4,
                                                            S->Ds, S->P.geq, S->dcond, S->baug);
    CKL();
    CKR(ipm_condense(S->sym, num, S->Wv, S->sigma, S->Jv, S->dcond, dw, s));
    CKR(ipm_factor(S->sym, num, S->info, s));
    int hinfo = 0;
    CK(cudaMemcpyAsync(&hinfo, S->info, sizeof(int), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    ++nfac;
    if (hinfo == -2) return IPM_ERR_TIMEOUT;
    if (hinfo != -1) continue;
    // ---- solve
    int st;
    if (S->opt.kkt != 1) {
      // LiftedKKT, or the dual-regularized form (delta_c = 1/gamma, Remark in Sec. 3): one
      // condensed solve refined on the augmented system whose equality block is -delta_c I
      st = ipm_aug_solve(S->sym, num, S->Wv, S->sigma, S->Jv, S->dcond, dw, S->a, S->baug,
                         S->dx, S->dzc, S->opt.max_refine, 1e-10, S->eta, S->steps, s);
    } else {
      int its = 0;
      double rel = 0;
      st = hykkt_cg(S->sym, num, D.me0, S->Jv, S->dcond, gamma, S->a, S->baug,
                    S->opt.cg_rtol, S->opt.cg_maxit > 0 ? S->opt.cg_maxit : std::max(D.me0, 1),
                    S->dx, S->dy, S->dzH, &its, &rel, s);
      info->cg_iters = its;
    }
    if (st < 0 || st == IPM_ERR_TIMEOUT || st == IPM_ERR_NONFINITE) return st;
    if (st == IPM_ERR_NOT_PD && num == S->num32) {
      // the FP32 factor no longer preconditions K to FP64 accuracy: FP64 factor from now on,
      // redoing this inertia search from delta_w = 0
      ipm_num_destroy(S->num32);
      S->num32 = nullptr;
      attempt = -1;
      next = S->delta_last > 0 ? std::max(1e-20, S->delta_last / 3.0) : 1e-4;
      continue;
    }
    if (st == IPM_ERR_NOT_PD) continue;
    ok = true;
    info->precision = num == S->num32 ? 32 : 64;
    if (S->opt.kkt == 1) info->eta = num->last_eta;
    info->pcg_iters = num->last_pcg_iters;
    break;
  }
  if (!ok) return IPM_ERR_INERTIA;
  S->have_kkt = true;
  S->kkt_resto = false;
  S->last_dw = dw;
  if (dw > 0) S->delta_last = dw;
  info->delta_w = dw;
  info->n_factor = nfac;
  SA.dw = dw;
  const double *dy_step = S->dy;
  if (S->opt.kkt == 2) {  // dy = dz over the G rows, dz over the H rows
    SA.dzH = S->dzc + D.me0;
    dy_step = S->dzc;
  }
  if (S->opt.kkt != 1) {
    double eta = 0;
    int steps = 0;
    CK(cudaMemcpyAsync(&eta, S->eta, sizeof(double), cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(&steps, S->steps, sizeof(int), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    info->eta = eta;
    info->refine_steps = steps;
    if (D.lifted) {
      k_jv<<<grid1(m), 256, 0, s>>>(m, M.J_rowptr, M.J_colind, S->Jv, S->dx, S->jdx);
      CKL();
    }
  }
  k_recover<<<grid1(nmax), 256, 0, s>>>(SA);
  CKL();
  // ---- fraction to the boundary and d phi
  CKR(reduce_reset(S, {R_AMAX, R_AZ}, 1.0));
  CKR(reduce_reset(S, {R_GPHI_X, R_GPHI_S}, 0.0));
  k_ftb<<<grid1(nmax), 256, 0, s>>>(SA, S->tau, S->sig, S->R);
  CKL();
  CKR(read_R(S));
  const double amax = S->hR[R_AMAX], az = S->hR[R_AZ];
  const double gphi = S->hR[R_GPHI_X] + S->hR[R_GPHI_S];
  CKR(merit(S, S->P.x, S->P.s, S->P.geq, S->P.hin, S->f, mu, &theta, &phi));
  double amin;
  if (gphi < 0)
    amin = GAMMA_ALPHA * std::min({GAMMA_THETA, GAMMA_PHI * theta / -gphi,
                                   DELTA_SW * std::pow(theta, S_THETA) / std::pow(-gphi, S_PHI)});
  else
    amin = GAMMA_ALPHA * GAMMA_THETA;
  // ---- backtracking filter line search
  double alpha = amax;
  bool accepted = false, ftype = false;
  int ls = 0;
  while (true) {
    k_trial<<<grid1(std::max(n, D.mi)), 256, 0, s>>>(n, D.mi, alpha, S->P.x, S->dx, S->P.s, S->ds,
                                                     S->xt, S->st);
    CKL();
    CKR(eval_point(S, S->xt, S->gst, S->hst, S->geqt, S->hint, S->ft, false));
    double tht, pht;
    CKR(merit(S, S->xt, S->st, S->geqt, S->hint, S->ft, mu, &tht, &pht));
    int ft = 0;
    accepted = filter_accept(theta, phi, gphi, alpha, tht, pht, S->filter.data(),
                             (int)(S->filter.size() / 2), S->theta_min, S->theta_max, &ft);
    ftype = ft != 0;
    if (accepted) break;
    ++ls;
    alpha *= 0.5;
    if (alpha < amin) break;
  }
  info->ls_steps = ls;
  info->alpha = alpha;
  info->theta = theta;
  if (!accepted) {
    // no restoration phase at a point already feasible within the tolerance: it cannot reduce
    // a violation at rounding level; the direction is recomputed with the next delta_w of this
    // iteration's inertia-correction schedule (a better conditioned, more gradient-like step)
    // at most MAX_LS_REGULARIZE times before the method stops there
    if (!S->opt.no_resto && S->prim_inf <= S->opt.tol && n_reg < MAX_LS_REGULARIZE) {
      ++n_reg;
      resume = true;
      goto retry_solve;
    }
    if (S->opt.no_resto || S->prim_inf <= S->opt.tol) return IPM_ERR_RESTORATION;
    // feasibility restoration (Waechter & Biegler 2006, Sec. 3.3): the following calls iterate
    // on the restoration problem until its return test passes
    CKR(resto_begin(S, theta, phi));
    info->resto = 2;
    S->k++;
    return IPM_OK;
  }
  if (!ftype) {
    S->filter.push_back((1 - GAMMA_THETA) * theta);
    S->filter.push_back(phi - GAMMA_PHI * theta);
  }
  k_accept<<<grid1(nmax), 256, 0, s>>>(SA, alpha, az, S->xt, S->st, dy_step);
  CKL();
  CK(cudaStreamSynchronize(s));
  S->k++;
  return IPM_OK;
}

extern "C" int ipm_step(ipm_state_t S, ipm_iter_info *info) {
  NvtxRange nvtx_range("ipm_step");
  if (!S || !info) return IPM_ERR_BAD_ARG;
  if (S->status != 0) {
    *info = ipm_iter_info{};
    info->k = S->k;
    info->status = S->status;
    return IPM_OK;
  }
  int rc;
  if (S->in_resto) {
    *info = ipm_iter_info{};
    info->k = S->k;
    rc = resto_step(S, info);
  } else {
    rc = step_impl(S, info);
  }
  if (rc != IPM_OK) {
    S->status = rc;
    info->status = rc;
  }
  return rc < 0 ? rc : IPM_OK;
}

extern "C" int ipm_state_export(ipm_state_t S, double *x, double *obj) {
  if (!S) return IPM_ERR_BAD_ARG;
  if (x) {
    CK(cudaMemcpyAsync(x, S->P.x, sizeof(double) * S->D.n, cudaMemcpyDeviceToHost, S->stream));
    CK(cudaStreamSynchronize(S->stream));
  }
  if (obj) {
    CKR(opf_eval(S->opf->M, S->P.x, nullptr, nullptr, 1.0, S->ft, nullptr, S->gst, S->hst,
                 nullptr, nullptr, S->stream));
    CK(cudaMemcpyAsync(obj, S->ft, sizeof(double), cudaMemcpyDeviceToHost, S->stream));
    CK(cudaStreamSynchronize(S->stream));
  }
  return IPM_OK;
}

// ---- checkpoint / resume: the iterate and the host-side algorithm state in one flat host
// buffer of doubles: a header (format tag, version, sizes, scalars, filter length), the filter
// entries, then x, s, y, z, v, zl, zu and the row scaling
static constexpr double STATE_TAG = 2405.14236;
static constexpr int STATE_HEAD = 18;

static int64_t state_len(const ipm_state_t S) {
  const Dims &D = S->D;
  return STATE_HEAD + (int64_t)S->filter.size() + 3 * (int64_t)D.n + 3 * (int64_t)D.mi + D.me +
         D.me0 + D.mi0;
}

extern "C" int ipm_state_save(ipm_state_t S, double *buf, int64_t cap, int64_t *len) {
  if (!S || !len) return IPM_ERR_BAD_ARG;
  if (S->in_resto) {
    set_error_msg("ipm_state_save: the state is in the restoration phase (save between main "
                  "iterations)");
    return IPM_ERR_BAD_ARG;
  }
  const int64_t need = state_len(S);
  *len = need;
  if (!buf) return IPM_OK;
  if (cap < need) {
    set_error_msg("ipm_state_save: buffer too small");
    return IPM_ERR_BAD_ARG;
  }
  const Dims &D = S->D;
  const double head[STATE_HEAD] = {STATE_TAG, 1.0, (double)D.n, (double)D.me, (double)D.mi,
                                   (double)(D.me0 + D.mi0), S->sig, S->mu, S->tau, S->delta_last,
                                   S->theta_max, S->theta_min, S->have_theta0 ? 1.0 : 0.0,
                                   (double)S->k, (double)S->status, S->num32 ? 1.0 : 0.0,
                                   S->prim_inf, (double)S->filter.size()};
  std::copy(head, head + STATE_HEAD, buf);
  double *o = buf + STATE_HEAD;
  std::copy(S->filter.begin(), S->filter.end(), o);
  o += S->filter.size();
  CK(cudaStreamSynchronize(S->stream));
  const std::pair<const double *, int64_t> parts[] = {
      {S->P.x, D.n}, {S->P.s, D.mi}, {S->P.y, D.me}, {S->P.z, D.mi}, {S->P.v, D.mi},
      {S->P.zl, D.n}, {S->P.zu, D.n}, {S->dscale, D.me0 + D.mi0}};
  for (const auto &pt : parts) {
    if (pt.second > 0)
      CK(cudaMemcpy(o, pt.first, sizeof(double) * pt.second, cudaMemcpyDeviceToHost));
    o += pt.second;
  }
  return IPM_OK;
}

extern "C" int ipm_state_load(ipm_state_t S, const double *buf, int64_t len) {
  if (!S || !buf || len < STATE_HEAD) return IPM_ERR_BAD_ARG;
  const Dims &D = S->D;
  if (buf[0] != STATE_TAG || buf[1] != 1.0 || buf[2] != D.n || buf[3] != D.me ||
      buf[4] != D.mi || buf[5] != D.me0 + D.mi0 || !(buf[17] >= 0) ||
      len != STATE_HEAD + (int64_t)buf[17] + 3 * (int64_t)D.n + 3 * (int64_t)D.mi + D.me +
                 D.me0 + D.mi0) {
    set_error_msg("ipm_state_load: not a saved state of this model and formulation");
    return IPM_ERR_BAD_ARG;
  }
  S->sig = buf[6];
  S->mu = buf[7];
  S->tau = buf[8];
  S->delta_last = buf[9];
  S->theta_max = buf[10];
  S->theta_min = buf[11];
  S->have_theta0 = buf[12] != 0.0;
  S->k = (int)buf[13];
  S->status = (int)buf[14];
  S->prim_inf = buf[16];
  const int64_t nf = (int64_t)buf[17];
  S->filter.assign(buf + STATE_HEAD, buf + STATE_HEAD + nf);
  const double *o = buf + STATE_HEAD + nf;
  const std::pair<double *, int64_t> parts[] = {
      {S->P.x, D.n}, {S->P.s, D.mi}, {S->P.y, D.me}, {S->P.z, D.mi}, {S->P.v, D.mi},
      {S->P.zl, D.n}, {S->P.zu, D.n}, {S->dscale, D.me0 + D.mi0}};
  CK(cudaStreamSynchronize(S->stream));
  for (const auto &pt : parts) {
    if (pt.second > 0)
      CK(cudaMemcpyAsync(pt.first, o, sizeof(double) * pt.second, cudaMemcpyHostToDevice,
                         S->stream));
    o += pt.second;
  }
  CK(cudaStreamSynchronize(S->stream));
  // a state saved after its FP32 factor had stopped serving goes on in FP64
  if (buf[15] == 0.0 && S->num32) {
    ipm_num_destroy(S->num32);
    S->num32 = nullptr;
  }
  S->in_resto = false;
  S->have_kkt = false;
  return IPM_OK;
}

extern "C" int ipm_state_export_kkt(ipm_state_t S, double *W_val, double *sigma, double *J_val,
                                    double *d_row, double *delta_w, double *a, double *b,
                                    double *dx, double *dyz, int *m_e) {
  if (!S || !S->have_kkt) {
    set_error_msg("ipm_state_export_kkt: no KKT solve has completed");
    return IPM_ERR_BAD_ARG;
  }
  const int n = S->D.n, me0 = S->D.me0, mi0 = S->D.mi0, m = me0 + mi0;
  CK(cudaStreamSynchronize(S->stream));
  auto get = [&](double *dst, const double *src, int64_t count) -> int {
    if (dst && count > 0)
      CK(cudaMemcpy(dst, src, sizeof(double) * count, cudaMemcpyDeviceToHost));
    return IPM_OK;
  };
  CKR(get(W_val, S->Wv, S->nnzW));
  CKR(get(sigma, S->sigma, n));
  CKR(get(J_val, S->Jv, S->nnzJ));
  CKR(get(d_row, S->dcond, m));
  CKR(get(a, S->a, n));
  CKR(get(b, S->baug, m));
  CKR(get(dx, S->dx, n));
  const bool kept_eq = S->opt.kkt == 1 && !S->kkt_resto;
  if (kept_eq) {
    CKR(get(dyz, S->dy, me0));
    CKR(get(dyz ? dyz + me0 : nullptr, S->dzH, mi0));
  } else {
    CKR(get(dyz, S->dzc, m));
  }
  if (delta_w) *delta_w = S->last_dw;
  if (m_e) *m_e = kept_eq ? me0 : 0;
  return IPM_OK;
}
