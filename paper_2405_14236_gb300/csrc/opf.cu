// AC optimal power flow model on the GPU: sparsity patterns of J = [G; H] and of the lower
// triangle of W, and the evaluation of f, grad f, g, h, J and W = sigma_f grad^2 f +
// sum y grad^2 g + sum z grad^2 h (the "AD" part of each IPM iteration, Section 5,
// "Evaluation of the nonlinear models", written here as hand-derived derivative kernels).
//
// Layout: x = [V (nb) | theta (nb) | Pg (ng) | Qg (ng)];
// g = [P balance (nb) | Q balance (nb) | theta_ref]; h = [|S_from|^2 - rate^2 | |S_to|^2 - rate^2].
// Branch pi-model: series 1/(r + j x), shunt j b/2 per end, unit tap.  Cost on MW (base 100).
#include <climits>
#include <cmath>
#include <vector>

#include "internal.cuh"
#include "opf.cuh"
#include "opf_dev.cuh"

namespace cipm {

static constexpr int SORT_CAP2 = 1024;

// --- pattern construction: every model term lists its (row, col) coordinates in a fixed
// order; rows are then sorted/uniqued and each term records the entry it writes.
// J terms: per gen 2, per branch end 12 (compact: 4 P-balance, 4 Q-balance, 4 thermal) or 14
// (flow form: balance P and Q, p and q definitions with 5 each, thermal 2), theta_ref 1
__host__ __device__ __forceinline__ int jterm_count(const OpfDims &D) {
  return 2 * D.ng + 2 * jterms_per_end(D) * D.nbr + 1;
}
// W terms: per gen 1, per branch end 10 (lower 4x4 block) or 12 (plus p_end, q_end diagonals)
__host__ __device__ __forceinline__ int wterm_count(const OpfDims &D) {
  return D.ng + 2 * wterms_per_end(D) * D.nbr;
}

__device__ __forceinline__ void jterm(const OpfDims &D, const int *f_bus, const int *t_bus,
                                      const int *gen_bus, int ref, int t, int *row, int *col) {
  if (t < 2 * D.ng) {
    int g = t >> 1;
    if ((t & 1) == 0) {
      *row = gen_bus[g];
      *col = 2 * D.nb + g;
    } else {
      *row = D.nb + gen_bus[g];
      *col = 2 * D.nb + D.ng + g;
    }
    return;
  }
  t -= 2 * D.ng;
  if (D.form && t < 28 * D.nbr) {
    const int e = t / 14, k = t % 14;
    int bus, v[4];
    end_vars(D, f_bus, t_bus, e, &bus, v);
    const int pv = flow_pvar(D, e), qv = flow_qvar(D, e);
    const int rp = flow_prow(D, e), rq = flow_qrow(D, e);
    if (k == 0) { *row = bus; *col = pv; }
    else if (k == 1) { *row = D.nb + bus; *col = qv; }
    else if (k == 2) { *row = rp; *col = pv; }
    else if (k < 7) { *row = rp; *col = v[k - 3]; }
    else if (k == 7) { *row = rq; *col = qv; }
    else if (k < 12) { *row = rq; *col = v[k - 8]; }
    else { *row = D.me + e; *col = k == 12 ? pv : qv; }
    return;
  }
  if (!D.form && t < 24 * D.nbr) {
    int e = t / 12, k = t % 12;
    int bus, v[4];
    end_vars(D, f_bus, t_bus, e, &bus, v);
    int which = k >> 2, c = k & 3;
    *col = v[c];
    if (which == 0) *row = bus;
    else if (which == 1) *row = D.nb + bus;
    else *row = D.me + e;  // thermal row of this end
    return;
  }
  *row = 2 * D.nb;
  *col = D.nb + ref;
}

__device__ __forceinline__ void wterm(const OpfDims &D, const int *f_bus, const int *t_bus, int t,
                                      int *row, int *col) {
  if (t < D.ng) {
    *row = *col = 2 * D.nb + t;
    return;
  }
  t -= D.ng;
  const int per = wterms_per_end(D);
  int e = t / per, k = t % per;
  if (k >= 10) {  // flow form: (p_end, p_end), (q_end, q_end)
    *row = *col = k == 10 ? flow_pvar(D, e) : flow_qvar(D, e);
    return;
  }
  int bus, v[4];
  end_vars(D, f_bus, t_bus, e, &bus, v);
  int a = v[c_lowpairs[k][0]], b = v[c_lowpairs[k][1]];
  *row = max(a, b);
  *col = min(a, b);
}

template <bool IsJ>
__global__ void k_terms(OpfDims D, const int *f_bus, const int *t_bus, const int *gen_bus,
                        int ref, int *trow, int *tcol, int *rowcnt) {
  int nt = IsJ ? jterm_count(D) : wterm_count(D);
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nt) return;
  int r, c;
  if (IsJ) jterm(D, f_bus, t_bus, gen_bus, ref, t, &r, &c);
  else wterm(D, f_bus, t_bus, t, &r, &c);
  trow[t] = r;
  tcol[t] = c;
  atomicAdd(&rowcnt[r], 1);
}

__global__ void k_terms_fill(int nt, const int *trow, const int *tcol, const int *ptr, int *fill,
                             int *cand) {
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nt) return;
  int r = trow[t];
  cand[ptr[r] + atomicAdd(&fill[r], 1)] = tcol[t];
}

__global__ void k_row_unique(int nrows, const int *ptr, int *cand, int *ucnt) {
  __shared__ int smem[SORT_CAP2 + 1];
  int r = blockIdx.x;
  if (r >= nrows) return;
  int b = ptr[r], len = ptr[r + 1] - b;
  int u = block_sort_unique(cand + b, len, smem, SORT_CAP2, INT_MIN);
  if (threadIdx.x == 0) ucnt[r] = u;
}

__global__ void k_row_compact(int nrows, const int *ptr, const int *cand, const int *rowptr,
                              int *colind) {
  int r = blockIdx.x;
  if (r >= nrows) return;
  int len = rowptr[r + 1] - rowptr[r];
  for (int k = threadIdx.x; k < len; k += blockDim.x) colind[rowptr[r] + k] = cand[ptr[r] + k];
}

__global__ void k_term_entry(int nt, const int *trow, const int *tcol, const int *rowptr,
                             const int *colind, int *entry) {
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nt) return;
  int r = trow[t], c = tcol[t];
  int lo = rowptr[r], hi = rowptr[r + 1] - 1;
  while (lo < hi) {
    int mid = (lo + hi) >> 1;
    if (colind[mid] < c) lo = mid + 1; else hi = mid;
  }
  entry[t] = lo;
}

static int build_pattern(bool isJ, const OpfDims &D, const OpfData &M, int nrows, int **rowptr,
                         int **colind, int **entry, int *nnz, cudaStream_t s) {
  DevTemp T;
  int nt = isJ ? jterm_count(D) : wterm_count(D);
  int *trow, *tcol, *cnt, *ptr, *fill, *cand, *ucnt;
  CKR(T.alloc(&trow, nt));
  CKR(T.alloc(&tcol, nt));
  CKR(T.alloc(&cnt, nrows + 1));
  CKR(T.alloc(&ptr, nrows + 1));
  CKR(T.alloc(&fill, nrows + 1));
  CKR(T.alloc(&cand, nt));
  CKR(T.alloc(&ucnt, nrows + 1));
  CK(cudaMemsetAsync(cnt, 0, sizeof(int) * (nrows + 1), s));
  CK(cudaMemsetAsync(fill, 0, sizeof(int) * (nrows + 1), s));
  if (isJ)
    k_terms<true><<<grid_for(nt, 256), 256, 0, s>>>(D, M.f_bus, M.t_bus, M.gen_bus, M.ref, trow,
                                                    tcol, cnt);
  else
    k_terms<false><<<grid_for(nt, 256), 256, 0, s>>>(D, M.f_bus, M.t_bus, M.gen_bus, M.ref, trow,
                                                     tcol, cnt);
  CKL();
  CKR(exclusive_scan_i32(cnt, ptr, nrows, s));
  k_terms_fill<<<grid_for(nt, 256), 256, 0, s>>>(nt, trow, tcol, ptr, fill, cand);
  CKL();
  k_row_unique<<<nrows, 64, 0, s>>>(nrows, ptr, cand, ucnt);
  CKL();
  CKR(dev_alloc(rowptr, nrows + 1));
  CKR(exclusive_scan_i32(ucnt, *rowptr, nrows, s));
  CK(cudaMemcpyAsync(nnz, *rowptr + nrows, sizeof(int), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  CKR(dev_alloc(colind, *nnz));
  k_row_compact<<<nrows, 64, 0, s>>>(nrows, ptr, cand, *rowptr, *colind);
  CKL();
  CKR(dev_alloc(entry, nt));
  k_term_entry<<<grid_for(nt, 256), 256, 0, s>>>(nt, trow, tcol, *rowptr, *colind, *entry);
  CKL();
  CK(cudaStreamSynchronize(s));
  return IPM_OK;
}

// --- evaluation
__global__ void k_branch_admittance(int nbr, const double *r, const double *x, const double *b,
                                    double4_32a *adm) {
  int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= nbr) return;
  double den = r[k] * r[k] + x[k] * x[k];
  double gs = r[k] / den, bs = -x[k] / den;
  adm[k] = make_double4_32a(gs, bs + 0.5 * b[k], -gs, -bs);  // G1, B1, G2, B2 (both ends)
}

__global__ void k_eval_init(OpfDims D, const double *pd, const double *qd, const double *x,
                            int ref, double *g, double *Jv, int nnzJ, double *Wv, int nnzW) {
  eval_init_at(D, pd, qd, x, ref, g, Jv, nnzJ, Wv, nnzW, blockIdx.x * blockDim.x + threadIdx.x,
               gridDim.x * blockDim.x);
}

// one thread per branch end
__global__ void k_eval_branch(OpfDims D, OpfData M, const double *x, const double *y,
                              const double *z, double *g, double *h, double *Jv, double *Wv) {
  int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e < 2 * D.nbr) eval_branch_at(D, M, x, y, z, g, h, Jv, Wv, e);
}

__global__ void k_eval_gen(OpfDims D, OpfData M, const double *x, double sigma_f, double *g,
                           double *grad, double *Jv, double *Wv, double *fpart) {
  __shared__ double sh[32];
  int gi = blockIdx.x * blockDim.x + threadIdx.x;
  double fc = gi < D.ng ? eval_gen_at(D, M, x, sigma_f, g, grad, Jv, Wv, gi) : 0.0;
  block_sum_to(fpart + blockIdx.x, fc, sh);
}

__global__ void k_eval_finish(OpfDims D, OpfData M, const double *fpart, int nparts, double *f,
                              double *grad, double *Jv) {
  eval_finish_at(D, M, fpart, nparts, f, grad, Jv, blockIdx.x * blockDim.x + threadIdx.x,
                 gridDim.x * blockDim.x);
}

int opf_eval(const OpfData &M, const double *x, const double *y, const double *z, double sigma_f,
             double *f, double *grad, double *g, double *h, double *Jv, double *Wv,
             cudaStream_t s) {
  OpfDims D{M.nb, M.nbr, M.ng, M.n, M.me, M.mi, M.form};
  int nthreads = max(max(D.nb, 1), 256);
  k_eval_init<<<grid_for(nthreads, 256), 256, 0, s>>>(D, M.pd, M.qd, x, M.ref, g, Jv,
                                                      Jv ? M.nnzJ : 0, Wv, Wv ? M.nnzW : 0);
  CKL();
  if (D.nbr > 0) {
    k_eval_branch<<<grid_for(2 * D.nbr, 128), 128, 0, s>>>(D, M, x, y, z, g, h, Jv, Wv);
    CKL();
  }
  int gb = grid_for(max(D.ng, 1), 256);
  k_eval_gen<<<gb, 256, 0, s>>>(D, M, x, sigma_f, g, grad, Jv, Wv, M.fpart);
  CKL();
  k_eval_finish<<<grid_for(max(2 * D.nb, 1), 256), 256, 0, s>>>(D, M, M.fpart, gb, f, grad, Jv);
  CKL();
  return IPM_OK;
}

__global__ void k_flow_start(OpfDims D, OpfData M, double *x) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e < 2 * D.nbr) flow_start_at(D, M, x, e);
}

int opf_flow_start(const OpfData &M, double *x, cudaStream_t s) {
  if (!M.form || M.nbr == 0) return IPM_OK;
  OpfDims D{M.nb, M.nbr, M.ng, M.n, M.me, M.mi, M.form};
  k_flow_start<<<grid_for(2 * M.nbr, 128), 128, 0, s>>>(D, M, x);
  CKL();
  return IPM_OK;
}

void opf_free(OpfData &M) {
  void *ps[] = {M.f_bus, M.t_bus, M.gen_bus, M.adm, M.rate, M.pd, M.qd, M.c2, M.c1, M.xl, M.xu,
                M.J_rowptr, M.J_colind, M.W_rowptr, M.W_colind, M.jentry, M.wentry, M.fpart};
  for (void *p : ps)
    if (p) cudaFree(p);
}

int opf_create(OpfData &M, int nb, int nbr, int ng, const int *f_bus, const int *t_bus,
               const double *r, const double *x, const double *b, const double *rate,
               const double *pd, const double *qd, const int *gen_bus, const double *c2,
               const double *c1, const double *xl, const double *xu, cudaStream_t s, int form) {
  M.nb = nb;
  M.nbr = nbr;
  M.ng = ng;
  M.form = form;
  M.n = 2 * nb + 2 * ng + (form ? 4 * nbr : 0);
  M.me = 2 * nb + 1 + (form ? 4 * nbr : 0);
  M.mi = 2 * nbr;
  const int n = M.n;
  const int nc = 2 * nb + 2 * ng;  // the caller's bounds cover the compact variables
  CKR(dev_alloc(&M.f_bus, nbr));
  CKR(dev_alloc(&M.t_bus, nbr));
  CKR(dev_alloc(&M.gen_bus, ng));
  CKR(dev_alloc(&M.adm, nbr));
  CKR(dev_alloc(&M.rate, nbr));
  CKR(dev_alloc(&M.pd, nb));
  CKR(dev_alloc(&M.qd, nb));
  CKR(dev_alloc(&M.c2, ng));
  CKR(dev_alloc(&M.c1, ng));
  CKR(dev_alloc(&M.xl, n));
  CKR(dev_alloc(&M.xu, n));
  CKR(dev_alloc(&M.fpart, grid_for(max(ng, 1), 256) + 1));
  DevTemp T;
  double *dr, *dx, *db;
  CKR(T.alloc(&dr, nbr));
  CKR(T.alloc(&dx, nbr));
  CKR(T.alloc(&db, nbr));
  auto up = [&](void *dst, const void *src, size_t bytes) -> int {
    if (bytes) CK(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, s));
    return IPM_OK;
  };
  CKR(up(M.f_bus, f_bus, sizeof(int) * nbr));
  CKR(up(M.t_bus, t_bus, sizeof(int) * nbr));
  CKR(up(M.gen_bus, gen_bus, sizeof(int) * ng));
  CKR(up(dr, r, sizeof(double) * nbr));
  CKR(up(dx, x, sizeof(double) * nbr));
  CKR(up(db, b, sizeof(double) * nbr));
  CKR(up(M.rate, rate, sizeof(double) * nbr));
  CKR(up(M.pd, pd, sizeof(double) * nb));
  CKR(up(M.qd, qd, sizeof(double) * nb));
  CKR(up(M.c2, c2, sizeof(double) * ng));
  CKR(up(M.c1, c1, sizeof(double) * ng));
  CKR(up(M.xl, xl, sizeof(double) * nc));
  CKR(up(M.xu, xu, sizeof(double) * nc));
  if (n > nc) {  // flow variables are free
    std::vector<double> lo(n - nc, -INFINITY), hi(n - nc, INFINITY);
    CK(cudaMemcpyAsync(M.xl + nc, lo.data(), sizeof(double) * (n - nc), cudaMemcpyHostToDevice,
                       s));
    CK(cudaMemcpyAsync(M.xu + nc, hi.data(), sizeof(double) * (n - nc), cudaMemcpyHostToDevice,
                       s));
    CK(cudaStreamSynchronize(s));  // lo and hi end with this block
  }
  M.ref = gen_bus[0];
  if (nbr > 0) {
    k_branch_admittance<<<grid_for(nbr, 256), 256, 0, s>>>(nbr, dr, dx, db, M.adm);
    CKL();
  }
  OpfDims D{nb, nbr, ng, M.n, M.me, M.mi, M.form};
  CKR(build_pattern(true, D, M, M.me + M.mi, &M.J_rowptr, &M.J_colind, &M.jentry, &M.nnzJ, s));
  CKR(build_pattern(false, D, M, n, &M.W_rowptr, &M.W_colind, &M.wentry, &M.nnzW, s));
  CK(cudaStreamSynchronize(s));
  return IPM_OK;
}

}  // namespace cipm

using namespace cipm;

static int opf_create_form(int form, int nb, int nbr, int ng, const int *f_bus,
                           const int *t_bus, const double *r, const double *x, const double *b,
                           const double *rate, const double *pd, const double *qd,
                           const int *gen_bus, const double *c2, const double *c1,
                           const double *xl, const double *xu, cudaStream_t s, ipm_opf_t *out);

extern "C" int ipm_opf_create(int nb, int nbr, int ng, const int *f_bus, const int *t_bus,
                              const double *r, const double *x, const double *b,
                              const double *rate, const double *pd, const double *qd,
                              const int *gen_bus, const double *c2, const double *c1,
                              const double *xl, const double *xu, cudaStream_t s,
                              ipm_opf_t *out) {
  return opf_create_form(0, nb, nbr, ng, f_bus, t_bus, r, x, b, rate, pd, qd, gen_bus, c2, c1,
                         xl, xu, s, out);
}

extern "C" int ipm_opf_create_flow(int nb, int nbr, int ng, const int *f_bus, const int *t_bus,
                                   const double *r, const double *x, const double *b,
                                   const double *rate, const double *pd, const double *qd,
                                   const int *gen_bus, const double *c2, const double *c1,
                                   const double *xl, const double *xu, cudaStream_t s,
                                   ipm_opf_t *out) {
  return opf_create_form(1, nb, nbr, ng, f_bus, t_bus, r, x, b, rate, pd, qd, gen_bus, c2, c1,
                         xl, xu, s, out);
}

static int opf_create_form(int form, int nb, int nbr, int ng, const int *f_bus,
                           const int *t_bus, const double *r, const double *x, const double *b,
                           const double *rate, const double *pd, const double *qd,
                           const int *gen_bus, const double *c2, const double *c1,
                           const double *xl, const double *xu, cudaStream_t s, ipm_opf_t *out) {
  if (!out || nb <= 0 || nbr < 0 || ng <= 0 || !f_bus || !t_bus || !r || !x || !b || !rate ||
      !pd || !qd || !gen_bus || !c2 || !c1 || !xl || !xu) {
    set_error_msg("ipm_opf_create: bad argument");
    return IPM_ERR_BAD_ARG;
  }
  for (int k = 0; k < nbr; ++k)
    if (f_bus[k] < 0 || f_bus[k] >= nb || t_bus[k] < 0 || t_bus[k] >= nb || f_bus[k] == t_bus[k]) {
      set_error_msg("ipm_opf_create: branch bus index out of range");
      return IPM_ERR_BAD_ARG;
    }
  for (int g = 0; g < ng; ++g)
    if (gen_bus[g] < 0 || gen_bus[g] >= nb) {
      set_error_msg("ipm_opf_create: generator bus index out of range");
      return IPM_ERR_BAD_ARG;
    }
  *out = nullptr;
  s = setup_stream(s);
  ipm_opf_t P = new ipm_opf_s();
  int rc = opf_create(P->M, nb, nbr, ng, f_bus, t_bus, r, x, b, rate, pd, qd, gen_bus, c2, c1, xl,
                      xu, s, form);
  if (rc != IPM_OK) {
    opf_free(P->M);
    delete P;
    return rc;
  }
  *out = P;
  return IPM_OK;
}

extern "C" int ipm_opf_info(ipm_opf_t P, int *n, int *m_e, int *m_i, int *nnzJ, int *nnzW) {
  if (!P) return IPM_ERR_BAD_ARG;
  if (n) *n = P->M.n;
  if (m_e) *m_e = P->M.me;
  if (m_i) *m_i = P->M.mi;
  if (nnzJ) *nnzJ = P->M.nnzJ;
  if (nnzW) *nnzW = P->M.nnzW;
  return IPM_OK;
}

extern "C" int ipm_opf_patterns(ipm_opf_t P, int *J_rowptr, int *J_colind, int *W_rowptr,
                                int *W_colind) {
  if (!P) return IPM_ERR_BAD_ARG;
  const OpfData &M = P->M;
  if (J_rowptr) CK(cudaMemcpy(J_rowptr, M.J_rowptr, sizeof(int) * (M.me + M.mi + 1), cudaMemcpyDefault));
  if (J_colind) CK(cudaMemcpy(J_colind, M.J_colind, sizeof(int) * M.nnzJ, cudaMemcpyDefault));
  if (W_rowptr) CK(cudaMemcpy(W_rowptr, M.W_rowptr, sizeof(int) * (M.n + 1), cudaMemcpyDefault));
  if (W_colind) CK(cudaMemcpy(W_colind, M.W_colind, sizeof(int) * M.nnzW, cudaMemcpyDefault));
  // device-to-device copies may return before they land: done before any stream reads them
  CK(cudaStreamSynchronize(cudaStreamLegacy));
  return IPM_OK;
}

extern "C" int ipm_opf_eval(ipm_opf_t P, const double *x, const double *y, const double *z,
                            double sigma_f, double *f, double *grad, double *g, double *h,
                            double *J_val, double *W_val, cudaStream_t s) {
  if (!P || !x || !g || !h || (W_val && (!y || !z))) return IPM_ERR_BAD_ARG;
  return opf_eval(P->M, x, y, z, sigma_f, f, grad, g, h, J_val, W_val, s);
}

extern "C" int ipm_opf_set_loads(ipm_opf_t P, const double *pd, const double *qd,
                                 cudaStream_t s) {
  if (!P || !pd || !qd) return IPM_ERR_BAD_ARG;
  const OpfData &M = P->M;
  CK(cudaMemcpyAsync(M.pd, pd, sizeof(double) * M.nb, cudaMemcpyDefault, s));
  CK(cudaMemcpyAsync(M.qd, qd, sizeof(double) * M.nb, cudaMemcpyDefault, s));
  return IPM_OK;
}

extern "C" void ipm_opf_destroy(ipm_opf_t P) {
  if (!P) return;
  opf_free(P->M);
  delete P;
}
