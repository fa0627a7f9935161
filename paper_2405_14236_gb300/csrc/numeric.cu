// Numeric phase of the condensed KKT solve: condensation, supernodal Cholesky, triangular
// solves, FP64 iterative refinement (LiftedKKT) and the HyKKT Schur-complement CG.
//
// Storage: each supernode s (columns f..f+w-1, row list rows[0..ld) whose first w entries are
// its own columns) keeps a column-major ld x w panel at Lx + lptr[s].  After ipm_condense the
// panels hold the lower triangle of P K P^T (fill zeroed); after ipm_factor they hold L.
// The supernodal elimination tree is processed level by level (deepest level first for the
// factorization and the forward solve, root first for the backward solve); all supernodes of a
// level are independent.
#include <algorithm>
#include <climits>
#include <cmath>
#include <mutex>

#include "numeric_dev.cuh"

using namespace cipm;

template <typename V>
static int set_smem_limits_t() {
  const int big = 64 * 1024;
  CK(cudaFuncSetAttribute(k_factor_dag<V>, cudaFuncAttributeMaxDynamicSharedMemorySize, big));
  CK(cudaFuncSetAttribute(k_fwd_dag<V>, cudaFuncAttributeMaxDynamicSharedMemorySize, big));
  CK(cudaFuncSetAttribute(k_bwd_dag<V>, cudaFuncAttributeMaxDynamicSharedMemorySize, big));
  return IPM_OK;
}

static int set_smem_limits() {
  static bool done = false;
  if (done) return IPM_OK;
  CKR(set_smem_limits_t<double>());
  CKR(set_smem_limits_t<float>());
  done = true;
  return IPM_OK;
}

extern "C" int ipm_num_create(ipm_sym_t S, int precision, ipm_num_t *out) {
  if (!S || !out || (precision != 64 && precision != 32)) {
    set_error_msg("ipm_num_create: bad argument (precision must be 64 or 32)");
    return IPM_ERR_BAD_ARG;
  }
  *out = nullptr;
  CKR(set_smem_limits());
  ipm_num_t N = new ipm_num_s();
  N->sym = S;
  N->precision = precision;
  const size_t es = precision == 64 ? sizeof(double) : sizeof(float);
  int rc = IPM_OK;
  auto bytes = [&](void **p, int64_t count) {
    if (rc == IPM_OK && cudaMalloc(p, es * (size_t)std::max<int64_t>(count, 1)) != cudaSuccess)
      rc = IPM_ERR_OOM;
    if (rc == IPM_OK && poison_allocations())
      cudaMemset(*p, 0xFF, es * (size_t)std::max<int64_t>(count, 1));
  };
  bytes(&N->Lx, S->panel_len);
  bytes(&N->Dx, S->diag_len);
  if (rc == IPM_OK && cudaMalloc(&N->tJ, sizeof(double) * (size_t)std::max(S->nnzJ, 1)) != cudaSuccess)
    rc = IPM_ERR_OOM;
  if (rc == IPM_OK) poison_fresh((double *)N->tJ, std::max(S->nnzJ, 1));
  if (rc == IPM_OK) rc = dev_alloc(&N->sync, 4 * (int64_t)S->nsuper + 16);
  if (rc == IPM_OK && cudaMemset(N->sync, 0, sizeof(int) * (4 * (size_t)S->nsuper + 16)) != cudaSuccess)
    rc = IPM_ERR_CUDA;
  for (int k = 0; k < 12 && rc == IPM_OK; ++k) rc = dev_alloc(&N->vn[k], S->n);
  for (int k = 0; k < 8 && rc == IPM_OK; ++k) rc = dev_alloc(&N->vm[k], S->m > 0 ? S->m : 1);
  if (rc == IPM_OK) rc = dev_alloc(&N->scal, 64 + DOT_BLOCKS);
  if (rc == IPM_OK && cudaMallocHost((void **)&N->h_scal, sizeof(double) * 64) != cudaSuccess)
    rc = IPM_ERR_OOM;
  if (rc != IPM_OK) {
    ipm_num_destroy(N);
    return rc;
  }
  *out = N;
  return IPM_OK;
}

extern "C" void ipm_num_destroy(ipm_num_t N) {
  if (!N) return;
  if (N->Lx) cudaFree(N->Lx);
  if (N->Dx) cudaFree(N->Dx);
  if (N->tJ) cudaFree(N->tJ);
  if (N->sync) cudaFree(N->sync);
  for (auto *p : N->vn)
    if (p) cudaFree(p);
  for (auto *p : N->vm)
    if (p) cudaFree(p);
  if (N->scal) cudaFree(N->scal);
  if (N->h_scal) cudaFreeHost(N->h_scal);
  delete N;
}

template <typename V>
static int copy_to_double(std::vector<double> &out, const void *src, int64_t count) {
  std::vector<V> tmp(count);
  if (count) CK(cudaMemcpy(tmp.data(), src, sizeof(V) * count, cudaMemcpyDeviceToHost));
  out.assign(tmp.begin(), tmp.end());
  return IPM_OK;
}

extern "C" int ipm_num_export(ipm_num_t N, double *Lx_host) {
  if (!N || !Lx_host) return IPM_ERR_BAD_ARG;
  ipm_sym_t S = N->sym;
  CK(cudaDeviceSynchronize());
  std::vector<double> L, D;
  if (N->precision == 64) {
    CKR(copy_to_double<double>(L, N->Lx, S->panel_len));
    CKR(copy_to_double<double>(D, N->Dx, S->diag_len));
  } else {
    CKR(copy_to_double<float>(L, N->Lx, S->panel_len));
    CKR(copy_to_double<float>(D, N->Dx, S->diag_len));
  }
  std::copy(L.begin(), L.end(), Lx_host);
  if (N->factored) {
    // the factor keeps L11 in a separate array: put it into the panels' diagonal blocks
    const int ns = S->nsuper;
    std::vector<int64_t> lp(ns + 1), dp(ns + 1);
    std::vector<int> sp(ns + 1), rp(ns + 1);
    CK(cudaMemcpy(lp.data(), S->lptr, sizeof(int64_t) * (ns + 1), cudaMemcpyDeviceToHost));
    CK(cudaMemcpy(dp.data(), S->dptr, sizeof(int64_t) * (ns + 1), cudaMemcpyDeviceToHost));
    CK(cudaMemcpy(sp.data(), S->sptr, sizeof(int) * (ns + 1), cudaMemcpyDeviceToHost));
    CK(cudaMemcpy(rp.data(), S->srow_ptr, sizeof(int) * (ns + 1), cudaMemcpyDeviceToHost));
    for (int s = 0; s < ns; ++s) {
      int w = sp[s + 1] - sp[s], ld = rp[s + 1] - rp[s];
      for (int k = 0; k < w; ++k)
        for (int i = 0; i < w; ++i)
          Lx_host[lp[s] + (int64_t)k * ld + i] = i >= k ? D[dp[s] + (int64_t)k * w + i] : 0.0;
    }
  }
  return IPM_OK;
}

extern "C" int ipm_num_info(ipm_num_t N, int *precision, int *last_pcg_iters) {
  if (!N) return IPM_ERR_BAD_ARG;
  if (precision) *precision = N->precision;
  if (last_pcg_iters) *last_pcg_iters = N->last_pcg_iters;
  return IPM_OK;
}

extern "C" int ipm_num_status(ipm_num_t N, int *status) {
  if (!N || !status) return IPM_ERR_BAD_ARG;
  CK(cudaDeviceSynchronize());
  CK(cudaMemcpy(status, N->sync + 4 * N->sym->nsuper + 4, sizeof(int), cudaMemcpyDeviceToHost));
  return IPM_OK;
}

extern "C" int ipm_set_spin_limit(long long polls) {
  if (polls < 1) return IPM_ERR_BAD_ARG;
  CK(cudaMemcpyToSymbol(g_spin_limit, &polls, sizeof(polls)));
  return batch_set_spin_limit(polls);
}

extern "C" int ipm_debug_add_dependency(ipm_sym_t S, int supernode, int extra) {
  if (!S || supernode < 0 || supernode >= S->nsuper) return IPM_ERR_BAD_ARG;
  int v = 0;
  CK(cudaMemcpy(&v, S->upd_need + supernode, sizeof(int), cudaMemcpyDeviceToHost));
  v += extra;
  CK(cudaMemcpy(S->upd_need + supernode, &v, sizeof(int), cudaMemcpyHostToDevice));
  return IPM_OK;
}

static int device_status(ipm_num_t N) {
  int st = 0;
  CK(cudaMemcpy(&st, N->sync + 4 * N->sym->nsuper + 4, sizeof(int), cudaMemcpyDeviceToHost));
  return st;
}

template <typename V>
static int condense_t(ipm_sym_t S, ipm_num_t N, const double *W_val, const double *sigma_x,
                      const double *J_val, const double *d_row, double delta_w, cudaStream_t s) {
  double *tJ = (double *)N->tJ;
  if (S->nnzJ > 0) {
    k_scale_jv<<<grid_for(S->nnzJ, 256), 256, 0, s>>>(S->nnzJ, S->J_rowidx, J_val, d_row, tJ);
    count_launches(1);
    CKL();
  }
  k_condense<V><<<S->nsuper, 128, 0, s>>>(S->sptr, S->srow_ptr, S->lptr, S->slot_ptr, S->items,
                                          S->perm, W_val, sigma_x, J_val, tJ, delta_w,
                                          (V *)N->Lx);
  count_launches(1);
  CKL();
  return IPM_OK;
}

extern "C" int ipm_condense(ipm_sym_t S, ipm_num_t N, const double *W_val, const double *sigma_x,
                            const double *J_val, const double *d_row, double delta_w,
                            cudaStream_t s) {
  NvtxRange nvtx_range("ipm_condense");
  if (!S || !N || N->sym != S || !sigma_x || (S->nnzW && !W_val) || (S->nnzJ && (!J_val || !d_row)))
    return IPM_ERR_BAD_ARG;
  N->cW = W_val;
  N->cSig = sigma_x;
  N->cJ = J_val;
  N->cD = d_row;
  N->cDw = delta_w;
  if (S->nsuper == 0) return IPM_OK;
  N->factored = false;
  return N->precision == 64 ? condense_t<double>(S, N, W_val, sigma_x, J_val, d_row, delta_w, s)
                            : condense_t<float>(S, N, W_val, sigma_x, J_val, d_row, delta_w, s);
}

static int persistent_grid(const void *kernel, int threads, size_t smem) {
  static int nsm = 0;
  if (nsm == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    if (nsm <= 0) nsm = 1;
  }
  int occ = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kernel, threads, smem);
  occ = std::max(1, std::min(occ, 4));
  return nsm * occ;
}

static SyncCtl sync_ctl(ipm_sym_t S, ipm_num_t N, int region, int ticket) {
  const int ns = S->nsuper;
  int *tail = N->sync + 4 * ns;
  return SyncCtl{N->sync + region * ns, tail + ticket, tail + 3, tail + 4};
}

template <typename V>
static int factor_t(ipm_sym_t S, ipm_num_t N, int *d_info, cudaStream_t s) {
  FactTaskArgs<V> T;
  T.F = FactArgs<V>{S->level_sn, S->sptr, S->srow_ptr, S->srow, S->snode, S->lptr, S->dptr,
                    (V *)N->Lx, (V *)N->Dx, d_info};
  T.tasks = S->ftasks;
  T.ntasks = S->nftasks;
  T.upd_need = S->upd_need;
  T.C = sync_ctl(S, N, 0, 0);
  T.ns = S->nsuper;
  const int w = S->max_w;
  size_t sm = sizeof(V) * std::max((size_t)w * w + (size_t)CIPM_RB * (w + 1),
                                   2 * (size_t)CIPM_RB * (w + 1));
  if (T.ntasks > 0) {
    k_factor_dag<V><<<persistent_grid((const void *)k_factor_dag<V>, 256, sm), 256, sm, s>>>(T);
    count_launches(1);
    CKL();
  }
  return IPM_OK;
}

extern "C" int ipm_factor(ipm_sym_t S, ipm_num_t N, int *d_info, cudaStream_t s) {
  NvtxRange nvtx_range("ipm_factor");
  if (!S || !N || N->sym != S || !d_info) return IPM_ERR_BAD_ARG;
  const int ns = S->nsuper;
  // counters of the factorization (update arrivals, panel tasks done), its ticket, abort, status
  CK(cudaMemsetAsync(N->sync, 0, sizeof(int) * 2 * ns, s));
  CK(cudaMemsetAsync(N->sync + 4 * ns, 0, sizeof(int) * 8, s));
  k_info_set<<<1, 1, 0, s>>>(d_info);
  count_launches(1);
  CKL();
  CKR(N->precision == 64 ? factor_t<double>(S, N, d_info, s) : factor_t<float>(S, N, d_info, s));
  k_info_fix<<<1, 1, 0, s>>>(d_info, N->sync + 4 * ns + 4);
  count_launches(1);
  CKL();
  N->factored = true;
  return IPM_OK;
}

// y (permuted, length n, value type V) <- L^{-T} L^{-1} y in place, counters in C_fwd / C_bwd
template <typename V>
static int solve_permuted_t(ipm_sym_t S, ipm_num_t N, double *y, SyncCtl C_fwd, SyncCtl C_bwd,
                            cudaStream_t s) {
  SolveTaskArgs<V> T;
  T.A = SolveArgs<V>{S->level_sn, S->sptr, S->srow_ptr, S->srow, S->lptr, S->dptr,
                     (const V *)N->Lx, (const V *)N->Dx, y};
  T.snode = S->snode;
  T.fwd_need = S->fwd_need;
  T.ns = S->nsuper;
  size_t sm = sizeof(double) * (size_t)S->max_w * S->max_w;
  T.C = C_fwd;
  k_fwd_dag<V><<<persistent_grid((const void *)k_fwd_dag<V>, 128, sm), 128, sm, s>>>(T);
  count_launches(1);
  CKL();
  T.C = C_bwd;
  k_bwd_dag<V><<<persistent_grid((const void *)k_bwd_dag<V>, 128, sm), 128, sm, s>>>(T);
  count_launches(1);
  CKL();
  return IPM_OK;
}

// x = (L L^T)^{-1} b with the factor, any precision (b, x: double, original order; may alias);
// y_work: n doubles of scratch; cnt: 2 nsuper counters, tail: tickets (2), abort, status
template <typename V>
static int factor_solve_t(ipm_sym_t S, ipm_num_t N, const double *b, double *x, void *y_work,
                          int *cnt, int *tail, cudaStream_t s) {
  const int ns = S->nsuper;
  double *y = (double *)y_work;
  CK(cudaMemsetAsync(cnt, 0, sizeof(int) * 2 * (size_t)ns, s));
  CK(cudaMemsetAsync(tail, 0, sizeof(int) * 2, s));
  k_gather_perm<<<grid_for(S->n, 256), 256, 0, s>>>(S->perm, S->n, b, y);
  count_launches(1);
  CKL();
  if (ns > 0)
    CKR(solve_permuted_t<V>(S, N, y, SyncCtl{cnt, tail + 0, tail + 2, tail + 3},
                            SyncCtl{cnt + ns, tail + 1, tail + 2, tail + 3}, s));
  k_scatter_perm<<<grid_for(S->n, 256), 256, 0, s>>>(S->perm, S->n, y, x);
  count_launches(1);
  CKL();
  return IPM_OK;
}

// x = K^{-1} b with the handle's factor and workspace
static int solve_full(ipm_sym_t S, ipm_num_t N, const double *b, double *x, cudaStream_t s) {
  const int ns = S->nsuper;
  int *cnt = N->sync + 2 * ns, *tail = N->sync + 4 * ns + 1;
  return N->precision == 64 ? factor_solve_t<double>(S, N, b, x, N->vn[7], cnt, tail, s)
                            : factor_solve_t<float>(S, N, b, x, N->vn[7], cnt, tail, s);
}

extern "C" int ipm_solve(ipm_sym_t S, ipm_num_t N, const double *b, double *x, int nrhs,
                         cudaStream_t s) {
  NvtxRange nvtx_range("ipm_solve");
  if (!S || !N || N->sym != S || !b || !x || nrhs < 1) return IPM_ERR_BAD_ARG;
  // the columns one after another (each solve is one forward and one backward launch that
  // read the factor once)
  for (int k = 0; k < nrhs; ++k)
    CKR(solve_full(S, N, b + (int64_t)k * S->n, x + (int64_t)k * S->n, s));
  return IPM_OK;
}

// --- K x = b solved to FP64 accuracy with an FP32 factor: conjugate gradients in FP64 on K
// (K p = (W + Sigma_x + delta_w I) p + J^T (d o (J p)) from the condensation inputs),
// preconditioned by the FP32 factor (L L^T)^{-1}.
__global__ void k_kmat_rows(int m, const int *J_rowptr, const int *J_colind, const double *Jv,
                            const double *d, const double *p, double *t) {
  int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= m) return;
  double acc = 0.0;
  for (int q = J_rowptr[r]; q < J_rowptr[r + 1]; ++q) acc += Jv[q] * p[J_colind[q]];
  t[r] = d[r] * acc;
}
__global__ void k_kmat_cols(int n, const int *W_rowptr, const int *W_colind, const int *W_rowidx,
                            const int *WT_ptr, const int *WT_ent, const double *Wv,
                            const double *sigma, double dw, const int *JT_ptr, const int *JT_ent,
                            const int *J_rowidx, const double *Jv, const double *t,
                            const double *p, double *out) {
  int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  double acc = (sigma[j] + dw) * p[j];
  for (int q = W_rowptr[j]; q < W_rowptr[j + 1]; ++q) acc += Wv[q] * p[W_colind[q]];
  for (int u = WT_ptr[j]; u < WT_ptr[j + 1]; ++u) {
    int e = WT_ent[u];
    int r = W_rowidx[e];
    if (r != j) acc += Wv[e] * p[r];
  }
  for (int u = JT_ptr[j]; u < JT_ptr[j + 1]; ++u) {
    int q = JT_ent[u];
    acc += Jv[q] * t[J_rowidx[q]];
  }
  out[j] = acc;
}
__global__ void k_pcg_xr(int n, const double *sc, const double *p, const double *Ap, double *x,
                         double *r) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double alpha = sc[0] / sc[1];  // rz / pAp
  x[i] += alpha * p[i];
  r[i] -= alpha * Ap[i];
}
__global__ void k_pcg_p(int n, const double *sc, const double *z, double *p) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  p[i] = z[i] + (sc[2] / sc[0]) * p[i];  // beta = rz_new / rz
}

__global__ void k_absmax(int n, const double *v, double *out) {
  __shared__ double sh[32];
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  block_max_to(out, i < n ? fabs(v[i]) : 0.0, sh);
}

// max over rows of the row sums of |W + Sigma_x + delta_w I| + |J|^T |d| |J| (an upper bound of
// ||K||_inf used by the normwise stopping test)
__global__ void k_knorm(int n, const int *W_rowptr, const int *W_colind, const int *W_rowidx,
                        const int *WT_ptr, const int *WT_ent, const double *Wv,
                        const double *sigma, double dw, const int *JT_ptr, const int *JT_ent,
                        const int *J_rowidx, const int *J_rowptr, const double *Jv,
                        const double *d, double *out) {
  __shared__ double sh[32];
  int j = blockIdx.x * blockDim.x + threadIdx.x;
  double acc = 0.0;
  if (j < n) {
    double diag = sigma[j] + dw;
    for (int q = W_rowptr[j]; q < W_rowptr[j + 1]; ++q) {
      if (W_colind[q] == j) diag += Wv[q];
      else acc += fabs(Wv[q]);
    }
    for (int u = WT_ptr[j]; u < WT_ptr[j + 1]; ++u) {
      int e = WT_ent[u];
      if (W_rowidx[e] != j) acc += fabs(Wv[e]);
    }
    acc += fabs(diag);
    for (int u = JT_ptr[j]; u < JT_ptr[j + 1]; ++u) {
      int q = JT_ent[u];
      int r = J_rowidx[q];
      double rs = 0.0;
      for (int t = J_rowptr[r]; t < J_rowptr[r + 1]; ++t) rs += fabs(Jv[t]);
      acc += fabs(d[r]) * fabs(Jv[q]) * rs;
    }
  }
  block_max_to(out, acc, sh);
}

static int kmat(ipm_sym_t S, ipm_num_t N, const double *p, double *out, cudaStream_t s) {
  double *t = N->vm[5];
  if (S->m > 0) {
    k_kmat_rows<<<grid_for(S->m, 256), 256, 0, s>>>(S->m, S->J_rowptr, S->J_colind, N->cJ, N->cD, p,
                                                    t);
    count_launches(1);
  }
  k_kmat_cols<<<grid_for(S->n, 256), 256, 0, s>>>(S->n, S->W_rowptr, S->W_colind, S->W_rowidx,
                                                  S->WT_ptr, S->WT_ent, N->cW, N->cSig, N->cDw,
                                                  S->JT_ptr, S->JT_ent, S->J_rowidx, N->cJ, t, p,
                                                  out);
  count_launches(1);
  CKL();
  return IPM_OK;
}

// Conjugate gradients in FP64 on K x = b (K from the condensation inputs), preconditioned by the
// factor (L L^T)^{-1} of either precision; from x0 = M^{-1} b, or from the x given (use_x0).
// Stops at ||r|| <= 1e-14 ||b|| or (normwise = true) a normwise backward error of K x = b of
// 1e-14; maxit iterations without that, or negative curvature, return IPM_ERR_NOT_PD.
static int pcg_k(ipm_sym_t S, ipm_num_t N, const double *b, double *x, bool use_x0, int maxit,
                 cudaStream_t s, bool normwise = true);

// FP64 accuracy from the factor of any precision; FP64 factors solve directly
static int ksolve(ipm_sym_t S, ipm_num_t N, const double *b, double *x, cudaStream_t s) {
  if (N->precision == 64) return solve_full(S, N, b, x, s);
  return pcg_k(S, N, b, x, false, 100, s);
}

static int pcg_k(ipm_sym_t S, ipm_num_t N, const double *b, double *x, bool use_x0, int maxit,
                 cudaStream_t s, bool normwise) {
  const int n = S->n;
  double *r = N->vn[8], *z = N->vn[9], *p = N->vn[10], *Ap = N->vn[11];
  double *sc = N->scal + 8, *partial = N->scal + 64;
  CKR(dot(b, b, n, partial, sc + 4, s));
  CK(cudaMemcpyAsync(N->h_scal + 4, sc + 4, sizeof(double), cudaMemcpyDeviceToHost, s));
  // ||K||_inf bound, ||b||_inf for the normwise backward error of K x = b
  CK(cudaMemsetAsync(sc + 5, 0, sizeof(double) * 3, s));
  k_knorm<<<grid_for(n, 256), 256, 0, s>>>(n, S->W_rowptr, S->W_colind, S->W_rowidx, S->WT_ptr,
                                           S->WT_ent, N->cW, N->cSig, N->cDw, S->JT_ptr,
                                           S->JT_ent, S->J_rowidx, S->J_rowptr, N->cJ, N->cD,
                                           sc + 5);
  count_launches(1);
  k_absmax<<<grid_for(n, 256), 256, 0, s>>>(n, b, sc + 6);
  count_launches(1);
  CKL();
  if (!use_x0) CKR(solve_full(S, N, b, x, s));  // x0 = M^{-1} b
  CKR(kmat(S, N, x, Ap, s));
  CK(cudaMemcpyAsync(r, b, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
  k_axpy<<<grid_for(n, 256), 256, 0, s>>>(n, -1.0, Ap, r);
  count_launches(1);
  CKR(solve_full(S, N, r, z, s));
  CK(cudaMemcpyAsync(p, z, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
  CKR(dot(r, z, n, partial, sc + 0, s));
  CK(cudaStreamSynchronize(s));
  const double bnorm = std::sqrt(N->h_scal[4]);
  int it = 0;
  bool converged = false;
  for (; it < maxit; ++it) {
    CKR(dot(r, r, n, partial, sc + 3, s));
    CK(cudaMemsetAsync(sc + 7, 0, sizeof(double) * 2, s));
    k_absmax<<<grid_for(n, 256), 256, 0, s>>>(n, r, sc + 7);
    k_absmax<<<grid_for(n, 256), 256, 0, s>>>(n, x, sc + 8);
    count_launches(2);
    CK(cudaMemcpyAsync(N->h_scal + 3, sc + 3, sizeof(double) * 6, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    const double rn = std::sqrt(N->h_scal[3]);
    if (!std::isfinite(rn)) return IPM_ERR_NONFINITE;
    // stop at a relative residual of 1e-14 or a normwise backward error of K x = b of 1e-14
    const double knorm = N->h_scal[5], binf = N->h_scal[6], rinf = N->h_scal[7], xinf = N->h_scal[8];
    if (rn <= 1e-14 * bnorm || (normwise && rinf <= 1e-14 * (knorm * xinf + binf))) {
      converged = true;
      break;
    }
    CKR(kmat(S, N, p, Ap, s));
    CKR(dot(p, Ap, n, partial, sc + 1, s));
    CK(cudaMemcpyAsync(N->h_scal + 1, sc + 1, sizeof(double), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    if (!(N->h_scal[1] > 0.0)) {  // negative curvature: K is not positive definite
      N->last_pcg_iters += it;
      return IPM_ERR_NOT_PD;
    }
    k_pcg_xr<<<grid_for(n, 256), 256, 0, s>>>(n, sc, p, Ap, x, r);
    count_launches(1);
    CKR(solve_full(S, N, r, z, s));
    CKR(dot(r, z, n, partial, sc + 2, s));
    k_pcg_p<<<grid_for(n, 256), 256, 0, s>>>(n, sc, z, p);
    count_launches(1);
    k_copy_scalar<<<1, 1, 0, s>>>(sc + 2, sc + 0);
    count_launches(1);
    CKL();
  }
  N->last_pcg_iters += it;
  // an FP32 factor that does not precondition K to FP64 accuracy within the iteration limit is
  // reported like a failed factorization: the caller regularizes more (larger delta_w)
  return converged ? IPM_OK : IPM_ERR_NOT_PD;
}

// condensed solve of the augmented system: dx = K^{-1}(ra + J^T (d o rb)), dz = d o (J dx - rb)
static int aug_condensed(ipm_sym_t S, ipm_num_t N, const double *Jv, const double *d,
                         const double *ra, const double *rb, double *dx, double *dz,
                         cudaStream_t s) {
  const int n = S->n, m = S->m;
  double *t = N->vn[6];
  k_jt_apply<<<grid_for(n, 256), 256, 0, s>>>(n, S->JT_ptr, S->JT_ent, S->J_rowidx, Jv, d, rb, 0,
                                              m, ra, 1.0, t);
  count_launches(1);
  CKL();
  CKR(ksolve(S, N, t, dx, s));  // (IPM_ERR_NOT_PD on an FP32 factor that fails to precondition)
  if (m > 0) {
    k_recover_dz<<<grid_for(m, 256), 256, 0, s>>>(0, m, S->J_rowptr, S->J_colind, Jv, d, dx, rb,
                                                  dz);
    count_launches(1);
    CKL();
  }
  return IPM_OK;
}

extern "C" int ipm_aug_solve(ipm_sym_t S, ipm_num_t N, const double *W_val, const double *sigma_x,
                             const double *J_val, const double *d_row, double delta_w,
                             const double *a, const double *b, double *dx, double *dz,
                             int max_refine, double tol, double *d_eta, int *d_steps,
                             cudaStream_t s) {
  NvtxRange nvtx_range("ipm_aug_solve");
  if (!S || !N || N->sym != S || !a || !dx || !sigma_x || (S->m && (!b || !dz || !d_row)) ||
      max_refine < 0)
    return IPM_ERR_BAD_ARG;
  const int n = S->n, m = S->m;
  N->last_pcg_iters = 0;
  CKR(aug_condensed(S, N, J_val, d_row, a, b, dx, dz, s));
  AugArgs A;
  A.n = n;
  A.m = m;
  A.m_e = 0;
  A.J_rowptr = S->J_rowptr;
  A.J_colind = S->J_colind;
  A.J_rowidx = S->J_rowidx;
  A.JT_ptr = S->JT_ptr;
  A.JT_ent = S->JT_ent;
  A.W_rowptr = S->W_rowptr;
  A.W_colind = S->W_colind;
  A.W_rowidx = S->W_rowidx;
  A.WT_ptr = S->WT_ptr;
  A.WT_ent = S->WT_ent;
  A.Wv = W_val;
  A.sigma = sigma_x;
  A.Jv = J_val;
  A.d = d_row;
  A.dw = delta_w;
  A.sx = dx;
  A.sz = dz;
  A.ra = a;
  A.rb = b;
  A.outx = N->vn[0];
  A.outz = N->vm[0];
  A.scal = N->scal;
  double *cx = N->vn[1], *cz = N->vm[1];
  double normA = 0.0, eta = INFINITY, eta_prev = INFINITY;
  int steps = 0;
  for (int it = 0;; ++it) {
    A.want_norm_a = it == 0;
    CK(cudaMemsetAsync(N->scal, 0, sizeof(double) * (it == 0 ? 4 : 3), s));
    k_aug_resid_x<<<grid_for(n, 256), 256, 0, s>>>(A);
    count_launches(1);
    CKL();
    if (m > 0) k_aug_resid_z<<<grid_for(m, 256), 256, 0, s>>>(A);
    if (m > 0) count_launches(1);
    CKL();
    CK(cudaMemcpyAsync(N->h_scal, N->scal, sizeof(double) * 4, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    if (it == 0) normA = N->h_scal[3];
    double den = normA * N->h_scal[1] + N->h_scal[2];
    eta = den > 0 ? N->h_scal[0] / den : 0.0;
    if (!std::isfinite(eta) && it == 0) break;
    if (it > 0 && !(eta <= eta_prev)) {
      // the last correction made the solution worse: take it back and stop
      k_axpy<<<grid_for(n, 256), 256, 0, s>>>(n, -1.0, cx, dx);
      count_launches(1);
      CKL();
      if (m > 0) k_axpy<<<grid_for(m, 256), 256, 0, s>>>(m, -1.0, cz, dz);
      if (m > 0) count_launches(1);
      CKL();
      eta = eta_prev;
      --steps;
      break;
    }
    if (eta <= tol || it >= max_refine || (it > 0 && eta > 0.5 * eta_prev)) break;
    eta_prev = eta;
    CKR(aug_condensed(S, N, J_val, d_row, A.outx, A.outz, cx, cz, s));
    k_axpy<<<grid_for(n, 256), 256, 0, s>>>(n, 1.0, cx, dx);
    count_launches(1);
    CKL();
    if (m > 0) k_axpy<<<grid_for(m, 256), 256, 0, s>>>(m, 1.0, cz, dz);
    if (m > 0) count_launches(1);
    CKL();
    ++steps;
  }
  if (std::isfinite(eta) && eta > tol && N->precision == 64 && max_refine > 0) {
    // Richardson stagnated above tol (cond(K) eps_mach near 1): conjugate gradients on the
    // condensed system K dx = a + J^T (d o b), preconditioned by the same factor and started
    // from the refined dx, then dz = d o (J dx - b); the better of the two solutions is kept
    double *t = N->vn[5];
    CK(cudaMemcpyAsync(cx, dx, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
    if (m > 0) CK(cudaMemcpyAsync(cz, dz, sizeof(double) * m, cudaMemcpyDeviceToDevice, s));
    k_jt_apply<<<grid_for(n, 256), 256, 0, s>>>(n, S->JT_ptr, S->JT_ent, S->J_rowidx, J_val, d_row,
                                                b, 0, m, a, 1.0, t);
    count_launches(1);
    CKL();
    // (K's normwise test is far looser than the augmented system's when D is large: the
    // relative residual alone stops these iterations)
    const int prc = pcg_k(S, N, t, dx, true, 50, s, false);
    if (prc < 0 || prc == IPM_ERR_TIMEOUT) return prc;
    if (m > 0) {
      k_recover_dz<<<grid_for(m, 256), 256, 0, s>>>(0, m, S->J_rowptr, S->J_colind, J_val, d_row,
                                                    dx, b, dz);
      count_launches(1);
      CKL();
    }
    A.want_norm_a = 0;
    CK(cudaMemsetAsync(N->scal, 0, sizeof(double) * 3, s));
    k_aug_resid_x<<<grid_for(n, 256), 256, 0, s>>>(A);
    count_launches(1);
    CKL();
    if (m > 0) {
      k_aug_resid_z<<<grid_for(m, 256), 256, 0, s>>>(A);
      count_launches(1);
      CKL();
    }
    CK(cudaMemcpyAsync(N->h_scal, N->scal, sizeof(double) * 3, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    const double den = normA * N->h_scal[1] + N->h_scal[2];
    const double eta2 = den > 0 ? N->h_scal[0] / den : 0.0;
    if (std::isfinite(eta2) && eta2 < eta) {
      eta = eta2;
    } else {
      CK(cudaMemcpyAsync(dx, cx, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
      if (m > 0) CK(cudaMemcpyAsync(dz, cz, sizeof(double) * m, cudaMemcpyDeviceToDevice, s));
    }
  }
  if (d_eta) CK(cudaMemcpyAsync(d_eta, &eta, sizeof(double), cudaMemcpyHostToDevice, s));
  if (d_steps) CK(cudaMemcpyAsync(d_steps, &steps, sizeof(int), cudaMemcpyHostToDevice, s));
  CK(cudaStreamSynchronize(s));
  if (int st = device_status(N)) return st;
  if (!std::isfinite(eta)) return IPM_ERR_NONFINITE;
  return IPM_OK;
}

// One HyKKT solve (Eq. (10)): rhs1 = a + J^T (d o b); CG on S_gamma dy = G K^{-1} rhs1 - b_G from
// dy = 0; dx = K^{-1}(rhs1 - G^T dy); dz = d o (H dx - b_H).  dyz: dy over the G rows, then dz.
static int hykkt_once(ipm_sym_t S, ipm_num_t N, int m_e, const double *J_val, const double *d_row,
                      const double *a, const double *b, double rtol, int maxit, double *dx,
                      double *dyz, int *h_iters, double *h_relres, cudaStream_t s) {
  const int n = S->n, m = S->m;
  double *rhs1 = N->vn[0], *w = N->vn[1], *u = N->vn[2];
  double *r = N->vm[0], *p = N->vm[1], *Sp = N->vm[2];
  double *sc = N->scal, *partial = N->scal + 64;
  double *dy = dyz;
  // rhs1 = a + J^T (d o b)  ( = r1 + gamma G^T r2 with r1 = a + H^T D_H b_H, r2 = b_G )
  k_jt_apply<<<grid_for(n, 256), 256, 0, s>>>(n, S->JT_ptr, S->JT_ent, S->J_rowidx, J_val, d_row,
                                              b, 0, m, a, 1.0, rhs1);
  count_launches(1);
  CKL();
  CKR(ksolve(S, N, rhs1, w, s));
  int iters = 0;
  double relres = 0.0;
  int rc = IPM_OK;
  if (m_e > 0) {
    // r = G w - b_G ; dy = 0 ; p = r
    k_j_apply<<<grid_for(m_e, 256), 256, 0, s>>>(0, m_e, S->J_rowptr, S->J_colind, J_val, w, b, r);
    count_launches(1);
    CKL();
    CK(cudaMemsetAsync(dy, 0, sizeof(double) * m_e, s));
    CK(cudaMemcpyAsync(p, r, sizeof(double) * m_e, cudaMemcpyDeviceToDevice, s));
    CKR(dot(r, r, m_e, partial, sc + 0, s));
    CK(cudaMemcpyAsync(N->h_scal, sc, sizeof(double), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    const double r0 = std::sqrt(N->h_scal[0]);
    const double stop = std::max(rtol * r0, 1e-14);
    double rn = r0;
    while (rn > stop && iters < maxit) {
      // Sp = G K^{-1} G^T p
      k_jt_apply<<<grid_for(n, 256), 256, 0, s>>>(n, S->JT_ptr, S->JT_ent, S->J_rowidx, J_val,
                                                  nullptr, p, 0, m_e, nullptr, 1.0, u);
      count_launches(1);
      CKL();
      CKR(ksolve(S, N, u, N->vn[6], s));
      k_j_apply<<<grid_for(m_e, 256), 256, 0, s>>>(0, m_e, S->J_rowptr, S->J_colind, J_val,
                                                   N->vn[6], nullptr, Sp);
      count_launches(1);
      CKL();
      CKR(dot(p, Sp, m_e, partial, sc + 1, s));
      k_cg_update_xr<<<grid_for(m_e, 256), 256, 0, s>>>(m_e, sc, p, Sp, dy, r);
      count_launches(1);
      CKL();
      CKR(dot(r, r, m_e, partial, sc + 2, s));
      k_cg_update_p<<<grid_for(m_e, 256), 256, 0, s>>>(m_e, sc, r, p);
      count_launches(1);
      CKL();
      k_copy_scalar<<<1, 1, 0, s>>>(sc + 2, sc + 0);
      count_launches(1);
      CKL();
      CK(cudaMemcpyAsync(N->h_scal, sc + 2, sizeof(double), cudaMemcpyDeviceToHost, s));
      CK(cudaStreamSynchronize(s));
      rn = std::sqrt(N->h_scal[0]);
      ++iters;
      if (!std::isfinite(rn)) break;
    }
    relres = r0 > 0 ? rn / r0 : 0.0;
    if (!std::isfinite(rn)) rc = IPM_ERR_NONFINITE;
    else if (rn > stop) rc = IPM_ERR_CG_MAXIT;
    // dx = K^{-1}(rhs1 - G^T dy)
    k_jt_apply<<<grid_for(n, 256), 256, 0, s>>>(n, S->JT_ptr, S->JT_ent, S->J_rowidx, J_val,
                                                nullptr, dy, 0, m_e, rhs1, -1.0, u);
    count_launches(1);
    CKL();
    CKR(ksolve(S, N, u, dx, s));
  } else {
    CK(cudaMemcpyAsync(dx, w, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
  }
  if (m > m_e) {
    k_recover_dz<<<grid_for(m - m_e, 256), 256, 0, s>>>(m_e, m, S->J_rowptr, S->J_colind, J_val,
                                                        d_row, dx, b, dyz + m_e);
    count_launches(1);
    CKL();
  }
  if (h_iters) *h_iters += iters;
  if (h_relres) *h_relres = relres;
  return rc;
}

// HyKKT solve of the augmented system (Eq. (10)) followed, when its normwise backward error on
// the augmented system exceeds 1e-10, by iterative refinement on that system (Sec. 2.2): the
// residual is solved by the same HyKKT procedure and added, at most three times, stopping when
// the error no longer halves.  An FP32 factor enters only through ksolve (FP64-accurate solves).
extern "C" int hykkt_cg(ipm_sym_t S, ipm_num_t N, int m_e, const double *J_val,
                        const double *d_row, double gamma, const double *a, const double *b,
                        double rtol, int maxit, double *dx, double *dy, double *dz, int *h_iters,
                        double *h_relres, cudaStream_t s) {
  NvtxRange nvtx_range("hykkt_cg");
  const int n = S ? S->n : 0, m = S ? S->m : 0;
  if (!S || !N || N->sym != S || m_e < 0 || m_e > m || !a || !dx || (m && (!b || !d_row)) ||
      (m_e && !dy) || (m > m_e && !dz) || maxit < 0)
    return IPM_ERR_BAD_ARG;
  (void)gamma;  // gamma enters through d_row[0..m_e), the weights K_gamma was condensed with
  N->last_pcg_iters = 0;
  double *dyz = N->vm[3], *cz = N->vm[6], *cx = N->vn[3];
  int iters = 0;
  double relres = 0.0;
  int rc = hykkt_once(S, N, m_e, J_val, d_row, a, b, rtol, maxit, dx, dyz, &iters, &relres, s);
  if (rc < 0 || rc == IPM_ERR_NOT_PD || rc == IPM_ERR_NONFINITE) return rc;
  AugArgs A;
  A.n = n;
  A.m = m;
  A.m_e = m_e;
  A.J_rowptr = S->J_rowptr;
  A.J_colind = S->J_colind;
  A.J_rowidx = S->J_rowidx;
  A.JT_ptr = S->JT_ptr;
  A.JT_ent = S->JT_ent;
  A.W_rowptr = S->W_rowptr;
  A.W_colind = S->W_colind;
  A.W_rowidx = S->W_rowidx;
  A.WT_ptr = S->WT_ptr;
  A.WT_ent = S->WT_ent;
  A.Wv = N->cW;
  A.sigma = N->cSig;
  A.Jv = J_val;
  A.d = d_row;
  A.dw = N->cDw;
  A.sx = dx;
  A.sz = dyz;
  A.ra = a;
  A.rb = b;
  A.outx = N->vn[4];
  A.outz = N->vm[4];
  A.scal = N->scal;
  double normA = 0.0, eta = INFINITY, eta_prev = INFINITY, corr_scale = 1.0;
  for (int it = 0;; ++it) {
    A.want_norm_a = it == 0;
    CK(cudaMemsetAsync(N->scal, 0, sizeof(double) * (it == 0 ? 4 : 3), s));
    k_aug_resid_x<<<grid_for(n, 256), 256, 0, s>>>(A);
    count_launches(1);
    CKL();
    if (m > 0) {
      k_aug_resid_z<<<grid_for(m, 256), 256, 0, s>>>(A);
      count_launches(1);
      CKL();
    }
    CK(cudaMemcpyAsync(N->h_scal, N->scal, sizeof(double) * 4, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    if (it == 0) normA = N->h_scal[3];
    const double den = normA * N->h_scal[1] + N->h_scal[2];
    eta = den > 0 ? N->h_scal[0] / den : 0.0;
    if (it > 0 && !(eta <= eta_prev)) {
      // the last correction made the solution worse: take it back and stop
      k_axpy<<<grid_for(n, 256), 256, 0, s>>>(n, -corr_scale, cx, dx);
      count_launches(1);
      CKL();
      if (m > 0) {
        k_axpy<<<grid_for(m, 256), 256, 0, s>>>(m, -corr_scale, cz, dyz);
        count_launches(1);
        CKL();
      }
      eta = eta_prev;
      break;
    }
    if (!std::isfinite(eta) || eta <= 1e-10 || it >= 3 || (it > 0 && eta > 0.5 * eta_prev)) break;
    eta_prev = eta;
    // the residual scaled to unit size, so that the CG's absolute floor (1e-14) does not end the
    // correction solve early; the correction is scaled back when it is added
    corr_scale = N->h_scal[0] > 0 ? N->h_scal[0] : 1.0;
    k_scale<<<grid_for(n, 256), 256, 0, s>>>(n, 1.0 / corr_scale, A.outx);
    count_launches(1);
    CKL();
    if (m > 0) {
      k_scale<<<grid_for(m, 256), 256, 0, s>>>(m, 1.0 / corr_scale, A.outz);
      count_launches(1);
      CKL();
    }
    const int rc2 = hykkt_once(S, N, m_e, J_val, d_row, A.outx, A.outz, rtol, maxit, cx, cz,
                               &iters, nullptr, s);
    if (rc2 < 0 || rc2 == IPM_ERR_NOT_PD || rc2 == IPM_ERR_NONFINITE) return rc2;
    k_axpy<<<grid_for(n, 256), 256, 0, s>>>(n, corr_scale, cx, dx);
    count_launches(1);
    CKL();
    if (m > 0) {
      k_axpy<<<grid_for(m, 256), 256, 0, s>>>(m, corr_scale, cz, dyz);
      count_launches(1);
      CKL();
    }
  }
  N->last_eta = eta;
  if (m_e > 0) CK(cudaMemcpyAsync(dy, dyz, sizeof(double) * m_e, cudaMemcpyDeviceToDevice, s));
  if (m > m_e)
    CK(cudaMemcpyAsync(dz, dyz + m_e, sizeof(double) * (m - m_e), cudaMemcpyDeviceToDevice, s));
  CK(cudaStreamSynchronize(s));
  if (h_iters) *h_iters = iters;
  if (h_relres) *h_relres = relres;
  if (int st = device_status(N)) return st;
  if (!std::isfinite(eta)) return IPM_ERR_NONFINITE;
  return rc;
}

// ---------------------------------------------------------------- allocation-free solve
// ipm_solve_noalloc: the same triangular solves as ipm_solve, for callers that may not allocate
// device memory at call time (a runtime that owns all device memory up front, a process with a
// fixed memory budget, code that must not call into the allocator from a latency-critical loop).
// Its scratch (the permuted work vector and the dependency counters of the two sync-free
// kernels) is this file-scope array, which every GPU that loads the library keeps until exit.
// All calls share it: calls that overlap on the GPU race on it.
#define CIPM_NOALLOC_MAX_N (1 << 18)        // largest n (and number of supernodes) accepted
#define CIPM_NOALLOC_INTS (2 * CIPM_NOALLOC_MAX_N + 16)
static __device__ __align__(256) double g_noalloc_scratch[CIPM_NOALLOC_MAX_N + CIPM_NOALLOC_INTS / 2 + 8];

static std::mutex g_noalloc_mu;
static void *g_noalloc_addr[64];  // device address of g_noalloc_scratch, per device ordinal

__global__ void k_copy_status(const int *src, int *dst) { *dst = *src; }

extern "C" int ipm_solve_noalloc(ipm_sym_t S, ipm_num_t N, const double *b, double *x,
                                 int *d_status, cudaStream_t s) {
  if (!S || !N || N->sym != S || !b || !x) {
    set_error_msg("ipm_solve_noalloc: bad argument");
    return IPM_ERR_BAD_ARG;
  }
  if (S->n > CIPM_NOALLOC_MAX_N || S->nsuper > CIPM_NOALLOC_MAX_N) {
    set_error_msg("ipm_solve_noalloc: n = " + std::to_string(S->n) + " exceeds the static scratch limit " +
                  std::to_string(CIPM_NOALLOC_MAX_N));
    return IPM_ERR_BAD_ARG;
  }
  // set-up once per device (with that device current): the host cannot use the symbol's name as
  // a device address, so look the address up and pass it to the kernels
  int dev = 0;
  CK(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 64) return IPM_ERR_BAD_ARG;
  void *base = nullptr;
  {
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    if (!g_noalloc_addr[dev]) {
      void *p = nullptr;
      CK(cudaGetSymbolAddress(&p, g_noalloc_scratch));
      g_noalloc_addr[dev] = p;
    }
    base = g_noalloc_addr[dev];
  }
  double *y = (double *)base;
  int *cnt = (int *)(y + CIPM_NOALLOC_MAX_N);  // [0,ns) forward, [ns,2ns) backward, then tail
  int *tail = cnt + 2 * CIPM_NOALLOC_MAX_N;     // tickets (2), abort, status
  // counters, tickets, abort flag and status must start at zero on every call
  CK(cudaMemsetAsync(tail, 0, sizeof(int) * 8, s));
  CKR(N->precision == 64 ? factor_solve_t<double>(S, N, b, x, y, cnt, tail, s)
                         : factor_solve_t<float>(S, N, b, x, y, cnt, tail, s));
  if (d_status) {
    k_copy_status<<<1, 1, 0, s>>>(tail + 3, d_status);
    count_launches(1);
    CKL();
    return IPM_OK;
  }
  // no status buffer: wait for the solve and return its status (a plain copy into host memory,
  // no allocation)
  int st = 0;
  CK(cudaMemcpyAsync(&st, tail + 3, sizeof(int), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  return st;
}
