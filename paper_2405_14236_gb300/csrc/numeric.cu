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

#include "internal.cuh"

namespace cipm {

// ---------------------------------------------------------------- condensation
// K = W + diag(sigma_x) + delta_w I + J^T diag(d) J.  One block per supernode writes every slot
// of its panel as a fixed-order sum over the slot's items (sorted-pattern condensation).
__global__ void k_condense(const int *sptr, const int *srow_ptr, const int64_t *lptr,
                           const int *slot_ptr, const int2 *items, const int *J_rowidx,
                           const int *perm, const double *Wv, const double *sigma,
                           const double *Jv, const double *d, double dw, double *Lx) {
  int s = blockIdx.x;
  int f = sptr[s], w = sptr[s + 1] - f;
  int ld = srow_ptr[s + 1] - srow_ptr[s];
  int64_t base = lptr[s];
  int64_t area = (int64_t)ld * w;
  for (int64_t t = threadIdx.x; t < area; t += blockDim.x) {
    int c = (int)(t / ld), r = (int)(t - (int64_t)c * ld);
    int64_t slot = base + t;
    double v = 0.0;
    if (r >= c) {
      if (r == c) v = sigma[perm[f + c]] + dw;
      for (int it = slot_ptr[slot]; it < slot_ptr[slot + 1]; ++it) {
        int2 pq = items[it];
        if (pq.y < 0) v += Wv[pq.x];
        else v += d[J_rowidx[pq.x]] * Jv[pq.x] * Jv[pq.y];
      }
    }
    Lx[slot] = v;
  }
}

// ---------------------------------------------------------------- factorization
__device__ __forceinline__ int find_row(const int *rows, int ld, int i) {
  int lo = 0, hi = ld - 1;
  while (lo < hi) {
    int mid = (lo + hi) >> 1;
    if (rows[mid] < i) lo = mid + 1; else hi = mid;
  }
  return lo;
}

struct FactArgs {
  const int *level_sn, *sptr, *srow_ptr, *srow, *snode;
  const int64_t *lptr;
  double *Lx;
  int *info;
};

// One block per supernode of the level: dense right-looking Cholesky of the ld x w panel
// (diagonal block and the rows below it), then the update -L21 L21^T scattered into the
// ancestors' panels with FP64 atomics.
__global__ void __launch_bounds__(256) k_factor_level(FactArgs A, int lvl_begin) {
  const int s = A.level_sn[lvl_begin + blockIdx.x];
  const int f = A.sptr[s], w = A.sptr[s + 1] - f;
  const int rb = A.srow_ptr[s], ld = A.srow_ptr[s + 1] - rb;
  const int *rows = A.srow + rb;
  double *P = A.Lx + A.lptr[s];
  __shared__ double s_piv;
  for (int k = 0; k < w; ++k) {
    __syncthreads();
    if (threadIdx.x == 0) {
      double d = P[k + (int64_t)k * ld];
      if (!(d > 0.0) || !isfinite(d)) {
        atomicMin(A.info, f + k);
        d = 1.0;
      }
      double piv = sqrt(d);
      P[k + (int64_t)k * ld] = piv;
      s_piv = piv;
    }
    __syncthreads();
    const double inv = 1.0 / s_piv;
    double *colk = P + (int64_t)k * ld;
    for (int i = k + 1 + threadIdx.x; i < ld; i += blockDim.x) colk[i] *= inv;
    __syncthreads();
    const int nc = w - k - 1;
    const int64_t tot = (int64_t)nc * ld;
    for (int64_t t = threadIdx.x; t < tot; t += blockDim.x) {
      int j = k + 1 + (int)(t / ld);
      int i = (int)(t - (int64_t)(j - k - 1) * ld);
      if (i >= j) P[i + (int64_t)j * ld] -= colk[i] * colk[j];
    }
  }
  __syncthreads();
  const int B = ld - w;
  if (B <= 0) return;
  const int64_t npair = (int64_t)B * (B + 1) / 2;
  for (int64_t t = threadIdx.x; t < npair; t += blockDim.x) {
    // t -> (ii >= jj)
    int ii = (int)((sqrt(8.0 * (double)t + 1.0) - 1.0) * 0.5);
    while ((int64_t)(ii + 1) * (ii + 2) / 2 <= t) ++ii;
    while ((int64_t)ii * (ii + 1) / 2 > t) --ii;
    int jj = (int)(t - (int64_t)ii * (ii + 1) / 2);
    const int i = w + ii, j = w + jj;
    double v = 0.0;
    for (int k = 0; k < w; ++k) v += P[i + (int64_t)k * ld] * P[j + (int64_t)k * ld];
    const int col = rows[j], row = rows[i];
    const int ts = A.snode[col];
    const int tb = A.srow_ptr[ts], tld = A.srow_ptr[ts + 1] - tb;
    const int r = find_row(A.srow + tb, tld, row);
    atomicAdd(&A.Lx[A.lptr[ts] + (int64_t)(col - A.sptr[ts]) * tld + r], -v);
  }
}

// ---------------------------------------------------------------- triangular solves
__global__ void k_gather_perm(const int *perm, int n, const double *b, double *y) {
  int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k < n) y[k] = b[perm[k]];
}
__global__ void k_scatter_perm(const int *perm, int n, const double *y, double *x) {
  int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k < n) x[perm[k]] = y[k];
}

struct SolveArgs {
  const int *level_sn, *sptr, *srow_ptr, *srow;
  const int64_t *lptr;
  const double *Lx;
  double *y;
};

// forward: y_s = L11^{-1} y_s, then y[rows below] -= L21 y_s
__global__ void __launch_bounds__(128) k_fwd_level(SolveArgs A, int lvl_begin) {
  const int s = A.level_sn[lvl_begin + blockIdx.x];
  const int f = A.sptr[s], w = A.sptr[s + 1] - f;
  const int rb = A.srow_ptr[s], ld = A.srow_ptr[s + 1] - rb;
  const int *rows = A.srow + rb;
  const double *P = A.Lx + A.lptr[s];
  __shared__ double ys[CIPM_SN_MAXW];
  for (int k = threadIdx.x; k < w; k += blockDim.x) ys[k] = A.y[f + k];
  __syncthreads();
  if (threadIdx.x < 32) {
    const int lane = threadIdx.x;
    for (int k = 0; k < w; ++k) {
      if (lane == (k & 31)) ys[k] /= P[k + (int64_t)k * ld];
      __syncwarp();
      const double yk = ys[k];
      for (int i = k + 1 + lane; i < w; i += 32) ys[i] -= P[i + (int64_t)k * ld] * yk;
      __syncwarp();
    }
  }
  __syncthreads();
  for (int k = threadIdx.x; k < w; k += blockDim.x) A.y[f + k] = ys[k];
  for (int i = w + threadIdx.x; i < ld; i += blockDim.x) {
    double t = 0.0;
    for (int k = 0; k < w; ++k) t += P[i + (int64_t)k * ld] * ys[k];
    atomicAdd(&A.y[rows[i]], -t);
  }
}

// backward: y_s = L11^{-T} (y_s - L21^T y[rows below])
__global__ void __launch_bounds__(128) k_bwd_level(SolveArgs A, int lvl_begin) {
  const int s = A.level_sn[lvl_begin + blockIdx.x];
  const int f = A.sptr[s], w = A.sptr[s + 1] - f;
  const int rb = A.srow_ptr[s], ld = A.srow_ptr[s + 1] - rb;
  const int *rows = A.srow + rb;
  const double *P = A.Lx + A.lptr[s];
  __shared__ double zs[CIPM_SN_MAXW];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  for (int k = warp; k < w; k += nw) {
    double acc = 0.0;
    for (int i = w + lane; i < ld; i += 32) acc += P[i + (int64_t)k * ld] * A.y[rows[i]];
    acc = warp_sum(acc);
    if (lane == 0) zs[k] = A.y[f + k] - acc;
  }
  __syncthreads();
  if (threadIdx.x < 32) {
    for (int k = w - 1; k >= 0; --k) {
      if (lane == (k & 31)) zs[k] /= P[k + (int64_t)k * ld];
      __syncwarp();
      const double xk = zs[k];
      for (int j = lane; j < k; j += 32) zs[j] -= P[k + (int64_t)j * ld] * xk;
      __syncwarp();
    }
  }
  __syncthreads();
  for (int k = threadIdx.x; k < w; k += blockDim.x) A.y[f + k] = zs[k];
}

// ---------------------------------------------------------------- sparse products
// out = alpha * out_init + J^T (wt o u) where wt = d (if given) and only rows >= row_from count.
__global__ void k_jt_apply(int n, const int *JT_ptr, const int *JT_ent, const int *J_rowidx,
                           const double *Jv, const double *d, const double *u, int row_from,
                           int row_to, const double *base, double sign, double *out) {
  int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  double acc = 0.0;
  for (int t = JT_ptr[j]; t < JT_ptr[j + 1]; ++t) {
    int p = JT_ent[t];
    int r = J_rowidx[p];
    if (r < row_from || r >= row_to) continue;
    double v = Jv[p] * u[r];
    if (d) v *= d[r];
    acc += v;
  }
  out[j] = (base ? base[j] : 0.0) + sign * acc;
}

// out[r] = (J x)[r] for rows [row_from, row_to) (out indexed from 0)
__global__ void k_j_apply(int row_from, int row_to, const int *J_rowptr, const int *J_colind,
                          const double *Jv, const double *x, const double *sub, double *out) {
  int r = row_from + blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= row_to) return;
  double acc = 0.0;
  for (int p = J_rowptr[r]; p < J_rowptr[r + 1]; ++p) acc += Jv[p] * x[J_colind[p]];
  out[r - row_from] = acc - (sub ? sub[r - row_from] : 0.0);
}

// ---------------------------------------------------------------- reductions
__device__ __forceinline__ void atomic_max_nonneg(double *addr, double v) {
  atomicMax((unsigned long long *)addr, (unsigned long long)__double_as_longlong(v));
}

// partial[b] = sum over the block's range of x.y
__global__ void k_dot_partial(const double *x, const double *y, int n, double *partial) {
  __shared__ double sh[32];
  double acc = 0.0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    acc += x[i] * y[i];
  acc = warp_sum(acc);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x < 32) {
    double v = threadIdx.x < (blockDim.x >> 5) ? sh[threadIdx.x] : 0.0;
    v = warp_sum(v);
    if (threadIdx.x == 0) partial[blockIdx.x] = v;
  }
}
__global__ void k_dot_final(const double *partial, int np, double *out) {
  __shared__ double sh[32];
  double acc = 0.0;
  for (int i = threadIdx.x; i < np; i += blockDim.x) acc += partial[i];
  acc = warp_sum(acc);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x < 32) {
    double v = threadIdx.x < (blockDim.x >> 5) ? sh[threadIdx.x] : 0.0;
    v = warp_sum(v);
    if (threadIdx.x == 0) *out = v;
  }
}

static constexpr int DOT_BLOCKS = 152;
static int dot(const double *x, const double *y, int n, double *partial, double *out,
               cudaStream_t s) {
  k_dot_partial<<<DOT_BLOCKS, 256, 0, s>>>(x, y, n, partial);
  CKL();
  k_dot_final<<<1, 256, 0, s>>>(partial, DOT_BLOCKS, out);
  CKL();
  return IPM_OK;
}

// ---------------------------------------------------------------- augmented residual
// res = rhs - A sol for A = [[W + diag(sigma) + dw I, J^T], [J, -E]] where E_r = 1/d_r for
// rows r >= m_e and 0 for r < m_e.  Also max-norms of res, sol, rhs and (optionally) the
// row sums |A| into scal[0..3].
struct AugArgs {
  int n, m, m_e;
  const int *J_rowptr, *J_colind, *J_rowidx, *JT_ptr, *JT_ent;
  const int *W_rowptr, *W_colind, *W_rowidx, *WT_ptr, *WT_ent;
  const double *Wv, *sigma, *Jv, *d;
  double dw;
  const double *sx, *sz;    // solution parts
  const double *ra, *rb;    // rhs parts
  double *outx, *outz;      // residual parts
  double *scal;             // [0] ||res||, [1] ||sol||, [2] ||rhs||, [3] ||A||
  int want_norm_a;
};

__global__ void k_aug_resid_x(AugArgs A) {
  int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= A.n) return;
  double acc = (A.sigma[j] + A.dw) * A.sx[j];
  double asum = 0.0;
  double diag = A.sigma[j] + A.dw;
  for (int p = A.W_rowptr[j]; p < A.W_rowptr[j + 1]; ++p) {
    int c = A.W_colind[p];
    acc += A.Wv[p] * A.sx[c];
    if (c == j) diag += A.Wv[p];
    else asum += fabs(A.Wv[p]);
  }
  for (int t = A.WT_ptr[j]; t < A.WT_ptr[j + 1]; ++t) {
    int e = A.WT_ent[t];
    int r = A.W_rowidx[e];
    if (r == j) continue;
    acc += A.Wv[e] * A.sx[r];
    asum += fabs(A.Wv[e]);
  }
  asum += fabs(diag);
  for (int t = A.JT_ptr[j]; t < A.JT_ptr[j + 1]; ++t) {
    int p = A.JT_ent[t];
    acc += A.Jv[p] * A.sz[A.J_rowidx[p]];
    asum += fabs(A.Jv[p]);
  }
  double res = A.ra[j] - acc;
  A.outx[j] = res;
  atomic_max_nonneg(&A.scal[0], fabs(res));
  atomic_max_nonneg(&A.scal[1], fabs(A.sx[j]));
  atomic_max_nonneg(&A.scal[2], fabs(A.ra[j]));
  if (A.want_norm_a) atomic_max_nonneg(&A.scal[3], asum);
}

__global__ void k_aug_resid_z(AugArgs A) {
  int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= A.m) return;
  double acc = 0.0, asum = 0.0;
  for (int p = A.J_rowptr[r]; p < A.J_rowptr[r + 1]; ++p) {
    acc += A.Jv[p] * A.sx[A.J_colind[p]];
    asum += fabs(A.Jv[p]);
  }
  double e = r >= A.m_e ? 1.0 / A.d[r] : 0.0;
  acc -= e * A.sz[r];
  asum += fabs(e);
  double res = A.rb[r] - acc;
  A.outz[r] = res;
  atomic_max_nonneg(&A.scal[0], fabs(res));
  atomic_max_nonneg(&A.scal[1], fabs(A.sz[r]));
  atomic_max_nonneg(&A.scal[2], fabs(A.rb[r]));
  if (A.want_norm_a) atomic_max_nonneg(&A.scal[3], asum);
}

// elementwise helpers
__global__ void k_axpy(int n, double alpha, const double *x, double *y) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) y[i] += alpha * x[i];
}
// dz = d o (J dx - b) for rows [row_from, m): out indexed from row_from
__global__ void k_recover_dz(int row_from, int m, const int *J_rowptr, const int *J_colind,
                             const double *Jv, const double *d, const double *dx, const double *b,
                             double *dz) {
  int r = row_from + blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= m) return;
  double acc = 0.0;
  for (int p = J_rowptr[r]; p < J_rowptr[r + 1]; ++p) acc += Jv[p] * dx[J_colind[p]];
  dz[r - row_from] = d[r] * (acc - b[r]);
}

// CG updates with device-side scalars: scal[0] = rr, scal[1] = p.Sp, scal[2] = rr_new
__global__ void k_cg_update_xr(int n, const double *scal, const double *p, const double *Sp,
                               double *x, double *r) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double alpha = scal[0] / scal[1];
  x[i] += alpha * p[i];
  r[i] -= alpha * Sp[i];
}
__global__ void k_cg_update_p(int n, const double *scal, const double *r, double *p) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double beta = scal[2] / scal[0];
  p[i] = r[i] + beta * p[i];
}
__global__ void k_copy_scalar(const double *src, double *dst) { *dst = *src; }
__global__ void k_info_set(int *info) { *info = INT_MAX; }
__global__ void k_info_fix(int *info) {
  if (*info == INT_MAX) *info = -1;
}

}  // namespace cipm

using namespace cipm;

extern "C" int ipm_num_create(ipm_sym_t S, int precision, ipm_num_t *out) {
  if (!S || !out || precision != 64) {
    set_error_msg("ipm_num_create: bad argument (precision must be 64)");
    return IPM_ERR_BAD_ARG;
  }
  *out = nullptr;
  ipm_num_t N = new ipm_num_s();
  N->sym = S;
  N->precision = precision;
  int rc = dev_alloc(&N->Lx, S->panel_len);
  for (int k = 0; k < 8 && rc == IPM_OK; ++k) rc = dev_alloc(&N->vn[k], S->n);
  for (int k = 0; k < 6 && rc == IPM_OK; ++k) rc = dev_alloc(&N->vm[k], S->m > 0 ? S->m : 1);
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
  for (auto *p : N->vn)
    if (p) cudaFree(p);
  for (auto *p : N->vm)
    if (p) cudaFree(p);
  if (N->scal) cudaFree(N->scal);
  if (N->h_scal) cudaFreeHost(N->h_scal);
  delete N;
}

extern "C" int ipm_num_export(ipm_num_t N, double *Lx_host) {
  if (!N || !Lx_host) return IPM_ERR_BAD_ARG;
  CK(cudaDeviceSynchronize());
  CK(cudaMemcpy(Lx_host, N->Lx, sizeof(double) * N->sym->panel_len, cudaMemcpyDeviceToHost));
  return IPM_OK;
}

extern "C" int ipm_condense(ipm_sym_t S, ipm_num_t N, const double *W_val, const double *sigma_x,
                            const double *J_val, const double *d_row, double delta_w,
                            cudaStream_t s) {
  if (!S || !N || N->sym != S || !sigma_x || (S->nnzW && !W_val) || (S->nnzJ && (!J_val || !d_row)))
    return IPM_ERR_BAD_ARG;
  if (S->nsuper == 0) return IPM_OK;
  k_condense<<<S->nsuper, 128, 0, s>>>(S->sptr, S->srow_ptr, S->lptr, S->slot_ptr, S->items,
                                       S->J_rowidx, S->perm, W_val, sigma_x, J_val, d_row,
                                       delta_w, N->Lx);
  CKL();
  return IPM_OK;
}

extern "C" int ipm_factor(ipm_sym_t S, ipm_num_t N, int *d_info, cudaStream_t s) {
  if (!S || !N || N->sym != S || !d_info) return IPM_ERR_BAD_ARG;
  k_info_set<<<1, 1, 0, s>>>(d_info);
  CKL();
  FactArgs A{S->level_sn, S->sptr, S->srow_ptr, S->srow, S->snode, S->lptr, N->Lx, d_info};
  for (int L = 0; L < S->nlevels; ++L) {
    int b = S->h_level_ptr[L], e = S->h_level_ptr[L + 1];
    if (e > b) k_factor_level<<<e - b, 256, 0, s>>>(A, b);
  }
  CKL();
  k_info_fix<<<1, 1, 0, s>>>(d_info);
  CKL();
  return IPM_OK;
}

// y (permuted, length n) <- L^{-T} L^{-1} y in place
static int solve_permuted(ipm_sym_t S, ipm_num_t N, double *y, cudaStream_t s) {
  SolveArgs A{S->level_sn, S->sptr, S->srow_ptr, S->srow, S->lptr, N->Lx, y};
  for (int L = 0; L < S->nlevels; ++L) {
    int b = S->h_level_ptr[L], e = S->h_level_ptr[L + 1];
    if (e > b) k_fwd_level<<<e - b, 128, 0, s>>>(A, b);
  }
  for (int L = S->nlevels - 1; L >= 0; --L) {
    int b = S->h_level_ptr[L], e = S->h_level_ptr[L + 1];
    if (e > b) k_bwd_level<<<e - b, 128, 0, s>>>(A, b);
  }
  CKL();
  return IPM_OK;
}

// x = K^{-1} b (b, x of length n in the original order; may alias)
static int solve_full(ipm_sym_t S, ipm_num_t N, const double *b, double *x, cudaStream_t s) {
  double *y = N->vn[7];
  k_gather_perm<<<grid_for(S->n, 256), 256, 0, s>>>(S->perm, S->n, b, y);
  CKL();
  CKR(solve_permuted(S, N, y, s));
  k_scatter_perm<<<grid_for(S->n, 256), 256, 0, s>>>(S->perm, S->n, y, x);
  CKL();
  return IPM_OK;
}

extern "C" int ipm_solve(ipm_sym_t S, ipm_num_t N, const double *b, double *x, int nrhs,
                         cudaStream_t s) {
  if (!S || !N || N->sym != S || !b || !x || nrhs != 1) return IPM_ERR_BAD_ARG;
  return solve_full(S, N, b, x, s);
}

// condensed solve of the augmented system: dx = K^{-1}(ra + J^T (d o rb)), dz = d o (J dx - rb)
static int aug_condensed(ipm_sym_t S, ipm_num_t N, const double *Jv, const double *d,
                         const double *ra, const double *rb, double *dx, double *dz,
                         cudaStream_t s) {
  const int n = S->n, m = S->m;
  double *t = N->vn[6];
  k_jt_apply<<<grid_for(n, 256), 256, 0, s>>>(n, S->JT_ptr, S->JT_ent, S->J_rowidx, Jv, d, rb, 0,
                                              m, ra, 1.0, t);
  CKL();
  CKR(solve_full(S, N, t, dx, s));
  if (m > 0) {
    k_recover_dz<<<grid_for(m, 256), 256, 0, s>>>(0, m, S->J_rowptr, S->J_colind, Jv, d, dx, rb,
                                                  dz);
    CKL();
  }
  return IPM_OK;
}

extern "C" int ipm_aug_solve(ipm_sym_t S, ipm_num_t N, const double *W_val, const double *sigma_x,
                             const double *J_val, const double *d_row, double delta_w,
                             const double *a, const double *b, double *dx, double *dz,
                             int max_refine, double tol, double *d_eta, int *d_steps,
                             cudaStream_t s) {
  if (!S || !N || N->sym != S || !a || !dx || !sigma_x || (S->m && (!b || !dz || !d_row)) ||
      max_refine < 0)
    return IPM_ERR_BAD_ARG;
  const int n = S->n, m = S->m;
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
    CKL();
    if (m > 0) k_aug_resid_z<<<grid_for(m, 256), 256, 0, s>>>(A);
    CKL();
    CK(cudaMemcpyAsync(N->h_scal, N->scal, sizeof(double) * 4, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    if (it == 0) normA = N->h_scal[3];
    double den = normA * N->h_scal[1] + N->h_scal[2];
    eta = den > 0 ? N->h_scal[0] / den : 0.0;
    if (!std::isfinite(eta)) {
      eta_prev = eta;
      break;
    }
    if (eta <= tol || it >= max_refine || (it > 0 && eta > 0.5 * eta_prev)) break;
    eta_prev = eta;
    CKR(aug_condensed(S, N, J_val, d_row, A.outx, A.outz, cx, cz, s));
    k_axpy<<<grid_for(n, 256), 256, 0, s>>>(n, 1.0, cx, dx);
    CKL();
    if (m > 0) k_axpy<<<grid_for(m, 256), 256, 0, s>>>(m, 1.0, cz, dz);
    CKL();
    ++steps;
  }
  if (d_eta) CK(cudaMemcpyAsync(d_eta, &eta, sizeof(double), cudaMemcpyHostToDevice, s));
  if (d_steps) CK(cudaMemcpyAsync(d_steps, &steps, sizeof(int), cudaMemcpyHostToDevice, s));
  CK(cudaStreamSynchronize(s));
  if (!std::isfinite(eta)) return IPM_ERR_NONFINITE;
  return IPM_OK;
}

extern "C" int hykkt_cg(ipm_sym_t S, ipm_num_t N, int m_e, const double *J_val,
                        const double *d_row, double gamma, const double *a, const double *b,
                        double rtol, int maxit, double *dx, double *dy, double *dz, int *h_iters,
                        double *h_relres, cudaStream_t s) {
  const int n = S ? S->n : 0, m = S ? S->m : 0;
  if (!S || !N || N->sym != S || m_e < 0 || m_e > m || !a || !dx || (m && (!b || !d_row)) ||
      (m_e && !dy) || (m > m_e && !dz) || maxit < 0)
    return IPM_ERR_BAD_ARG;
  (void)gamma;  // gamma enters through d_row[0..m_e), the weights K_gamma was condensed with
  double *rhs1 = N->vn[0], *w = N->vn[1], *u = N->vn[2];
  double *r = N->vm[0], *p = N->vm[1], *Sp = N->vm[2];
  double *sc = N->scal, *partial = N->scal + 64;
  // rhs1 = a + J^T (d o b)  ( = r1 + gamma G^T r2 with r1 = a + H^T D_H b_H, r2 = b_G )
  k_jt_apply<<<grid_for(n, 256), 256, 0, s>>>(n, S->JT_ptr, S->JT_ent, S->J_rowidx, J_val, d_row,
                                              b, 0, m, a, 1.0, rhs1);
  CKL();
  CKR(solve_full(S, N, rhs1, w, s));
  int iters = 0;
  double relres = 0.0;
  int rc = IPM_OK;
  if (m_e > 0) {
    // r = G w - b_G ; dy = 0 ; p = r
    k_j_apply<<<grid_for(m_e, 256), 256, 0, s>>>(0, m_e, S->J_rowptr, S->J_colind, J_val, w, b, r);
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
      CKL();
      CKR(solve_full(S, N, u, u, s));
      k_j_apply<<<grid_for(m_e, 256), 256, 0, s>>>(0, m_e, S->J_rowptr, S->J_colind, J_val, u,
                                                   nullptr, Sp);
      CKL();
      CKR(dot(p, Sp, m_e, partial, sc + 1, s));
      k_cg_update_xr<<<grid_for(m_e, 256), 256, 0, s>>>(m_e, sc, p, Sp, dy, r);
      CKL();
      CKR(dot(r, r, m_e, partial, sc + 2, s));
      k_cg_update_p<<<grid_for(m_e, 256), 256, 0, s>>>(m_e, sc, r, p);
      CKL();
      k_copy_scalar<<<1, 1, 0, s>>>(sc + 2, sc + 0);
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
    CKL();
    CKR(solve_full(S, N, u, dx, s));
  } else {
    CK(cudaMemcpyAsync(dx, w, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
  }
  if (m > m_e) {
    k_recover_dz<<<grid_for(m - m_e, 256), 256, 0, s>>>(m_e, m, S->J_rowptr, S->J_colind, J_val,
                                                        d_row, dx, b, dz);
    CKL();
  }
  CK(cudaStreamSynchronize(s));
  if (h_iters) *h_iters = iters;
  if (h_relres) *h_relres = relres;
  return rc;
}
