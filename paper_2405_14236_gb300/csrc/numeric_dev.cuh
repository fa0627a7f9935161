// Device side of the numeric phase (condensation, sync-free supernodal Cholesky, triangular
// solves, sparse products, residuals), shared by the single-problem entry points (numeric.cu)
// and the batched ones (batch.cu).  Every translation unit that includes it holds its own copy
// of the device variables declared here.
//
// Storage: each supernode s (columns f..f+w-1, row list rows[0..ld) whose first w entries are
// its own columns) keeps a column-major ld x w panel at Lx + lptr[s].  After condensation the
// panels hold the lower triangle of P K P^T (fill zeroed); after the factorization they hold L
// below the diagonal block, and the diagonal factors L11 (with reciprocal pivots) live in Dx.
#pragma once
#include <climits>

#include "internal.cuh"

namespace cipm {
// internal linkage: every translation unit that includes this header gets its own kernels
namespace {

// ---------------------------------------------------------------- condensation
// K = W + diag(sigma_x) + delta_w I + J^T diag(d) J.  First t_p = d_row(p) J_p for every J entry
// (one FP64 multiply per entry), then one block per supernode writes every slot of its panel as a
// fixed-order sum over the slot's items t_p J_q (one FP64 FMA per item; on this GPU every FP64
// warp instruction costs the same, so the per-item instruction count is what matters).
__global__ void k_scale_jv(int nnz, const int *J_rowidx, const double *Jv, const double *d,
                           double *t) {
  int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p < nnz) t[p] = d[J_rowidx[p]] * Jv[p];
}

// The sums are formed in FP64 (they cancel heavily when D spans many orders of magnitude) and
// stored as T (T = float for the FP32 factorization path).
template <typename T>
__device__ __forceinline__ void condense_block(int s, const int *sptr, const int *srow_ptr,
                                               const int64_t *lptr, const int *slot_ptr,
                                               const int2 *items, const int *perm,
                                               const double *Wv, const double *sigma,
                                               const double *Jv, const double *tJ, double dw,
                                               T *Lx, int tid, int nthreads) {
  int f = sptr[s], w = sptr[s + 1] - f;
  int ld = srow_ptr[s + 1] - srow_ptr[s];
  int64_t base = lptr[s];
  int64_t area = (int64_t)ld * w;
  for (int64_t t = tid; t < area; t += nthreads) {
    int c = (int)(t / ld), r = (int)(t - (int64_t)c * ld);
    int64_t slot = base + t;
    double v = 0.0;
    if (r >= c) {
      if (r == c) v = sigma[perm[f + c]] + dw;
      for (int it = slot_ptr[slot]; it < slot_ptr[slot + 1]; ++it) {
        int2 pq = items[it];
        v = pq.y < 0 ? v + Wv[pq.x] : fma(tJ[pq.x], Jv[pq.y], v);
      }
      // single precision: the factored matrix gets a relative diagonal shift of 2^-20 so that
      // rounding K to FP32 cannot make a positive definite K indefinite; the FP64 refinement
      // multiplies by the unshifted K, so the shift only changes the preconditioner
      if (sizeof(T) == 4 && r == c) v += v * 9.5367431640625e-07;
    }
    Lx[slot] = (T)v;
  }
}

template <typename T>
__global__ void k_condense(const int *sptr, const int *srow_ptr, const int64_t *lptr,
                           const int *slot_ptr, const int2 *items, const int *perm,
                           const double *Wv, const double *sigma, const double *Jv,
                           const double *tJ, double dw, T *Lx) {
  condense_block<T>(blockIdx.x, sptr, srow_ptr, lptr, slot_ptr, items, perm, Wv, sigma, Jv, tJ,
                    dw, Lx, threadIdx.x, blockDim.x);
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

// A pivot is usable when it is positive and finite: tested on the bits (sign clear, not +0,
// exponent below all ones), which keeps the test off the FP64 pipe.
__device__ __forceinline__ bool pivot_ok(double d) {
  const long long b = __double_as_longlong(d);
  return b > 0 && (b >> 52) < 0x7ff;
}

__device__ __forceinline__ bool pivot_ok(float d) {
  const int b = __float_as_int(d);
  return b > 0 && (b >> 23) < 0xff;
}

// 1/sqrt(d) from a single-precision seed y (relative error e0 below 2^-21) and one third-order
// correction of the Newton-Raphson family for 1/sqrt: with e = 1 - d y^2, y <- y (1 + e/2 +
// 3 e^2 / 8), which leaves an error of order e0^3, below double rounding.  Six dependent FP64
// instructions (two conversions, four multiply-adds) instead of the ~11 of two quadratic steps:
// on this GPU every FP64 warp instruction costs 64 cycles, and the pivots of a supernode are a
// dependent chain.  Inputs outside [2^-100, 2^100] (exponent test on the bits) use sqrt and
// division.
__device__ __forceinline__ double rsqrt_newton(double d) {
  const long long b = __double_as_longlong(d);
  const long long ex = b >> 52;  // the pivots passed here are positive: no sign bit
  if (ex < 1023 - 100 || ex > 1023 + 100) return 1.0 / sqrt(d);
  const double y = (double)rsqrtf((float)d);
  const double e = fma(-d * y, y, 1.0);
  return fma(y * e, fma(0.375, e, 0.5), y);
}

// single precision: hardware rsqrt plus one Newton step
__device__ __forceinline__ float rsqrt_newton(float d) {
  float y = rsqrtf(d);
  return y * fmaf(-0.5f * d * y, y, 1.5f);
}

template <typename T>
__device__ __forceinline__ T warp_sum_t(T v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

template <typename T>
struct FactArgs {
  const int *level_sn, *sptr, *srow_ptr, *srow, *snode;
  const int64_t *lptr, *dptr;
  T *Lx, *Dx;
  int *info;
};

// ---------------------------------------------------------------- triangular solves
__global__ void k_gather_perm(const int *perm, int n, const double *b, double *y) {
  int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k < n) y[k] = b[perm[k]];
}
__global__ void k_scatter_perm(const int *perm, int n, const double *y, double *x) {
  int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k < n) x[perm[k]] = y[k];
}

// Triangular solves read factors stored as T and compute in FP64: with an FP32 factor the
// preconditioner (L L^T)^{-1} is then applied exactly, as preconditioned CG requires.
template <typename T>
struct SolveArgs {
  const int *level_sn, *sptr, *srow_ptr, *srow;
  const int64_t *lptr, *dptr;
  const T *Lx, *Dx;
  double *y;
};

// ---------------------------------------------------------------- sync-free scheduling
// Persistent kernels take tasks in one topological order through an atomic ticket.  A task
// waits (thread 0, bounded) until its dependency counter is complete, works, makes its writes
// visible (every thread fences, then a barrier) and signals its dependents.  A block only
// waits on tasks with smaller tickets, which running blocks already hold, so the schedule
// cannot deadlock.  Data written inside the same launch is read through L2 (__ldcg).
// A wait that exceeds the spin limit records IPM_ERR_TIMEOUT and raises an abort flag that
// makes every block stop taking tasks.
static __device__ long long g_spin_limit = 1ll << 23;  // polls of ~0.2 us each before giving up

struct SyncCtl {
  int *cnt;      // per-supernode counters (layout in ipm_num_s::sync)
  int *ticket;   // this kernel's ticket
  int *abort_;   // shared abort flag
  int *status;   // IPM_ERR_TIMEOUT on a timed-out wait
};

__device__ __forceinline__ int ld_acquire(const int *p) {
  int v;
  asm volatile("ld.acquire.gpu.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// thread 0 only: wait until *p >= need; false when aborted or timed out
__device__ bool spin_geq(const int *p, int need, const SyncCtl &C) {
  long long it = 0;
  while (ld_acquire(p) < need) {
    if (ld_acquire(C.abort_)) return false;
    if (++it > g_spin_limit) {
      atomicExch(C.status, IPM_ERR_TIMEOUT);
      atomicExch(C.abort_, 1);
      return false;
    }
    __nanosleep(128);
  }
  return true;
}

// every thread: make this thread's writes/atomics visible device-wide, then a barrier
__device__ __forceinline__ void publish() {
  __threadfence();
  __syncthreads();
}

template <typename T>
struct FactTaskArgs {
  FactArgs<T> F;
  const int4 *tasks;
  int ntasks;
  const int *upd_need;
  SyncCtl C;  // cnt: [0,ns) update arrivals, [ns,2ns) panel tasks done
  int ns;
};

// Panel task (supernode s, row block rb): the w x w diagonal block is factored in shared memory
// (every row block of s repeats this small Cholesky, so no block waits for a sibling), then
// L21 = A21 L11^{-T} for the block's <= 32 rows.  The diagonal block of the panel keeps K
// (siblings read it in the same launch); row block 0 stores L11 in the separate array Dx.
// The reciprocal pivots are computed once by one thread: FP64 division is expensive here.
template <typename V>
__device__ void fact_panel_task(const FactTaskArgs<V> &T, int s, int rb, V *sm, int *s_ok) {
  const FactArgs<V> &A = T.F;
  if (threadIdx.x == 0) *s_ok = spin_geq(T.C.cnt + s, T.upd_need[s], T.C);
  __syncthreads();
  if (!*s_ok) return;
  const int f = A.sptr[s], w = A.sptr[s + 1] - f;
  const int ld = A.srow_ptr[s + 1] - A.srow_ptr[s];
  V *P = A.Lx + A.lptr[s];
  V *sL = sm, *sR = sm + w * w;
  __shared__ V s_inv[CIPM_SN_MAXW];
  const int tid = threadIdx.x, bd = blockDim.x;
  for (int t = tid; t < w * w; t += bd) {
    int k = t / w, i = t - k * w;
    sL[t] = i >= k ? __ldcg(P + i + (int64_t)k * ld) : 0.0;
  }
  __syncthreads();
  for (int k = 0; k < w; ++k) {
    if (tid == 0) {
      V d = sL[k + k * w];
      if (!(d > 0.0) || !isfinite(d)) {
        atomicMin(A.info, f + k);
        d = 1.0;
      }
      const V inv = rsqrt_newton(d);
      sL[k + k * w] = d * inv;
      s_inv[k] = inv;
    }
    __syncthreads();
    const V inv = s_inv[k];
    const int nr = w - k - 1;
    for (int i = k + 1 + tid; i < w; i += bd) sL[i + k * w] *= inv;
    __syncthreads();
    // trailing update: warps own columns, lanes rows (no divisions in the loop)
    for (int jj = tid / 32; jj < nr; jj += bd / 32) {
      const int j = k + 1 + jj;
      const V ljk = sL[j + k * w];
      for (int i = j + (tid & 31); i < w; i += 32) sL[i + j * w] -= sL[i + k * w] * ljk;
    }
    __syncthreads();
  }
  if (rb == 0) {
    V *Dd = A.Dx + A.dptr[s];
    for (int t = tid; t < w * w; t += bd) Dd[t] = sL[t];
    for (int k = tid; k < w; k += bd) Dd[w * w + k] = s_inv[k];
  }
  const int r0 = w + rb * CIPM_RB;
  const int nrow = min(CIPM_RB, ld - r0);
  if (nrow > 0) {
    const int sw = w + 1;
    for (int t = tid; t < nrow * w; t += bd) {
      int k = t / nrow, r = t - k * nrow;
      sR[r * sw + k] = __ldcg(P + (r0 + r) + (int64_t)k * ld);
    }
    __syncthreads();
    // each warp owns rows r = warp, warp + nwarps, ...; lanes split the columns
    const int warp = tid >> 5, lane = tid & 31, nw = bd >> 5;
    for (int k = 0; k < w; ++k) {
      const V inv = s_inv[k];
      for (int r = warp; r < nrow; r += nw) {
        V xk = sR[r * sw + k] * inv;
        __syncwarp();
        for (int j = k + 1 + lane; j < w; j += 32) sR[r * sw + j] -= xk * sL[j + k * w];
        if (lane == 0) sR[r * sw + k] = xk;
        __syncwarp();
      }
    }
    __syncthreads();
    for (int t = tid; t < nrow * w; t += bd) {
      int k = t / nrow, r = t - k * nrow;
      P[(r0 + r) + (int64_t)k * ld] = sR[r * sw + k];
    }
  }
  publish();
  if (tid == 0) atomicAdd(T.C.cnt + T.ns + s, 1);
}

template <typename V>
__device__ void fact_update_task(const FactTaskArgs<V> &T, int s, int ti, int tj, V *sm,
                                 int *s_ok) {
  const FactArgs<V> &A = T.F;
  const int f = A.sptr[s], w = A.sptr[s + 1] - f;
  const int rbase = A.srow_ptr[s], ld = A.srow_ptr[s + 1] - rbase;
  const int B = ld - w;
  const int npanel = (B + CIPM_RB - 1) / CIPM_RB;
  if (threadIdx.x == 0) *s_ok = spin_geq(T.C.cnt + T.ns + s, npanel, T.C);
  __syncthreads();
  if (!*s_ok) return;
  const int *rows = A.srow + rbase;
  const V *P = A.Lx + A.lptr[s];
  const int sw = w + 1;
  V *sI = sm, *sJ = sm + CIPM_RB * sw;
  const int i0 = w + ti * CIPM_RB, ni = min(CIPM_RB, ld - i0);
  const int j0 = w + tj * CIPM_RB, nj = min(CIPM_RB, ld - j0);
  const int tid = threadIdx.x, bd = blockDim.x;
  for (int t = tid; t < ni * w; t += bd) {
    int k = t / ni, r = t - k * ni;
    sI[r * sw + k] = __ldcg(P + (i0 + r) + (int64_t)k * ld);
  }
  for (int t = tid; t < nj * w; t += bd) {
    int k = t / nj, r = t - k * nj;
    sJ[r * sw + k] = __ldcg(P + (j0 + r) + (int64_t)k * ld);
  }
  __syncthreads();
  for (int p = tid; p < ni * nj; p += bd) {
    const int ii = p / nj, jj = p - (p / nj) * nj;
    const int i = i0 + ii, j = j0 + jj;
    if (i < j) continue;
    const V *a = sI + ii * sw, *b = sJ + jj * sw;
    V v = 0.0;
    for (int k = 0; k < w; ++k) v += a[k] * b[k];
    const int col = rows[j], row = rows[i];
    const int ts = A.snode[col];
    const int tb = A.srow_ptr[ts], tld = A.srow_ptr[ts + 1] - tb;
    const int r = find_row(A.srow + tb, tld, row);
    atomicAdd(&A.Lx[A.lptr[ts] + (int64_t)(col - A.sptr[ts]) * tld + r], -v);
  }
  publish();
  // one signal per distinct target supernode of the tile's rows (runs, rows are sorted)
  if (tid < 32 && tid < nj) {
    const int j = j0 + tid;
    const int t = A.snode[rows[j]];
    const int tp = tid > 0 ? A.snode[rows[j - 1]] : -1;
    if (t != tp) atomicAdd(T.C.cnt + t, 1);
  }
}

template <typename V>
__global__ void __launch_bounds__(256) k_factor_dag(FactTaskArgs<V> T) {
  extern __shared__ __align__(16) unsigned char sm_raw[];
  V *sm = reinterpret_cast<V *>(sm_raw);
  __shared__ int s_t, s_ok;
  while (true) {
    if (threadIdx.x == 0) s_t = ld_acquire(T.C.abort_) ? T.ntasks : atomicAdd(T.C.ticket, 1);
    __syncthreads();
    const int t = s_t;
    __syncthreads();
    if (t >= T.ntasks) break;
    const int4 tk = T.tasks[t];
    if (tk.w == 0) fact_panel_task(T, tk.x, tk.y, sm, &s_ok);
    else fact_update_task(T, tk.x, tk.y, tk.z, sm, &s_ok);
    __syncthreads();
  }
}

template <typename V>
struct SolveTaskArgs {
  SolveArgs<V> A;
  const int *snode;
  const int *fwd_need;
  SyncCtl C;  // cnt: forward arrivals (fwd) or backward done flags (bwd)
  int ns;
};

// forward solve of supernode s: wait for every contribution into y_s, solve with L11, push
// L21 y_s into the rows below (block of 128 threads; sL: w*w doubles of shared memory)
template <typename V>
__device__ void fwd_task(const SolveTaskArgs<V> &T, int s, double *sL, double *ys, int *s_ok) {
  const SolveArgs<V> &A = T.A;
  if (threadIdx.x == 0) *s_ok = spin_geq(T.C.cnt + s, T.fwd_need[s], T.C);
  __syncthreads();
  if (!*s_ok) return;
  const int f = A.sptr[s], w = A.sptr[s + 1] - f;
  const int rb = A.srow_ptr[s], ld = A.srow_ptr[s + 1] - rb;
  const int *rows = A.srow + rb;
  const V *P = A.Lx + A.lptr[s];
  const V *Dd = A.Dx + A.dptr[s];
  for (int q = threadIdx.x; q < w * w; q += blockDim.x) sL[q] = (double)Dd[q];
  for (int k = threadIdx.x; k < w; k += blockDim.x) ys[k] = __ldcg(A.y + f + k);
  __syncthreads();
  if (threadIdx.x < 32) {
    const int lane = threadIdx.x;
    const V *rinv = Dd + w * w;
    for (int k = 0; k < w; ++k) {
      if (lane == (k & 31)) ys[k] *= (double)rinv[k];
      __syncwarp();
      const double yk = ys[k];
      for (int i = k + 1 + lane; i < w; i += 32) ys[i] -= sL[i + k * w] * yk;
      __syncwarp();
    }
  }
  __syncthreads();
  for (int k = threadIdx.x; k < w; k += blockDim.x) A.y[f + k] = ys[k];
  for (int i = w + threadIdx.x; i < ld; i += blockDim.x) {
    double acc = 0.0;
    for (int k = 0; k < w; ++k) acc += (double)P[i + (int64_t)k * ld] * ys[k];
    atomicAdd(&A.y[rows[i]], -acc);
  }
  publish();
  for (int i = w + threadIdx.x; i < ld; i += blockDim.x) {
    const int tg = T.snode[rows[i]];
    const int tp = i > w ? T.snode[rows[i - 1]] : -1;
    if (tg != tp) atomicAdd(T.C.cnt + tg, 1);
  }
}

// backward solve of supernode s: wait until every supernode holding rows below s is done
template <typename V>
__device__ void bwd_task(const SolveTaskArgs<V> &T, int s, double *sL, double *zs, int *s_ok) {
  const SolveArgs<V> &A = T.A;
  const int f = A.sptr[s], w = A.sptr[s + 1] - f;
  const int rb = A.srow_ptr[s], ld = A.srow_ptr[s + 1] - rb;
  const int *rows = A.srow + rb;
  if (threadIdx.x == 0) *s_ok = 1;
  __syncthreads();
  for (int i = w + threadIdx.x; i < ld; i += blockDim.x) {
    const int tg = T.snode[rows[i]];
    const int tp = i > w ? T.snode[rows[i - 1]] : -1;
    if (tg != tp && !spin_geq(T.C.cnt + tg, 1, T.C)) *s_ok = 0;
  }
  __syncthreads();
  if (!*s_ok) return;
  const V *P = A.Lx + A.lptr[s];
  const V *Dd = A.Dx + A.dptr[s];
  for (int q = threadIdx.x; q < w * w; q += blockDim.x) sL[q] = (double)Dd[q];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  for (int k = warp; k < w; k += nw) {
    double acc = 0.0;
    for (int i = w + lane; i < ld; i += 32) acc += (double)P[i + (int64_t)k * ld] * __ldcg(A.y + rows[i]);
    acc = warp_sum(acc);
    if (lane == 0) zs[k] = __ldcg(A.y + f + k) - acc;
  }
  __syncthreads();
  if (threadIdx.x < 32) {
    const V *rinv = Dd + w * w;
    for (int k = w - 1; k >= 0; --k) {
      if (lane == (k & 31)) zs[k] *= (double)rinv[k];
      __syncwarp();
      const double xk = zs[k];
      for (int j = lane; j < k; j += 32) zs[j] -= sL[k + j * w] * xk;
      __syncwarp();
    }
  }
  __syncthreads();
  for (int k = threadIdx.x; k < w; k += blockDim.x) A.y[f + k] = zs[k];
  publish();
  if (threadIdx.x == 0) atomicExch(T.C.cnt + s, 1);
}

template <typename V>
__global__ void __launch_bounds__(128) k_fwd_dag(SolveTaskArgs<V> T) {
  extern __shared__ __align__(16) unsigned char sm_raw[];
  double *sL = reinterpret_cast<double *>(sm_raw);
  __shared__ double ys[CIPM_SN_MAXW];
  __shared__ int s_t, s_ok;
  while (true) {
    if (threadIdx.x == 0) s_t = ld_acquire(T.C.abort_) ? T.ns : atomicAdd(T.C.ticket, 1);
    __syncthreads();
    const int t = s_t;
    __syncthreads();
    if (t >= T.ns) break;
    fwd_task(T, T.A.level_sn[t], sL, ys, &s_ok);
    __syncthreads();
  }
}

template <typename V>
__global__ void __launch_bounds__(128) k_bwd_dag(SolveTaskArgs<V> T) {
  extern __shared__ __align__(16) unsigned char sm_raw[];
  double *sL = reinterpret_cast<double *>(sm_raw);
  __shared__ double zs[CIPM_SN_MAXW];
  __shared__ int s_t, s_ok;
  while (true) {
    if (threadIdx.x == 0) s_t = ld_acquire(T.C.abort_) ? T.ns : atomicAdd(T.C.ticket, 1);
    __syncthreads();
    const int t = s_t;
    __syncthreads();
    if (t >= T.ns) break;
    bwd_task(T, T.A.level_sn[T.ns - 1 - t], sL, zs, &s_ok);
    __syncthreads();
  }
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

__device__ __forceinline__ double warp_max(double v) {
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

// max over the block of v, then one atomic per block (all threads must call)
__device__ __forceinline__ void block_max_to(double *addr, double v, double *sh) {
  v = warp_max(v);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x < 32) {
    double x = threadIdx.x < (blockDim.x >> 5) ? sh[threadIdx.x] : 0.0;
    x = warp_max(x);
    if (threadIdx.x == 0) atomic_max_nonneg(addr, x);
  }
  __syncthreads();
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
  count_launches(1);
  CKL();
  k_dot_final<<<1, 256, 0, s>>>(partial, DOT_BLOCKS, out);
  count_launches(1);
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

// residual row j of the x block: returns res and accumulates |row| of A into *asum
__device__ __forceinline__ double aug_resid_x_at(const AugArgs &A, int j, double *asum_out) {
  double acc = (A.sigma[j] + A.dw) * A.sx[j];
  double diag = A.sigma[j] + A.dw, asum = 0.0;
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
  *asum_out = asum;
  return A.ra[j] - acc;
}

// residual row r of the z block
__device__ __forceinline__ double aug_resid_z_at(const AugArgs &A, int r, double *asum_out) {
  double acc = 0.0, asum = 0.0;
  for (int p = A.J_rowptr[r]; p < A.J_rowptr[r + 1]; ++p) {
    acc += A.Jv[p] * A.sx[A.J_colind[p]];
    asum += fabs(A.Jv[p]);
  }
  double e = r >= A.m_e ? 1.0 / A.d[r] : 0.0;
  acc -= e * A.sz[r];
  asum += fabs(e);
  *asum_out = asum;
  return A.rb[r] - acc;
}

__global__ void k_aug_resid_x(AugArgs A) {
  __shared__ double sh[32];
  int j = blockIdx.x * blockDim.x + threadIdx.x;
  double res = 0.0, solv = 0.0, rhsv = 0.0, asum = 0.0;
  if (j < A.n) {
    res = aug_resid_x_at(A, j, &asum);
    A.outx[j] = res;
    solv = fabs(A.sx[j]);
    rhsv = fabs(A.ra[j]);
  }
  block_max_to(&A.scal[0], fabs(res), sh);
  block_max_to(&A.scal[1], solv, sh);
  block_max_to(&A.scal[2], rhsv, sh);
  if (A.want_norm_a) block_max_to(&A.scal[3], asum, sh);
}

__global__ void k_aug_resid_z(AugArgs A) {
  __shared__ double sh[32];
  int r = blockIdx.x * blockDim.x + threadIdx.x;
  double res = 0.0, solv = 0.0, rhsv = 0.0, asum = 0.0;
  if (r < A.m) {
    res = aug_resid_z_at(A, r, &asum);
    A.outz[r] = res;
    solv = fabs(A.sz[r]);
    rhsv = fabs(A.rb[r]);
  }
  block_max_to(&A.scal[0], fabs(res), sh);
  block_max_to(&A.scal[1], solv, sh);
  block_max_to(&A.scal[2], rhsv, sh);
  if (A.want_norm_a) block_max_to(&A.scal[3], asum, sh);
}

// elementwise helpers
__global__ void k_axpy(int n, double alpha, const double *x, double *y) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) y[i] += alpha * x[i];
}
__global__ void k_scale(int n, double alpha, double *x) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) x[i] *= alpha;
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
__global__ void k_info_fix(int *info, const int *status) {
  if (*status != 0) *info = -2;  // a bounded device wait gave up
  else if (*info == INT_MAX) *info = -1;
}

}  // namespace
}  // namespace cipm
