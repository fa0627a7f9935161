// Multilayer perceptron for the learned warm start: BF16 weights and activations, FP32
// accumulation, GELU hidden layers, linear output, mean-squared-error loss, Adam.
//
// Layers l = 0 .. L-1 map width dims[l] to dims[l+1]: Z_l = A_l W_l + b_l with A_0 = bf16(X),
// A_{l+1} = bf16(gelu(Z_l)) for l < L-1 and Y = Z_{L-1}.  W_l is dims[l] x dims[l+1] row-major.
// The products run on the tensor cores (mma.sync m16n8k16, BF16 inputs, FP32 accumulators);
// FP32 master weights are updated by Adam and rounded to the BF16 copies the products read.
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <vector>

#include "common.cuh"

namespace cipm {
namespace {

using bf16 = __nv_bfloat16;

// C[M x N] (FP32, row-major, ldc) = opA[M x K] opB[K x N] with BF16 operands.
// TA: A is stored K x M (row-major, lda), else M x K.  TB: B is stored N x K, else K x N.
// 128 x 128 x 32 block tiles, 8 warps of 64 x 32, mma.sync m16n8k16 with ldmatrix fragment
// loads from shared memory (A as [m][k], B as [n][k]); the next k-tile is fetched into registers
// (16-byte loads where the row is aligned and in bounds, element loads at the edges) while the
// current one is multiplied, then stored to the other shared buffer.
constexpr int GBM = 128, GBN = 128, GBK = 32, GPAD = 8, GLD = GBK + GPAD;

// 8 consecutive bf16 of a row (contiguous in memory) starting at column c0, zero beyond len
__device__ __forceinline__ uint4 load8(const bf16 *row, int c0, int len, bool aligned) {
  if (aligned && c0 + 8 <= len) return *reinterpret_cast<const uint4 *>(row + c0);
  union {
    uint4 v;
    bf16 h[8];
  } u;
#pragma unroll
  for (int i = 0; i < 8; ++i) u.h[i] = c0 + i < len ? row[c0 + i] : __float2bfloat16(0.f);
  return u.v;
}

// one operand tile (128 rows of the [row][k] smem layout x 32 k) as two 16-byte chunks per
// thread.  Contiguous-k storage: chunk = (row, 8 k).  Transposed storage (contiguous along
// rows): chunk = (8 rows, k), scattered to the smem layout at store time.
template <bool KCONTIG>
__device__ __forceinline__ void tile_load(const bf16 *X, int ldx, int rows, int K, int r0, int k0,
                                          bool aligned, uint4 (&buf)[2]) {
#pragma unroll
  for (int q = 0; q < 2; ++q) {
    const int c = threadIdx.x + q * 256;
    if (KCONTIG) {
      const int r = c >> 2, kk = (c & 3) * 8;
      buf[q] = r0 + r < rows ? load8(X + (size_t)(r0 + r) * ldx, k0 + kk, K, aligned)
                             : make_uint4(0, 0, 0, 0);
    } else {
      const int kk = c >> 4, r = (c & 15) * 8;
      buf[q] = k0 + kk < K ? load8(X + (size_t)(k0 + kk) * ldx, r0 + r, rows, aligned)
                           : make_uint4(0, 0, 0, 0);
    }
  }
}

template <bool KCONTIG>
__device__ __forceinline__ void tile_store(bf16 (*S)[GLD], const uint4 (&buf)[2]) {
#pragma unroll
  for (int q = 0; q < 2; ++q) {
    const int c = threadIdx.x + q * 256;
    if (KCONTIG) {
      const int r = c >> 2, kk = (c & 3) * 8;
      *reinterpret_cast<uint4 *>(&S[r][kk]) = buf[q];
    } else {
      const int kk = c >> 4, r = (c & 15) * 8;
      union {
        uint4 v;
        bf16 h[8];
      } u;
      u.v = buf[q];
#pragma unroll
      for (int i = 0; i < 8; ++i) S[r + i][kk] = u.h[i];
    }
  }
}

__device__ __forceinline__ void ldsm_x4(uint32_t (&r)[4], const bf16 *p) {
  const uint32_t a = (uint32_t)__cvta_generic_to_shared(p);
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];\n"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
               : "r"(a));
}

// split K: block z multiplies k-tiles [z kchunk, (z + 1) kchunk) and adds its partial sums into
// C (zeroed by the caller) when gridDim.z > 1
template <bool TA, bool TB>
__global__ void __launch_bounds__(256) k_gemm_bf16(int M, int N, int K, const bf16 *A, int lda,
                                                   const bf16 *B, int ldb, float *C, int ldc,
                                                   int kchunk) {
  __shared__ __align__(16) bf16 As[2][GBM][GLD];
  __shared__ __align__(16) bf16 Bs[2][GBN][GLD];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int wm = warp >> 2, wn = warp & 3;  // 2 x 4 warps of 64 x 32
  const int m0 = blockIdx.y * GBM, n0 = blockIdx.x * GBN;
  // A rows are m (contiguous k unless TA), B rows are n (contiguous k when TB)
  const bool a_al = (lda % 8) == 0 && ((uintptr_t)A % 16) == 0;
  const bool b_al = (ldb % 8) == 0 && ((uintptr_t)B % 16) == 0;
  float acc[4][4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j)
#pragma unroll
      for (int q = 0; q < 4; ++q) acc[i][j][q] = 0.f;
  uint4 ra[2], rb[2];
  const int t0 = blockIdx.z * kchunk;
  const int nk = min((K + GBK - 1) / GBK, t0 + kchunk);
  if (t0 >= nk) return;
  tile_load<!TA>(A, lda, M, K, m0, t0 * GBK, a_al, ra);
  tile_load<TB>(B, ldb, N, K, n0, t0 * GBK, b_al, rb);
  tile_store<!TA>(As[0], ra);
  tile_store<TB>(Bs[0], rb);
  __syncthreads();
  for (int t = t0; t < nk; ++t) {
    const int cur = (t - t0) & 1;
    if (t + 1 < nk) {
      tile_load<!TA>(A, lda, M, K, m0, (t + 1) * GBK, a_al, ra);
      tile_load<TB>(B, ldb, N, K, n0, (t + 1) * GBK, b_al, rb);
    }
#pragma unroll
    for (int kk = 0; kk < GBK; kk += 16) {
      uint32_t af[4][4], bfr[2][4];
#pragma unroll
      for (int i = 0; i < 4; ++i)
        ldsm_x4(af[i], &As[cur][wm * 64 + i * 16 + (lane & 15)][kk + (lane >> 4) * 8]);
#pragma unroll
      for (int j = 0; j < 2; ++j)
        ldsm_x4(bfr[j], &Bs[cur][wn * 32 + j * 16 + (lane & 7) + ((lane >> 4) << 3)]
                            [kk + ((lane >> 3) & 1) * 8]);
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const uint32_t b0 = bfr[j >> 1][(j & 1) * 2], b1 = bfr[j >> 1][(j & 1) * 2 + 1];
          asm volatile(
              "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, "
              "{%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};\n"
              : "+f"(acc[i][j][0]), "+f"(acc[i][j][1]), "+f"(acc[i][j][2]), "+f"(acc[i][j][3])
              : "r"(af[i][0]), "r"(af[i][1]), "r"(af[i][2]), "r"(af[i][3]), "r"(b0), "r"(b1));
        }
    }
    if (t + 1 < nk) {
      tile_store<!TA>(As[cur ^ 1], ra);
      tile_store<TB>(Bs[cur ^ 1], rb);
    }
    __syncthreads();
  }
  const int g = lane >> 2, q4 = lane & 3;
  const bool split = gridDim.z > 1;
  auto put = [&](int r, int c, float v) {
    float *p = C + (size_t)r * ldc + c;
    if (split) atomicAdd(p, v);
    else *p = v;
  };
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int r = m0 + wm * 64 + i * 16 + g, c = n0 + wn * 32 + j * 8 + q4 * 2;
      if (r < M) {
        if (c < N) put(r, c, acc[i][j][0]);
        if (c + 1 < N) put(r, c + 1, acc[i][j][1]);
      }
      if (r + 8 < M) {
        if (c < N) put(r + 8, c, acc[i][j][2]);
        if (c + 1 < N) put(r + 8, c + 1, acc[i][j][3]);
      }
    }
}

// gelu(z) = z Phi(z), Phi the standard normal distribution function
__device__ __forceinline__ float gelu(float z) { return 0.5f * z * (1.f + erff(z * 0.70710678118654752f)); }
__device__ __forceinline__ float gelu_grad(float z) {
  return 0.5f * (1.f + erff(z * 0.70710678118654752f)) +
         z * 0.39894228040143268f * expf(-0.5f * z * z);
}

__global__ void k_to_bf16(int64_t n, const float *x, bf16 *y) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    y[i] = __float2bfloat16(x[i]);
}

// Z += b (per column); A = bf16(gelu(Z)) when gelu, else Y = Z
__global__ void k_bias_act(int rows, int cols, float *Z, const float *b, bf16 *A, int act,
                           float *Y) {
  const int64_t n = (int64_t)rows * cols;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const float z = Z[i] + b[i % cols];
    Z[i] = z;
    if (act) A[i] = __float2bfloat16(gelu(z));
    else if (Y) Y[i] = z;
  }
}

// d = scale (Y - T): dZ (FP32 and BF16); loss += sum (Y - T)^2 / count
__global__ void k_mse_grad(int64_t n, const float *Y, const float *T, float scale, float inv_count,
                           float *dZf, bf16 *dZb, float *loss) {
  __shared__ float sh[32];
  float acc = 0.f;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const float d = Y[i] - T[i];
    acc += d * d;
    const float gd = scale * d;
    dZf[i] = gd;
    dZb[i] = __float2bfloat16(gd);
  }
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x < 32) {
    float v = threadIdx.x < (blockDim.x >> 5) ? sh[threadIdx.x] : 0.f;
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (threadIdx.x == 0) atomicAdd(loss, v * inv_count);
  }
}

// gb[j] = sum_i dZ[i][j]
__global__ void k_col_sum(int rows, int cols, const float *dZ, float *gb) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= cols) return;
  float s = 0.f;
  for (int i = 0; i < rows; ++i) s += dZ[(size_t)i * cols + j];
  gb[j] = s;
}

// dZ = dA * gelu'(Z) (FP32 and BF16)
__global__ void k_gelu_back(int64_t n, const float *dA, const float *Z, float *dZf, bf16 *dZb) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const float d = dA[i] * gelu_grad(Z[i]);
    dZf[i] = d;
    dZb[i] = __float2bfloat16(d);
  }
}

// Adam (Kingma & Ba) on the FP32 master copy, then the BF16 copy (wb may be null for biases)
__global__ void k_adam(int64_t n, float *w, const float *g, float *m, float *v, bf16 *wb, float lr,
                       float b1, float b2, float eps, float c1, float c2) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    const float wi = w[i] - lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    w[i] = wi;
    if (wb) wb[i] = __float2bfloat16(wi);
  }
}

// rows of the batch: out[r] = src[idx[r]] (row length cols)
__global__ void k_gather_rows(int rows, int cols, const int *idx, const float *src, float *out) {
  const int r = blockIdx.y;
  if (r >= rows) return;
  const float *s = src + (size_t)idx[r] * cols;
  float *o = out + (size_t)r * cols;
  for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < cols; c += gridDim.x * blockDim.x) o[c] = s[c];
}

int grid_elems(int64_t n) { return (int)std::min<int64_t>((n + 255) / 256, 152 * 16); }

}  // namespace
}  // namespace cipm

using namespace cipm;

struct mlp_s {
  int L = 0, max_batch = 0;
  std::vector<int> dims;
  std::vector<float *> W, b, gW, gb, mW, vW, mb, vb, Z, dZf;
  std::vector<bf16 *> Wb, A, dZb;
  float *dA = nullptr;
  std::vector<void *> all;
};

template <typename T>
static int m_alloc(mlp_t P, T **p, int64_t n) {
  if (cudaMalloc((void **)p, sizeof(T) * (size_t)std::max<int64_t>(n, 1)) != cudaSuccess) {
    set_error_msg("mlp: out of device memory");
    return IPM_ERR_OOM;
  }
  P->all.push_back(*p);
  CK(cudaMemset(*p, 0, sizeof(T) * (size_t)std::max<int64_t>(n, 1)));
  return IPM_OK;
}

extern "C" void mlp_destroy(mlp_t P) {
  if (!P) return;
  for (void *p : P->all) cudaFree(p);
  delete P;
}

extern "C" int mlp_create(int nlayers, const int *dims, int max_batch, mlp_t *out) {
  if (nlayers < 1 || !dims || max_batch < 1 || !out) return IPM_ERR_BAD_ARG;
  for (int l = 0; l <= nlayers; ++l)
    if (dims[l] < 1) return IPM_ERR_BAD_ARG;
  *out = nullptr;
  mlp_t P = new mlp_s();
  P->L = nlayers;
  P->max_batch = max_batch;
  P->dims.assign(dims, dims + nlayers + 1);
  int rc = IPM_OK;
  int maxw = 0;
  for (int l = 0; l <= nlayers; ++l) maxw = std::max(maxw, dims[l]);
  auto F = [&](std::vector<float *> &v, int64_t n) {
    float *p = nullptr;
    if (rc == IPM_OK) rc = m_alloc(P, &p, n);
    v.push_back(p);
  };
  auto H = [&](std::vector<bf16 *> &v, int64_t n) {
    bf16 *p = nullptr;
    if (rc == IPM_OK) rc = m_alloc(P, &p, n);
    v.push_back(p);
  };
  for (int l = 0; l < nlayers; ++l) {
    const int64_t k = dims[l], n = dims[l + 1];
    F(P->W, k * n); F(P->b, n); F(P->gW, k * n); F(P->gb, n); F(P->mW, k * n); F(P->vW, k * n);
    F(P->mb, n); F(P->vb, n); F(P->Z, (int64_t)max_batch * n); F(P->dZf, (int64_t)max_batch * n);
    H(P->Wb, k * n); H(P->A, (int64_t)max_batch * k); H(P->dZb, (int64_t)max_batch * n);
  }
  if (rc == IPM_OK) rc = m_alloc(P, &P->dA, (int64_t)max_batch * maxw);
  if (rc != IPM_OK) {
    mlp_destroy(P);
    return rc;
  }
  *out = P;
  return IPM_OK;
}

extern "C" int mlp_param_count(mlp_t P, int64_t *count) {
  if (!P || !count) return IPM_ERR_BAD_ARG;
  int64_t c = 0;
  for (int l = 0; l < P->L; ++l) c += (int64_t)P->dims[l] * P->dims[l + 1] + P->dims[l + 1];
  *count = c;
  return IPM_OK;
}

// copies between a flat HOST array (per layer: W row-major, then b) and the device arrays
static int flat_copy(mlp_t P, const std::vector<float *> &W, const std::vector<float *> &b,
                     float *host, bool to_host) {
  size_t o = 0;
  for (int l = 0; l < P->L; ++l) {
    const size_t kn = (size_t)P->dims[l] * P->dims[l + 1], n = P->dims[l + 1];
    if (to_host) {
      CK(cudaMemcpy(host + o, W[l], sizeof(float) * kn, cudaMemcpyDeviceToHost));
      CK(cudaMemcpy(host + o + kn, b[l], sizeof(float) * n, cudaMemcpyDeviceToHost));
    } else {
      CK(cudaMemcpy(W[l], host + o, sizeof(float) * kn, cudaMemcpyHostToDevice));
      CK(cudaMemcpy(b[l], host + o + kn, sizeof(float) * n, cudaMemcpyHostToDevice));
    }
    o += kn + n;
  }
  return IPM_OK;
}

extern "C" int mlp_set_params(mlp_t P, const float *host) {
  if (!P || !host) return IPM_ERR_BAD_ARG;
  CKR(flat_copy(P, P->W, P->b, const_cast<float *>(host), false));
  for (int l = 0; l < P->L; ++l) {
    const int64_t kn = (int64_t)P->dims[l] * P->dims[l + 1];
    k_to_bf16<<<grid_elems(kn), 256>>>(kn, P->W[l], P->Wb[l]);
    CKL();
    CK(cudaMemset(P->mW[l], 0, sizeof(float) * kn));
    CK(cudaMemset(P->vW[l], 0, sizeof(float) * kn));
    CK(cudaMemset(P->mb[l], 0, sizeof(float) * P->dims[l + 1]));
    CK(cudaMemset(P->vb[l], 0, sizeof(float) * P->dims[l + 1]));
  }
  CK(cudaDeviceSynchronize());
  return IPM_OK;
}

extern "C" int mlp_get_params(mlp_t P, float *host) {
  if (!P || !host) return IPM_ERR_BAD_ARG;
  return flat_copy(P, P->W, P->b, host, true);
}

extern "C" int mlp_get_grads(mlp_t P, float *host) {
  if (!P || !host) return IPM_ERR_BAD_ARG;
  CK(cudaDeviceSynchronize());
  return flat_copy(P, P->gW, P->gb, host, true);
}

template <bool TA, bool TB>
static int gemm(int M, int N, int K, const bf16 *A, int lda, const bf16 *B, int ldb, float *C,
                int ldc, cudaStream_t s) {
  dim3 grid((N + GBN - 1) / GBN, (M + GBM - 1) / GBM);
  // too few output tiles for 152 SMs and a long K: split K over blocks (partial sums added)
  const int nk = (K + GBK - 1) / GBK, tiles = grid.x * grid.y;
  int split = 1;
  if (tiles < 2 * 152 && nk >= 8) split = std::min((2 * 152 + tiles - 1) / tiles, nk / 4);
  const int kchunk = (nk + split - 1) / split;
  grid.z = (nk + kchunk - 1) / kchunk;
  if (grid.z > 1) CK(cudaMemsetAsync(C, 0, sizeof(float) * ((size_t)(M - 1) * ldc + N), s));
  k_gemm_bf16<TA, TB><<<grid, 256, 0, s>>>(M, N, K, A, lda, B, ldb, C, ldc, kchunk);
  count_launches(1);
  CKL();
  return IPM_OK;
}

extern "C" int mlp_forward(mlp_t P, const float *X, int B, float *Y, cudaStream_t s) {
  if (!P || !X || B < 1 || B > P->max_batch) return IPM_ERR_BAD_ARG;
  const int64_t n0 = (int64_t)B * P->dims[0];
  k_to_bf16<<<grid_elems(n0), 256, 0, s>>>(n0, X, P->A[0]);
  count_launches(1);
  CKL();
  for (int l = 0; l < P->L; ++l) {
    const int k = P->dims[l], n = P->dims[l + 1];
    CKR((gemm<false, false>(B, n, k, P->A[l], k, P->Wb[l], n, P->Z[l], n, s)));
    const bool last = l == P->L - 1;
    k_bias_act<<<grid_elems((int64_t)B * n), 256, 0, s>>>(B, n, P->Z[l], P->b[l],
                                                          last ? nullptr : P->A[l + 1], !last,
                                                          last ? Y : nullptr);
    count_launches(1);
    CKL();
  }
  return IPM_OK;
}

extern "C" int mlp_loss_backward(mlp_t P, const float *T, int B, float *d_loss, cudaStream_t s) {
  if (!P || !T || !d_loss || B < 1 || B > P->max_batch) return IPM_ERR_BAD_ARG;
  const int L = P->L, nL = P->dims[L];
  const int64_t cnt = (int64_t)B * nL;
  CK(cudaMemsetAsync(d_loss, 0, sizeof(float), s));
  // the output of the last forward sits in Z[L-1]
  k_mse_grad<<<grid_elems(cnt), 256, 0, s>>>(cnt, P->Z[L - 1], T, 2.f / (float)cnt,
                                             1.f / (float)cnt, P->dZf[L - 1], P->dZb[L - 1],
                                             d_loss);
  count_launches(1);
  CKL();
  for (int l = L - 1; l >= 0; --l) {
    const int k = P->dims[l], n = P->dims[l + 1];
    // gW = A^T dZ, gb = column sums of dZ
    CKR((gemm<true, false>(k, n, B, P->A[l], k, P->dZb[l], n, P->gW[l], n, s)));
    k_col_sum<<<(n + 255) / 256, 256, 0, s>>>(B, n, P->dZf[l], P->gb[l]);
    count_launches(1);
    CKL();
    if (l > 0) {
      // dA = dZ W^T, dZ_{l-1} = dA gelu'(Z_{l-1})
      CKR((gemm<false, true>(B, k, n, P->dZb[l], n, P->Wb[l], n, P->dA, k, s)));
      k_gelu_back<<<grid_elems((int64_t)B * k), 256, 0, s>>>((int64_t)B * k, P->dA, P->Z[l - 1],
                                                             P->dZf[l - 1], P->dZb[l - 1]);
      count_launches(1);
      CKL();
    }
  }
  return IPM_OK;
}

extern "C" int mlp_adam_step(mlp_t P, float lr, float beta1, float beta2, float eps, int t,
                             cudaStream_t s) {
  if (!P || t < 1) return IPM_ERR_BAD_ARG;
  const float c1 = 1.f - powf(beta1, (float)t), c2 = 1.f - powf(beta2, (float)t);
  for (int l = 0; l < P->L; ++l) {
    const int64_t kn = (int64_t)P->dims[l] * P->dims[l + 1], n = P->dims[l + 1];
    k_adam<<<grid_elems(kn), 256, 0, s>>>(kn, P->W[l], P->gW[l], P->mW[l], P->vW[l], P->Wb[l], lr,
                                          beta1, beta2, eps, c1, c2);
    k_adam<<<grid_elems(n), 256, 0, s>>>(n, P->b[l], P->gb[l], P->mb[l], P->vb[l], nullptr, lr,
                                         beta1, beta2, eps, c1, c2);
    count_launches(2);
    CKL();
  }
  return IPM_OK;
}

// per-column mean and standard deviation (FP64 sums) of a rows x cols matrix; std floored at
// floor_std
__global__ void k_col_stats(int rows, int cols, const float *src, float *mean, float *stdv,
                            float floor_std) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= cols) return;
  double s = 0.0, q = 0.0;
  for (int i = 0; i < rows; ++i) {
    const double v = src[(size_t)i * cols + j];
    s += v;
    q += v * v;
  }
  const double m = rows ? s / rows : 0.0;
  const double var = rows ? fmax(q / rows - m * m, 0.0) : 0.0;
  mean[j] = (float)m;
  stdv[j] = fmaxf((float)sqrt(var), floor_std);
}

// out = (src - mean) / std, in place allowed
__global__ void k_normalize(int64_t n, int cols, const float *src, const float *mean,
                            const float *stdv, float *out) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const int j = (int)(i % cols);
    out[i] = (src[i] - mean[j]) / stdv[j];
  }
}

extern "C" int mlp_col_stats(int rows, int cols, const float *src, float *mean, float *stdv,
                             float floor_std, cudaStream_t s) {
  if (rows < 0 || cols < 1 || !src || !mean || !stdv) return IPM_ERR_BAD_ARG;
  k_col_stats<<<(cols + 255) / 256, 256, 0, s>>>(rows, cols, src, mean, stdv, floor_std);
  count_launches(1);
  CKL();
  return IPM_OK;
}

extern "C" int mlp_normalize(int rows, int cols, const float *src, const float *mean,
                             const float *stdv, float *out, cudaStream_t s) {
  if (rows < 0 || cols < 1 || !src || !mean || !stdv || !out) return IPM_ERR_BAD_ARG;
  const int64_t n = (int64_t)rows * cols;
  if (!n) return IPM_OK;
  k_normalize<<<grid_elems(n), 256, 0, s>>>(n, cols, src, mean, stdv, out);
  count_launches(1);
  CKL();
  return IPM_OK;
}

extern "C" int mlp_gather_rows(int rows, int cols, const int *idx, const float *src, float *out,
                               cudaStream_t s) {
  if (rows < 0 || cols < 0 || (rows && (!idx || !src || !out))) return IPM_ERR_BAD_ARG;
  if (!rows || !cols) return IPM_OK;
  dim3 grid(std::min((cols + 255) / 256, 64), rows);
  k_gather_rows<<<grid, 256, 0, s>>>(rows, cols, idx, src, out);
  count_launches(1);
  CKL();
  return IPM_OK;
}
