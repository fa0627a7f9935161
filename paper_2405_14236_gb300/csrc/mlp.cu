// Multilayer perceptron for the learned warm start: BF16 weights and activations, FP32
// accumulation, GELU hidden layers, linear output, mean-squared-error loss, Adam.
//
// Layers l = 0 .. L-1 map width dims[l] to dims[l+1]: Z_l = A_l W_l + b_l with A_0 = bf16(X),
// A_{l+1} = bf16(gelu(Z_l)) for l < L-1 and Y = Z_{L-1}.  W_l is dims[l] x dims[l+1] row-major.
// The products run on the tensor cores (mma.sync m16n8k16, BF16 inputs, FP32 accumulators);
// FP32 master weights are updated by Adam and rounded to the BF16 copies the products read.
#include <cuda_bf16.h>

#include <cmath>
#include <vector>

#include "common.cuh"

namespace cipm {
namespace {

using bf16 = __nv_bfloat16;

// C[M x N] (FP32, row-major, ldc) = opA[M x K] opB[K x N] with BF16 operands.
// TA: A is stored K x M (row-major, lda), else M x K.  TB: B is stored N x K, else K x N.
template <bool TA, bool TB>
__global__ void __launch_bounds__(128) k_gemm_bf16(int M, int N, int K, const bf16 *A, int lda,
                                                   const bf16 *B, int ldb, float *C, int ldc) {
  constexpr int BM = 64, BN = 64, BK = 32, PAD = 8;
  __shared__ __align__(16) bf16 As[BM][BK + PAD];
  __shared__ __align__(16) bf16 Bs[BN][BK + PAD];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int wm = warp >> 1, wn = warp & 1;  // 2 x 2 warps, 32 x 32 each
  const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
  const int g = lane >> 2, t = lane & 3;
  float acc[2][4][4];
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j)
#pragma unroll
      for (int q = 0; q < 4; ++q) acc[i][j][q] = 0.f;
  const bf16 zero = __float2bfloat16(0.f);
  for (int k0 = 0; k0 < K; k0 += BK) {
    for (int e = tid; e < BM * BK; e += 128) {
      int m, k;
      if (TA) { m = e % BM; k = e / BM; } else { k = e % BK; m = e / BK; }
      const int gm = m0 + m, gk = k0 + k;
      bf16 v = zero;
      if (gm < M && gk < K) v = TA ? A[(size_t)gk * lda + gm] : A[(size_t)gm * lda + gk];
      As[m][k] = v;
    }
    for (int e = tid; e < BN * BK; e += 128) {
      int n, k;
      if (TB) { k = e % BK; n = e / BK; } else { n = e % BN; k = e / BN; }
      const int gn = n0 + n, gk = k0 + k;
      bf16 v = zero;
      if (gn < N && gk < K) v = TB ? B[(size_t)gn * ldb + gk] : B[(size_t)gk * ldb + gn];
      Bs[n][k] = v;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < BK; kk += 16) {
      uint32_t a[2][4], b[4][2];
#pragma unroll
      for (int i = 0; i < 2; ++i) {
        const int r = wm * 32 + i * 16 + g;
        a[i][0] = *reinterpret_cast<const uint32_t *>(&As[r][kk + t * 2]);
        a[i][1] = *reinterpret_cast<const uint32_t *>(&As[r + 8][kk + t * 2]);
        a[i][2] = *reinterpret_cast<const uint32_t *>(&As[r][kk + t * 2 + 8]);
        a[i][3] = *reinterpret_cast<const uint32_t *>(&As[r + 8][kk + t * 2 + 8]);
      }
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int c = wn * 32 + j * 8 + g;
        b[j][0] = *reinterpret_cast<const uint32_t *>(&Bs[c][kk + t * 2]);
        b[j][1] = *reinterpret_cast<const uint32_t *>(&Bs[c][kk + t * 2 + 8]);
      }
#pragma unroll
      for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j)
          asm volatile(
              "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, "
              "{%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};\n"
              : "+f"(acc[i][j][0]), "+f"(acc[i][j][1]), "+f"(acc[i][j][2]), "+f"(acc[i][j][3])
              : "r"(a[i][0]), "r"(a[i][1]), "r"(a[i][2]), "r"(a[i][3]), "r"(b[j][0]),
                "r"(b[j][1]));
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int r = m0 + wm * 32 + i * 16 + g, c = n0 + wn * 32 + j * 8 + t * 2;
      if (r < M) {
        if (c < N) C[(size_t)r * ldc + c] = acc[i][j][0];
        if (c + 1 < N) C[(size_t)r * ldc + c + 1] = acc[i][j][1];
      }
      if (r + 8 < M) {
        if (c < N) C[(size_t)(r + 8) * ldc + c] = acc[i][j][2];
        if (c + 1 < N) C[(size_t)(r + 8) * ldc + c + 1] = acc[i][j][3];
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
  dim3 grid((N + 63) / 64, (M + 63) / 64);
  k_gemm_bf16<TA, TB><<<grid, 128, 0, s>>>(M, N, K, A, lda, B, ldb, C, ldc);
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
