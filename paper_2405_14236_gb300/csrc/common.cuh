// Shared device utilities of libcondipm: error plumbing, device-wide scans, block sorts.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>
#include <stdio.h>

#include <string>
#include <type_traits>
#include <vector>

#include "../../include/condipm.h"
#include <nvtx3/nvToolsExt.h>

namespace cipm {

void set_error(const char *where, cudaError_t e);
// Counts kernel launches issued by the numeric entry points (reported by ipm_launch_count).
void count_launches(long long k);
// Set-up entry points (symbolic analysis, model and IPM-state creation) copy between host and
// device with the synchronous copy calls, which run on the legacy default stream, between their
// kernels.  They run all of their device work there: after the caller's stream's earlier work
// (their inputs may come from it), and complete on return.  Returns the stream to use.
inline cudaStream_t setup_stream(cudaStream_t caller) {
  cudaStreamSynchronize(caller);
  return cudaStreamLegacy;
}

// ipm_debug_poison_allocations: floating-point buffers start as NaN (bytes 0xFF) while set
bool poison_allocations();
template <typename T>
inline void poison_fresh(T *p, int64_t count) {
  if (std::is_floating_point<T>::value && poison_allocations()) {
    cudaMemset(p, 0xFF, sizeof(T) * (size_t)count);
    cudaDeviceSynchronize();  // before any stream's work on the buffer
  }
}
void set_error_msg(const std::string &msg);

#define CK(call)                              \
  do {                                        \
    cudaError_t e_ = (call);                  \
    if (e_ != cudaSuccess) {                  \
      ::cipm::set_error(#call, e_);           \
      return e_ == cudaErrorMemoryAllocation  \
                 ? IPM_ERR_OOM                \
                 : IPM_ERR_CUDA;              \
    }                                         \
  } while (0)

#define CKL() CK(cudaGetLastError())

#define CKR(expr)            \
  do {                       \
    int r_ = (expr);         \
    if (r_ != IPM_OK) return r_; \
  } while (0)

inline int grid_for(int64_t n, int block) {
  int64_t g = (n + block - 1) / block;
  if (g < 1) g = 1;
  if (g > (1 << 30)) g = (1 << 30);
  return (int)g;
}

// RAII list of temporary device allocations freed at scope exit.
struct DevTemp {
  std::vector<void *> ptrs;
  ~DevTemp() {
    for (void *p : ptrs) cudaFree(p);
  }
  template <typename T>
  int alloc(T **p, int64_t count) {
    *p = nullptr;
    if (count <= 0) count = 1;
    cudaError_t e = cudaMalloc((void **)p, sizeof(T) * (size_t)count);
    if (e != cudaSuccess) {
      set_error("cudaMalloc(temp)", e);
      return IPM_ERR_OOM;
    }
    poison_fresh(*p, count);
    ptrs.push_back(*p);
    return IPM_OK;
  }
};

template <typename T>
int dev_alloc(T **p, int64_t count) {
  *p = nullptr;
  if (count <= 0) count = 1;
  cudaError_t e = cudaMalloc((void **)p, sizeof(T) * (size_t)count);
  if (e != cudaSuccess) {
    set_error("cudaMalloc", e);
    return IPM_ERR_OOM;
  }
  poison_fresh(*p, count);
  return IPM_OK;
}

// Exclusive prefix sum out[i] = sum_{k<i} in[i]; out[n] = total.  `in` and `out` may alias.
// TIn/TOut: int or int64_t.  Uses a three-pass block scan; scratch allocated internally.
int exclusive_scan_i32_to_i64(const int *in, int64_t *out, int64_t n, cudaStream_t s);
int exclusive_scan_i32(const int *in, int *out, int64_t n, cudaStream_t s);
int exclusive_scan_i64(const int64_t *in, int64_t *out, int64_t n, cudaStream_t s);
// Inclusive running maximum of int values.
int inclusive_max_scan_i32(const int *in, int *out, int64_t n, cudaStream_t s);

// Sorting network with ascending comparators only (bitonic merge in its "flip then
// half-clean" form), so that a length that is not a power of two behaves as if padded
// with +infinity: a comparator whose upper element lies past the end does nothing.
template <typename T>
__device__ __forceinline__ void bitonic_asc(T *a, int len) {
  int p2 = 1;
  while (p2 < len) p2 <<= 1;
  for (int k = 2; k <= p2; k <<= 1) {
    for (int i = threadIdx.x; i < p2; i += blockDim.x) {
      int l = i ^ (k - 1);
      if (l > i && l < len) {
        T x = a[i], y = a[l];
        if (x > y) {
          a[i] = y;
          a[l] = x;
        }
      }
    }
    __syncthreads();
    for (int j = k >> 2; j > 0; j >>= 1) {
      for (int i = threadIdx.x; i < p2; i += blockDim.x) {
        int l = i ^ j;
        if (l > i && l < len) {
          T x = a[i], y = a[l];
          if (x > y) {
            a[i] = y;
            a[l] = x;
          }
        }
      }
      __syncthreads();
    }
  }
}

// Sorts a[0..len) (global memory) ascending, drops duplicates and the value `exclude`,
// and writes the result back to a[0..new_len).  Returns new_len in every thread.
// smem: `cap` ints of shared memory (+1 int at smem[cap] for the broadcast).  Segments
// longer than cap are sorted in place in global memory and compacted by one thread.
__device__ __forceinline__ int block_sort_unique(int *a, int len, int *smem, int cap,
                                                 int exclude) {
  __syncthreads();
  if (len <= cap) {
    for (int i = threadIdx.x; i < len; i += blockDim.x) smem[i] = a[i];
    __syncthreads();
    bitonic_asc(smem, len);
    // chunked compaction: each thread owns a contiguous chunk of the sorted array
    int nt = blockDim.x;
    int chunk = (len + nt - 1) / nt;
    int b = threadIdx.x * chunk, e = min(len, b + chunk);
    int kept = 0;
    for (int i = b; i < e; ++i)
      if (smem[i] != exclude && (i == 0 || smem[i] != smem[i - 1])) ++kept;
    // block exclusive scan of `kept` through shared memory after the data region
    __shared__ int s_cnt[1024];
    s_cnt[threadIdx.x] = kept;
    __syncthreads();
    if (threadIdx.x == 0) {
      int run = 0;
      for (int t = 0; t < nt; ++t) {
        int c = s_cnt[t];
        s_cnt[t] = run;
        run += c;
      }
      smem[cap] = run;
    }
    __syncthreads();
    int o = s_cnt[threadIdx.x];
    for (int i = b; i < e; ++i)
      if (smem[i] != exclude && (i == 0 || smem[i] != smem[i - 1])) a[o++] = smem[i];
    __syncthreads();
    int r = smem[cap];
    __syncthreads();
    return r;
  }
  bitonic_asc(a, len);
  if (threadIdx.x == 0) {
    int o = 0;
    for (int i = 0; i < len; ++i)
      if (a[i] != exclude && (i == 0 || a[i] != a[i - 1])) a[o++] = a[i];
    smem[cap] = o;
  }
  __syncthreads();
  int r = smem[cap];
  __syncthreads();
  return r;
}

__device__ __forceinline__ double warp_sum(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// NVTX range over a host-side phase of an entry point (the paper's phase timers: analysis,
// condensation, factorization, solves, CG, IPM iteration, batched sweep); a profiler shows them,
// and without one they cost a call into an empty injection point
struct NvtxRange {
  explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange &) = delete;
  NvtxRange &operator=(const NvtxRange &) = delete;
};

}  // namespace cipm
