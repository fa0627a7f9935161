// Error plumbing and device-wide prefix scans for libcondipm.
#include <atomic>
#include <mutex>

#include "common.cuh"

namespace cipm {

static std::atomic<long long> g_launches{0};
void count_launches(long long k) { g_launches.fetch_add(k, std::memory_order_relaxed); }

static std::atomic<int> g_poison{0};
bool poison_allocations() { return g_poison.load(std::memory_order_relaxed) != 0; }

static std::mutex g_err_mu;
static std::string g_err;

void set_error(const char *where, cudaError_t e) {
  std::lock_guard<std::mutex> lk(g_err_mu);
  g_err = std::string(where) + ": " + cudaGetErrorString(e);
}

void set_error_msg(const std::string &msg) {
  std::lock_guard<std::mutex> lk(g_err_mu);
  g_err = msg;
}

static constexpr int SCAN_BLOCK = 512;
static constexpr int SCAN_ITEMS = 4;  // per thread
static constexpr int SCAN_TILE = SCAN_BLOCK * SCAN_ITEMS;

struct OpAdd {
  template <typename T>
  __device__ static T apply(T a, T b) { return a + b; }
  template <typename T>
  __device__ static T identity() { return T(0); }
};
struct OpMax {
  template <typename T>
  __device__ static T apply(T a, T b) { return a > b ? a : b; }
  template <typename T>
  __device__ static T identity() { return T(-2147483647 - 1); }
};

// Tile scan: each block scans SCAN_TILE items; writes exclusive (or inclusive) results and
// the tile total.
template <typename TI, typename TO, typename Op, bool Inclusive>
__global__ void k_tile_scan(const TI *in, TO *out, TO *tile_tot, int64_t n) {
  __shared__ TO s_thr[SCAN_BLOCK];
  int64_t base = (int64_t)blockIdx.x * SCAN_TILE + (int64_t)threadIdx.x * SCAN_ITEMS;
  TO v[SCAN_ITEMS];
  TO acc = Op::template identity<TO>();
#pragma unroll
  for (int k = 0; k < SCAN_ITEMS; ++k) {
    int64_t i = base + k;
    TO x = i < n ? (TO)in[i] : Op::template identity<TO>();
    if (Inclusive) {
      acc = Op::apply(acc, x);
      v[k] = acc;
    } else {
      v[k] = acc;
      acc = Op::apply(acc, x);
    }
  }
  s_thr[threadIdx.x] = acc;
  __syncthreads();
  // Hillis-Steele inclusive scan of the per-thread totals
  for (int off = 1; off < SCAN_BLOCK; off <<= 1) {
    TO t = threadIdx.x >= off ? s_thr[threadIdx.x - off] : Op::template identity<TO>();
    __syncthreads();
    s_thr[threadIdx.x] = Op::apply(s_thr[threadIdx.x], t);
    __syncthreads();
  }
  TO prefix = threadIdx.x > 0 ? s_thr[threadIdx.x - 1] : Op::template identity<TO>();
#pragma unroll
  for (int k = 0; k < SCAN_ITEMS; ++k) {
    int64_t i = base + k;
    if (i < n) out[i] = Op::apply(prefix, v[k]);
  }
  if (threadIdx.x == SCAN_BLOCK - 1) tile_tot[blockIdx.x] = s_thr[SCAN_BLOCK - 1];
}

template <typename TO, typename Op>
__global__ void k_tile_add(TO *out, const TO *tile_prefix, int64_t n) {
  int64_t base = (int64_t)blockIdx.x * SCAN_TILE;
  TO p = tile_prefix[blockIdx.x];
  for (int k = threadIdx.x; k < SCAN_TILE; k += blockDim.x) {
    int64_t i = base + k;
    if (i < n) out[i] = Op::apply(p, out[i]);
  }
}

template <typename TO>
__global__ void k_set_total(TO *out, int64_t n, const TO *tot) {
  out[n] = *tot;
}

// Generic scan driver.  For exclusive scans out has n+1 entries and out[n] = total.
template <typename TI, typename TO, typename Op, bool Inclusive>
static int scan_impl(const TI *in, TO *out, int64_t n, cudaStream_t s) {
  if (n <= 0) {
    if (!Inclusive) {
      TO z = 0;
      CK(cudaMemcpyAsync(out, &z, sizeof(TO), cudaMemcpyHostToDevice, s));
      CK(cudaStreamSynchronize(s));
    }
    return IPM_OK;
  }
  int64_t tiles = (n + SCAN_TILE - 1) / SCAN_TILE;
  DevTemp tmp;
  TO *tot = nullptr, *totscan = nullptr;
  CKR(tmp.alloc(&tot, tiles + 1));
  CKR(tmp.alloc(&totscan, tiles + 1));
  k_tile_scan<TI, TO, Op, Inclusive><<<(int)tiles, SCAN_BLOCK, 0, s>>>(in, out, tot, n);
  CKL();
  if (tiles > 1) {
    // exclusive scan of tile totals (recursive), then add
    CKR((scan_impl<TO, TO, Op, false>(tot, totscan, tiles, s)));
    k_tile_add<TO, Op><<<(int)tiles, SCAN_BLOCK, 0, s>>>(out, totscan, n);
    CKL();
    if (!Inclusive) {
      // total = exclusive prefix of last tile + last tile total
      k_set_total<TO><<<1, 1, 0, s>>>(out, n, totscan + tiles);
      CKL();
    }
  } else if (!Inclusive) {
    k_set_total<TO><<<1, 1, 0, s>>>(out, n, tot);
    CKL();
  }
  CK(cudaStreamSynchronize(s));  // temporaries are freed on return
  return IPM_OK;
}

int exclusive_scan_i32_to_i64(const int *in, int64_t *out, int64_t n, cudaStream_t s) {
  return scan_impl<int, int64_t, OpAdd, false>(in, out, n, s);
}
int exclusive_scan_i32(const int *in, int *out, int64_t n, cudaStream_t s) {
  return scan_impl<int, int, OpAdd, false>(in, out, n, s);
}
int exclusive_scan_i64(const int64_t *in, int64_t *out, int64_t n, cudaStream_t s) {
  return scan_impl<int64_t, int64_t, OpAdd, false>(in, out, n, s);
}
int inclusive_max_scan_i32(const int *in, int *out, int64_t n, cudaStream_t s) {
  return scan_impl<int, int, OpMax, true>(in, out, n, s);
}

}  // namespace cipm

extern "C" long long ipm_launch_count(void) { return cipm::g_launches.load(); }

extern "C" int ipm_debug_poison_allocations(int on) {
  cipm::g_poison.store(on ? 1 : 0);
  return IPM_OK;
}

extern "C" const char *ipm_last_error_message(void) {
  std::lock_guard<std::mutex> lk(cipm::g_err_mu);
  return cipm::g_err.c_str();
}
