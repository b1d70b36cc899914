// Allocation-free variant of the leaf batch (perm_leaf_batch_noalloc).
//
// For callers that must not allocate device memory while they run -- a host
// framework whose allocator must own every allocation, a latency-bound loop
// that forbids allocation after start-up (cudaMalloc and cudaFree can
// synchronise the device), or a process held to a fixed memory budget.
// The caller passes device inputs and outputs; the only other device memory
// the call touches is the file-scope array below, which every GPU that
// loads the library holds until the process exits.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <mutex>

#include "internal.h"
#include "ryser.cuh"

namespace {

constexpr int NA_WARPS = 8;
constexpr int NA_CHUNK_LOG2 = 10;

// Scratch: a task counter, then four accumulator words per matrix.
struct NoAllocScratch {
  unsigned long long counter;
  unsigned long long pad[31];
  unsigned long long acc[4 * PERM_NOALLOC_MAX_COUNT];
};
static_assert(sizeof(NoAllocScratch) == PERM_NOALLOC_SCRATCH_BYTES, "scratch size stated in perm.h");

static __device__ __align__(256) NoAllocScratch g_noalloc_scratch;

// m >= 2 codes split: lanes walk aligned blocks of 2^clog codes (as leaf.cu).
__host__ __device__ __forceinline__ void na_split(int m, int& lanes, int& clog, uint64_t& tasks) {
  const int e = m - 1;
  if (e <= 5) {
    clog = 1;
    lanes = 1 << (e - 1);
    tasks = 1;
    return;
  }
  lanes = 32;
  clog = e - 5 < NA_CHUNK_LOG2 ? e - 5 : NA_CHUNK_LOG2;
  tasks = 1ull << (e - 5 - clog);
}

__global__ void k_na_clear(NoAllocScratch* sc, int count) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k == 0) sc->counter = 0;
  if (k < 4 * count) sc->acc[k] = 0;
}

// Row sums must fit int32 and entries 2^30 (the leaf kernel's ranges).
__device__ __forceinline__ bool na_in_range(const int64_t* a, int n) {
  for (int i = 0; i < n; ++i) {
    int64_t ra = 0;
    for (int j = 0; j < n; ++j) {
      const int64_t v = a[(int64_t)i * n + j];
      if (v >= (1ll << 30) || v <= -(1ll << 30)) return false;
      ra += v < 0 ? -v : v;
    }
    if (ra >= (1ll << 31)) return false;
  }
  return true;
}

template <int NMAX>
__global__ void __launch_bounds__(NA_WARPS * 32)
    k_na_batch(const int64_t* __restrict__ a, int n, int count, NoAllocScratch* sc) {
  __shared__ __align__(16) int32_t delta_s[NA_WARPS][(PERM_MAX_LEAF - 1) * 32];
  __shared__ __align__(16) int32_t rho0_s[NA_WARPS][32];
  const int lane = threadIdx.x & 31;
  const int wib = threadIdx.x >> 5;
  int32_t* delta = delta_s[wib];
  int32_t* rho0 = rho0_s[wib];
  int lanes, clog;
  uint64_t tasks;
  na_split(n, lanes, clog, tasks);
  const uint64_t total = tasks * (uint64_t)count;
  int cur = -1;
  bool ok = false;
  for (;;) {
    unsigned long long t = 0;
    if (lane == 0) t = atomicAdd(&sc->counter, 1ull);
    t = __shfl_sync(0xffffffffu, t, 0);
    if (t >= total) break;
    const int k = (int)(t / tasks);
    const uint64_t lt = t % tasks;
    const int64_t* A = a + (int64_t)k * n * n;
    if (k != cur) {
      cur = k;
      ok = na_in_range(A, n);
      if (ok) {
        for (int q = lane; q < (n - 1) * NMAX; q += 32) delta[q] = 0;
        __syncwarp();
        for (int i = lane; i < NMAX; i += 32) {
          if (i >= n) {
            rho0[i] = 1;
            continue;
          }
          int64_t rs = 0;
          for (int j = 0; j < n; ++j) {
            const int64_t v = A[(int64_t)i * n + j];
            rs += v;
            if (j < n - 1) delta[j * NMAX + i] = (int32_t)(2 * v);
          }
          rho0[i] = (int32_t)(2 * A[(int64_t)i * n + n - 1] - rs);
        }
        __syncwarp();
      }
    }
    if (!ok) continue;
    const uint64_t cnt = 1ull << clog;
    const uint64_t gb = (lt * 32 + lane) * cnt;
    u256 s = ryser_lane<NMAX, 4, 31>(delta, rho0, n, gb, lane < lanes ? cnt : 0);
    s = warp_sum(s);
    if (lane == 0) atomic_add_words(sc->acc + 4ll * k, s.w, 4);
  }
}

// Sigma -> per = (-1)^(n-1) Sigma / 2^(n-1), exact in its low 257 - n bits;
// sign-extended from there.  The bound min(prod_i sum_j |a_ij|,
// prod_j sum_i |a_ij|) must not exceed 2^(254 - n) (checked in fp64 with one
// bit of margin: log2 bound + 1 > 255 - n fails), else the status is
// PERM_EOVERFLOW.
__global__ void k_na_finalize(const int64_t* __restrict__ a, int n, int count, const NoAllocScratch* sc,
                              uint64_t* __restrict__ out, int32_t* __restrict__ status) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= count) return;
  const int64_t* A = a + (int64_t)k * n * n;
  int st = 0;
  u256 v = u256_zero();
  if (!na_in_range(A, n)) {
    st = PERM_EOVERFLOW;
  } else if (n == 1) {
    v = u256_from_s64(A[0]);
  } else {
    double lr = 0.0, lc = 0.0;
    for (int i = 0; i < n; ++i) {
      double rs = 0.0, cs = 0.0;
      for (int j = 0; j < n; ++j) {
        rs += fabs((double)A[(int64_t)i * n + j]);
        cs += fabs((double)A[(int64_t)j * n + i]);
      }
      lr += rs > 0.0 ? log2(rs) : -1e30;
      lc += cs > 0.0 ? log2(cs) : -1e30;
    }
    const double lb = lr < lc ? lr : lc;
    if (lb + 1.0 > (double)(255 - n)) st = PERM_EOVERFLOW;
    for (int w = 0; w < 4; ++w) v.w[w] = sc->acc[4ll * k + w];
    v = u256_shr(v, n - 1);
    if ((n - 1) & 1) v = u256_neg(v);
    // sign-extend from bit 256 - n (exact bits: 257 - n)
    const int top = 256 - n;
    const int word = top / 64, bit = top % 64;
    const bool neg = (v.w[word] >> bit) & 1;
    const uint64_t keep = bit == 63 ? ~0ull : ((1ull << (bit + 1)) - 1);
    v.w[word] = neg ? (v.w[word] | ~keep) : (v.w[word] & keep);
    for (int w = word + 1; w < 4; ++w) v.w[w] = neg ? ~0ull : 0ull;
  }
  if (st != 0) v = u256_zero();
  for (int w = 0; w < 4; ++w) out[4ll * k + w] = v.w[w];
  status[k] = st;
}

// Device address of the scratch array, looked up once per device.
std::mutex g_na_mu;
NoAllocScratch* g_na_addr[64] = {nullptr};

cudaError_t na_scratch(int dev, NoAllocScratch** out) {
  std::lock_guard<std::mutex> lk(g_na_mu);
  if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  if (!g_na_addr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_na_addr[dev] = reinterpret_cast<NoAllocScratch*>(p);
  }
  *out = g_na_addr[dev];
  return cudaSuccess;
}

}  // namespace

static perm_status perm_leaf_batch_noalloc_impl(const int64_t* a, int32_t n, int32_t count, uint64_t* out,
                                                int32_t* status, void* stream) {
  if (!a || !out || !status) return PERM_EINVAL;
  if (n < 1 || n > PERM_MAX_LEAF) return PERM_EINVAL;
  if (count < 1 || count > PERM_NOALLOC_MAX_COUNT) return PERM_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  NoAllocScratch* sc = nullptr;
  if (e == cudaSuccess) e = na_scratch(dev, &sc);
  if (e != cudaSuccess) {
    set_last_error("perm_leaf_batch_noalloc setup", e);
    return PERM_ECUDA;
  }
  const int nacc = 4 * count;
  k_na_clear<<<(nacc + 255) / 256, 256, 0, s>>>(sc, count);
  if (n >= 2) {
    const int nmax = nmax_for(n);
    const unsigned grid = (unsigned)sms * 2u;
    switch (nmax) {
      case 8: k_na_batch<8><<<grid, NA_WARPS * 32, 0, s>>>(a, n, count, sc); break;
      case 16: k_na_batch<16><<<grid, NA_WARPS * 32, 0, s>>>(a, n, count, sc); break;
      case 24: k_na_batch<24><<<grid, NA_WARPS * 32, 0, s>>>(a, n, count, sc); break;
      default: k_na_batch<32><<<grid, NA_WARPS * 32, 0, s>>>(a, n, count, sc); break;
    }
  }
  k_na_finalize<<<(count + 127) / 128, 128, 0, s>>>(a, n, count, sc, out, status);
  e = cudaGetLastError();
  if (e != cudaSuccess) {
    set_last_error("perm_leaf_batch_noalloc launch", e);
    return PERM_ECUDA;
  }
  return PERM_OK;
}
extern "C" perm_status perm_leaf_batch_noalloc(const int64_t* a, int32_t n, int32_t count, uint64_t* out,
                                               int32_t* status, void* stream) {
  return guarded([&] { return perm_leaf_batch_noalloc_impl(a, n, count, out, status, stream); });
}
