// K4: Algorithm KKLLL (Section 2.3) on the 0/1 pattern of each job
// (Section 3's B).  Each nonzero becomes a cube root of unity drawn from a
// counter-based SplitMix64 stream; |det W|^2 is an unbiased estimate of
// per(B) (the paper's Theorem), and the job's approximate permanent is the
// mean over T trials.  One warp per job; the trial matrix sits in shared
// memory as complex FP32 and is reduced by Gaussian elimination with partial
// pivoting on |z| (lowest row on ties).  |det|^2 is the product of the
// pivots' squared moduli, kept as an FP32 mantissa with an integer exponent;
// the mean over trials is accumulated in FP64 as a log-sum-exp.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>

#include "internal.h"

namespace {

constexpr uint64_t K_JOB = 0xD1B54A32D192ED03ull;
constexpr uint64_t K_TRIAL = 0xABC98388FB8FAC03ull;
constexpr uint64_t K_ENTRY = 0x8CB92BA72F3D8DD7ull;

// SplitMix64's output function (Steele, Lea, Flood, OOPSLA 2014).
__device__ __forceinline__ uint64_t splitmix64_mix(uint64_t z) {
  z += 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

template <int TILE>
struct KCfg {
  static constexpr int STRIDE = TILE + 1;
  static constexpr int WARPS = TILE <= 32 ? 8 : 4;
  static constexpr size_t WARP_BYTES = sizeof(float2) * TILE * STRIDE + sizeof(uint64_t) * TILE;
  static constexpr size_t SMEM = WARPS * WARP_BYTES;
};

template <int TILE>
__global__ void __launch_bounds__(KCfg<TILE>::WARPS * 32)
    k_kklll(JobArrays jobs, int64_t njobs, const uint64_t* __restrict__ arena, int trials, uint64_t seed,
            float* __restrict__ log_ap) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  constexpr int S = KCfg<TILE>::STRIDE;
  constexpr int RPL = TILE / 32;
  const int lane = threadIdx.x & 31;
  const int wib = threadIdx.x >> 5;
  unsigned char* base = smem_raw + (size_t)wib * KCfg<TILE>::WARP_BYTES;
  float2* Wm = reinterpret_cast<float2*>(base);
  uint64_t* pat = reinterpret_cast<uint64_t*>(base + sizeof(float2) * TILE * S);
  const float RE[3] = {1.0f, -0.5f, -0.5f};
  const float IM[3] = {0.0f, 0.86602540378443864676f, -0.86602540378443864676f};
  const int64_t nwarps = (int64_t)gridDim.x * KCfg<TILE>::WARPS;
  for (int64_t job = (int64_t)blockIdx.x * KCfg<TILE>::WARPS + wib; job < njobs; job += nwarps) {
    __syncwarp();
    const int m = jobs.m[job];
    if (m > TILE || m <= 0) {
      if (lane == 0) log_ap[job] = m == 0 ? 0.0f : nanf("");
      continue;
    }
    CsrView v = csr_view(arena, jobs.off[job], m, jobs.nnz[job]);
    for (int r = lane; r < m; r += 32) {
      uint64_t b = 0;
      for (int q = v.rowptr[r]; q < v.rowptr[r + 1]; ++q) b |= 1ull << v.col[q];
      pat[r] = b;
    }
    __syncwarp();
    const int T = trials > 0 ? trials : m * m;
    const uint64_t jkey = seed ^ ((uint64_t)job * K_JOB);
    double lmax = -INFINITY, lsum = 0.0;  // running log-sum-exp (lane 0)
    for (int t = 0; t < T; ++t) {
      const uint64_t tkey = jkey ^ ((uint64_t)t * K_TRIAL);
      // trial matrix
      for (int r = 0; r < m; ++r) {
        const uint64_t b = pat[r];
#pragma unroll
        for (int u = 0; u < RPL; ++u) {
          const int c = lane + 32 * u;
          float2 z = make_float2(0.f, 0.f);
          if (c < m && ((b >> c) & 1)) {
            const uint64_t h = splitmix64_mix(tkey ^ ((uint64_t)(r * m + c) * K_ENTRY));
            const int w = (int)(((h >> 32) * 3ull) >> 32);
            z = make_float2(RE[w], IM[w]);
          }
          if (c < m) Wm[r * S + c] = z;
        }
      }
      __syncwarp();
      float pm = 1.0f;  // |det|^2 = pm * 2^pe
      int pe = 0;
      bool singular = false;
      for (int k = 0; k < m; ++k) {
        // pivot: largest |z|^2 in column k among rows >= k, lowest row on ties
        unsigned long long key = 0;
#pragma unroll
        for (int u = 0; u < RPL; ++u) {
          const int r = lane + 32 * u;
          if (r >= k && r < m) {
            const float2 z = Wm[r * S + k];
            const float mag = z.x * z.x + z.y * z.y;
            const unsigned long long kk =
                ((unsigned long long)__float_as_uint(mag) << 32) | (unsigned long long)(0xffffffffu - (uint32_t)r);
            key = kk > key ? kk : key;
          }
        }
#pragma unroll
        for (int d = 16; d > 0; d >>= 1) {
          unsigned long long o = __shfl_xor_sync(0xffffffffu, key, d);
          key = o > key ? o : key;
        }
        const float mag = __uint_as_float((uint32_t)(key >> 32));
        const int p = (int)(0xffffffffu - (uint32_t)(key & 0xffffffffu));
        if (!(mag > 0.0f)) {
          singular = true;
          break;
        }
        if (p != k) {
#pragma unroll
          for (int u = 0; u < RPL; ++u) {
            const int c = lane + 32 * u;
            if (c >= k && c < m) {
              const float2 a = Wm[k * S + c];
              Wm[k * S + c] = Wm[p * S + c];
              Wm[p * S + c] = a;
            }
          }
        }
        __syncwarp();
        int ex;
        pm = frexpf(pm * mag, &ex);
        pe += ex;
        const float2 piv = Wm[k * S + k];
        const float inv = 1.0f / mag;
        const float2 ipiv = make_float2(piv.x * inv, -piv.y * inv);  // 1 / piv
        float2 rowk[RPL];
#pragma unroll
        for (int u = 0; u < RPL; ++u) {
          const int c = lane + 32 * u;
          rowk[u] = (c > k && c < m) ? Wm[k * S + c] : make_float2(0.f, 0.f);
        }
        for (int r = k + 1; r < m; ++r) {
          const float2 a = Wm[r * S + k];
          const float2 f = make_float2(a.x * ipiv.x - a.y * ipiv.y, a.x * ipiv.y + a.y * ipiv.x);
#pragma unroll
          for (int u = 0; u < RPL; ++u) {
            const int c = lane + 32 * u;
            if (c > k && c < m) {
              float2 z = Wm[r * S + c];
              z.x -= f.x * rowk[u].x - f.y * rowk[u].y;
              z.y -= f.x * rowk[u].y + f.y * rowk[u].x;
              Wm[r * S + c] = z;
            }
          }
        }
        __syncwarp();
      }
      if (lane == 0 && !singular) {
        const double l = log((double)pm) + (double)pe * 0.69314718055994530942;
        if (l > lmax) {
          lsum = lsum * exp(lmax - l) + 1.0;
          lmax = l;
        } else {
          lsum += exp(l - lmax);
        }
      }
      __syncwarp();
    }
    if (lane == 0) {
      log_ap[job] = lmax == -INFINITY ? -INFINITY : (float)(lmax + log(lsum / (double)T));
    }
  }
}

template <int TILE>
cudaError_t launch_k(const JobArrays& jobs, int64_t njobs, const uint64_t* arena, int trials, uint64_t seed,
                     float* log_ap, cudaStream_t s) {
  typedef KCfg<TILE> C;
  static bool attr_set = false;
  if (!attr_set) {
    cudaError_t e = cudaFuncSetAttribute(k_kklll<TILE>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::SMEM);
    if (e != cudaSuccess) return e;
    attr_set = true;
  }
  int64_t blocks = (njobs + C::WARPS - 1) / C::WARPS;
  if (blocks > 152 * 32) blocks = 152 * 32;
  k_kklll<TILE><<<(unsigned)blocks, C::WARPS * 32, C::SMEM, s>>>(jobs, njobs, arena, trials, seed, log_ap);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_kklll(const JobArrays& jobs, int64_t njobs, const uint64_t* arena, int trials, uint64_t seed,
                         float* log_ap, int max_order, cudaStream_t s) {
  if (njobs <= 0) return cudaSuccess;
  if (max_order <= 32) return launch_k<32>(jobs, njobs, arena, trials, seed, log_ap, s);
  return launch_k<64>(jobs, njobs, arena, trials, seed, log_ap, s);
}
