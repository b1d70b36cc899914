// K4: Algorithm KKLLL (Section 2.3) on the 0/1 pattern of each job
// (Section 3's B).  Each nonzero becomes a cube root of unity drawn from a
// counter-based SplitMix64 stream; |det W|^2 is an unbiased estimate of
// per(B) (the paper's Theorem), and the job's approximate permanent is the
// mean over T trials.  Each trial matrix is complex FP32, reduced by
// Gaussian elimination with partial pivoting on |z| (lowest row on ties);
// |det|^2 is the product of the pivots' squared moduli, kept as an FP32
// mantissa with an integer exponent, and trials are summed in FP64 scaled
// by powers of two.  The form follows the launch's largest job order:
// one trial per thread in shared memory (<= 12), per group of lanes in
// registers (<= 16), per warp in shared memory (<= 64, the trials of a job
// split into parts merged by k_kklll_combine), one job per warp above 64.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>

#include "internal.h"

namespace {

constexpr uint64_t K_JOB = 0xD1B54A32D192ED03ull;
constexpr uint64_t K_TRIAL = 0xABC98388FB8FAC03ull;
constexpr uint64_t K_ENTRY = 0x8CB92BA72F3D8DD7ull;

constexpr double LN2 = 0.69314718055994530942;

// Running sum of the trials' |det W|^2 = pm * 2^pe (pm in [1/2, 1)), held as
// S * 2^E with S a double: adding a trial scales by a power of two and takes
// no logarithm or exponential.
struct Pow2Sum {
  double S = 0.0;
  int E = -(1 << 30);
  // 2^e for e <= 0; 0 below the normal range (such a term is below 2^-1022
  // of the running sum)
  __device__ __forceinline__ static double pow2(int e) {
    return e < -1022 ? 0.0 : __hiloint2double((e + 1023) << 20, 0);
  }
  __device__ __forceinline__ void add(float pm, int pe) {
    if (pe > E) {
      S = S * pow2(E - pe) + (double)pm;
      E = pe;
    } else {
      S += (double)pm * pow2(pe - E);
    }
  }
  __device__ __forceinline__ void merge(double oS, int oE) {
    const int e = oE > E ? oE : E;
    S = S * pow2(E - e) + oS * pow2(oE - e);
    E = e;
  }
  // butterfly merge with the lanes at xor distances d0, 2 d0, ..., 16
  __device__ __forceinline__ void warp_merge(int d0) {
    for (int d = d0; d < 32; d <<= 1) merge(__shfl_xor_sync(0xffffffffu, S, d), __shfl_xor_sync(0xffffffffu, E, d));
  }
  // as a log-sum-exp pair: the sum is lsum * e^lmax
  __device__ __forceinline__ void lse(double& lmax, double& lsum) const {
    if (S > 0.0) {
      lmax = (double)E * LN2;
      lsum = S;
    } else {
      lmax = -INFINITY;
      lsum = 0.0;
    }
  }
};

// z -= f * p in complex arithmetic, as four fused multiply-adds
__device__ __forceinline__ void cfms(float2& z, float2 f, float2 p) {
  z.x = fmaf(-f.x, p.x, z.x);
  z.x = fmaf(f.y, p.y, z.x);
  z.y = fmaf(-f.x, p.y, z.y);
  z.y = fmaf(-f.y, p.x, z.y);
}

// e^(2 pi i w / 3), w in {0, 1, 2}
__device__ __forceinline__ float2 cube_root(uint32_t w) {
  const float h = 0.86602540378443864676f;  // sqrt(3) / 2
  return make_float2(w == 0 ? 1.0f : -0.5f, w == 0 ? 0.0f : (w == 1 ? h : -h));
}

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
  static constexpr int MW = (TILE + 63) / 64;  // pattern words per row
  static constexpr int WARPS = TILE <= 32 ? 8 : (TILE <= 64 ? 4 : 1);
  static constexpr size_t WARP_BYTES = sizeof(float2) * TILE * STRIDE + sizeof(uint64_t) * TILE * MW;
  static constexpr size_t SMEM = WARPS * WARP_BYTES;
};

template <int TILE>
__global__ void __launch_bounds__(KCfg<TILE>::WARPS * 32)
    k_kklll(JobArrays jobs, int64_t njobs, const uint64_t* __restrict__ arena, int trials, uint64_t seed,
            float* __restrict__ log_ap) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  constexpr int S = KCfg<TILE>::STRIDE;
  constexpr int MW = KCfg<TILE>::MW;
  constexpr int RPL = TILE / 32;
  const int lane = threadIdx.x & 31;
  const int wib = threadIdx.x >> 5;
  unsigned char* base = smem_raw + (size_t)wib * KCfg<TILE>::WARP_BYTES;
  float2* Wm = reinterpret_cast<float2*>(base);
  uint64_t* pat = reinterpret_cast<uint64_t*>(base + sizeof(float2) * TILE * S);
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
      uint64_t b[MW];
#pragma unroll
      for (int w = 0; w < MW; ++w) b[w] = 0;
      for (int q = v.rowptr[r]; q < v.rowptr[r + 1]; ++q) {
        const int c = v.col[q];
#pragma unroll
        for (int w = 0; w < MW; ++w)
          if ((c >> 6) == w) b[w] |= 1ull << (c & 63);
      }
#pragma unroll
      for (int w = 0; w < MW; ++w) pat[r * MW + w] = b[w];
    }
    __syncwarp();
    const int T = trials > 0 ? trials : m * m;
    const uint64_t jkey = seed ^ ((uint64_t)job * K_JOB);
    Pow2Sum acc;  // lane 0
    for (int t = 0; t < T; ++t) {
      const uint64_t tkey = jkey ^ ((uint64_t)t * K_TRIAL);
      // trial matrix
      for (int r = 0; r < m; ++r) {
#pragma unroll
        for (int u = 0; u < RPL; ++u) {
          const int c = lane + 32 * u;
          const uint64_t b = pat[r * MW + (u >> 1)];  // column c lies in word c / 64 = u / 2
          float2 z = make_float2(0.f, 0.f);
          if (c < m && ((b >> (c & 63)) & 1)) {
            const uint64_t h = splitmix64_mix(tkey ^ ((uint64_t)(r * m + c) * K_ENTRY));
            const int w = (int)(((h >> 32) * 3ull) >> 32);
            z = cube_root((uint32_t)w);
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
              cfms(z, f, rowk[u]);
              Wm[r * S + c] = z;
            }
          }
        }
        __syncwarp();
      }
      if (lane == 0 && !singular) acc.add(pm, pe);
      __syncwarp();
    }
    if (lane == 0) {
      double lmax, lsum;
      acc.lse(lmax, lsum);
      log_ap[job] = lmax == -INFINITY ? -INFINITY : (float)(lmax + log(lsum / (double)T));
    }
  }
}

// Tile form for jobs of order 17 <= m <= MT (MT <= 64): a warp runs one
// trial at a time, the m x m trial matrix in shared memory with row stride
// S (S = 8 mod 16, so four consecutive rows by eight consecutive columns hit
// 32 distinct bank pairs).  Step k swaps the pivot row into row k (partial
// pivoting: largest |z|^2 in column k among rows >= k, the lowest row on
// ties, ties meaning within 2^-17 relative since the key keeps 63 - row in
// the magnitude's low 6 bits) and updates the trailing block, spread over
// the lanes as a 4 x 8 grid: lane (ly, lx) takes the rows r = ly (mod 4)
// and columns c = lx (mod 8) above k.  The lanes whose first column is k+1
// form the next step's pivot keys while they update it, so a step needs
// one warp reduction.  A warp takes chunk_trials trials of one job and
// writes their sum to part[]; k_kklll_combine merges a job's parts.
template <int MT>
struct TileCfg {
  static constexpr int JMAX = MT / 8;  // columns of a row per lane
  static constexpr int LIST = 512;     // nonzeros held as (row, column) pairs
  // one warp per block: the blocks per SM follow the launch's shared memory
  static constexpr int WARPS = 1;
};

__host__ __device__ __forceinline__ int tile_stride(int mmax) { return (mmax - 8 + 15) / 16 * 16 + 8; }

__device__ __forceinline__ uint32_t tile_key(float2 z, int r) {
  return (__float_as_uint(z.x * z.x + z.y * z.y) & ~63u) | (uint32_t)(63 - r);
}

template <int MT>
__global__ void __launch_bounds__(TileCfg<MT>::WARPS * 32, 16)
    k_kklll_tile(JobArrays jobs, int64_t njobs, const uint64_t* __restrict__ arena, int trials, uint64_t seed,
                 int chunks_per_job, int chunk_trials, int S, int wrows, int warp_bytes, double2* __restrict__ part) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  constexpr int JMAX = TileCfg<MT>::JMAX;
  constexpr int LIST = TileCfg<MT>::LIST;
  const int lane = threadIdx.x & 31;
  const int wib = threadIdx.x >> 5;
  const int ly = lane >> 3, lx = lane & 7;
  unsigned char* base = smem_raw + (size_t)wib * warp_bytes;
  float2* Wm = reinterpret_cast<float2*>(base);
  uint16_t* nzl = reinterpret_cast<uint16_t*>(base + (size_t)wrows * S * sizeof(float2));
  const int64_t items = njobs * (int64_t)chunks_per_job;
  const int64_t nwarps = (int64_t)gridDim.x * TileCfg<MT>::WARPS;
  for (int64_t item = (int64_t)blockIdx.x * TileCfg<MT>::WARPS + wib; item < items; item += nwarps) {
    const int64_t job = item / chunks_per_job;
    const int chunk = (int)(item % chunks_per_job);
    const int m = jobs.m[job];
    const int T = trials > 0 ? trials : m * m;
    const int t_begin = chunk * chunk_trials;
    const int t_end = min(T, t_begin + chunk_trials);
    Pow2Sum acc;
    if (m >= 1 && m <= wrows && t_begin < t_end) {
      const CsrView v = csr_view(arena, jobs.off[job], m, jobs.nnz[job]);
      const int nnz = jobs.nnz[job];
      const bool listed = nnz <= LIST;
      __syncwarp();
      if (listed)
        for (int r = lane; r < m; r += 32)
          for (int q = v.rowptr[r]; q < v.rowptr[r + 1]; ++q) nzl[q] = (uint16_t)((r << 8) | v.col[q]);
      __syncwarp();
      const uint64_t jkey = seed ^ ((uint64_t)job * K_JOB);
      for (int t = t_begin; t < t_end; ++t) {
        const uint64_t tkey = jkey ^ ((uint64_t)t * K_TRIAL);
        float4* W4 = reinterpret_cast<float4*>(Wm);
        for (int e = lane; e < m * S / 2; e += 32) W4[e] = make_float4(0.f, 0.f, 0.f, 0.f);
        __syncwarp();
        if (listed) {
          for (int q = lane; q < nnz; q += 32) {
            const int rc = nzl[q], r = rc >> 8, c = rc & 255;
            const uint64_t h = splitmix64_mix(tkey ^ ((uint64_t)(r * m + c) * K_ENTRY));
            Wm[r * S + c] = cube_root((uint32_t)(((h >> 32) * 3ull) >> 32));
          }
        } else {
          for (int r = 0; r < m; ++r)
            for (int q = v.rowptr[r] + lane; q < v.rowptr[r + 1]; q += 32) {
              const int c = v.col[q];
              const uint64_t h = splitmix64_mix(tkey ^ ((uint64_t)(r * m + c) * K_ENTRY));
              Wm[r * S + c] = cube_root((uint32_t)(((h >> 32) * 3ull) >> 32));
            }
        }
        __syncwarp();
        uint32_t key = 0;
        for (int r = lane; r < m; r += 32) key = max(key, tile_key(Wm[r * S], r));
        float pm = 1.0f;  // |det|^2 = pm * 2^pe
        int pe = 0;
        bool singular = false;
        for (int k = 0; k < m; ++k) {
          key = __reduce_max_sync(0xffffffffu, key);
          const int p = 63 - (int)(key & 63u);
          if (p != k) {
            for (int c = k + lane; c < m; c += 32) {
              const float2 a = Wm[k * S + c];
              Wm[k * S + c] = Wm[p * S + c];
              Wm[p * S + c] = a;
            }
            __syncwarp();
          }
          const float2 piv = Wm[k * S + k];
          const float mag = piv.x * piv.x + piv.y * piv.y;
          if (!(mag > 0.0f)) {
            singular = true;
            break;
          }
          int ex;
          pm = frexpf(pm * mag, &ex);
          pe += ex;
          const float inv = 1.0f / mag;
          const float2 ipiv = make_float2(piv.x * inv, -piv.y * inv);  // 1 / piv
          const int r0 = k + 1 + ((ly - (k + 1)) & 3);
          const int c0 = k + 1 + ((lx - (k + 1)) & 7);
          float2 pk[JMAX];
#pragma unroll
          for (int j = 0; j < JMAX; ++j) {
            const int c = c0 + 8 * j;
            pk[j] = c < m ? Wm[k * S + c] : make_float2(0.f, 0.f);
          }
          const bool keycol = c0 == k + 1;
          const int jw = (m - k - 1 + 7) >> 3;  // columns per lane and row, at most (warp-uniform)
          key = 0;
          for (int r = r0; r < m; r += 4) {
            const float2 a = Wm[r * S + k];
            const float2 f = make_float2(a.x * ipiv.x - a.y * ipiv.y, a.x * ipiv.y + a.y * ipiv.x);
#pragma unroll
            for (int j = 0; j < JMAX; ++j) {
              const int c = c0 + 8 * j;
              if (j < jw && c < m) {
                float2 z = Wm[r * S + c];
                cfms(z, f, pk[j]);
                Wm[r * S + c] = z;
                if (j == 0 && keycol) key = max(key, tile_key(z, r));
              }
            }
          }
          __syncwarp();
        }
        __syncwarp();
        if (!singular) acc.add(pm, pe);
      }
    }
    if (lane == 0) {
      double lmax, lsum;
      acc.lse(lmax, lsum);
      part[item] = make_double2(lmax, lsum);
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

// Thread form for jobs of order m <= MT: every thread runs one whole trial,
// its m x m complex matrix in shared memory laid out [element][lane] so the
// 32 lanes of a warp never conflict.  A warp takes 32 trials of one job;
// the (max, sum) log-sum-exp of each warp's trials goes to part[] and a
// second kernel combines a job's parts.
template <int MT>
struct TCfg {
  static constexpr size_t WARP_BYTES = sizeof(float2) * MT * MT * 32;
  // as many warps as 227 KB of shared memory holds (14 for MT = 8, 9 for 10,
  // 7 for 11, 6 for 12)
  static constexpr int WARPS = (int)(232448 / WARP_BYTES) < 16 ? (int)(232448 / WARP_BYTES) : 16;
  static constexpr size_t SMEM = WARPS * WARP_BYTES;
  static_assert(SMEM <= 232448, "at most 227 KB of dynamic shared memory per block");
};

template <int MT>
__global__ void __launch_bounds__(TCfg<MT>::WARPS * 32)
    k_kklll_thread(JobArrays jobs, int64_t njobs, const uint64_t* __restrict__ arena, int trials, uint64_t seed,
                   int chunks_per_job, double2* __restrict__ part) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int lane = threadIdx.x & 31;
  const int wib = threadIdx.x >> 5;
  float2* Wt = reinterpret_cast<float2*>(smem_raw + (size_t)wib * TCfg<MT>::WARP_BYTES);
#define WT(i, j) Wt[((i) * MT + (j)) * 32 + lane]
  const int64_t items = njobs * (int64_t)chunks_per_job;
  const int64_t nwarps = (int64_t)gridDim.x * TCfg<MT>::WARPS;
  for (int64_t item = (int64_t)blockIdx.x * TCfg<MT>::WARPS + wib; item < items; item += nwarps) {
    const int64_t job = item / chunks_per_job;
    const int chunk = (int)(item % chunks_per_job);
    const int m = jobs.m[job];
    const int T = trials > 0 ? trials : m * m;
    const int t = chunk * 32 + lane;
    Pow2Sum acc;
    if (m >= 1 && m <= MT && t < T) {
      CsrView v = csr_view(arena, jobs.off[job], m, jobs.nnz[job]);
      const uint64_t tkey = seed ^ ((uint64_t)job * K_JOB) ^ ((uint64_t)t * K_TRIAL);
      // the trial matrix padded to MT x MT with the identity: |det| and every
      // pivot of the first m steps are unchanged, the padded pivots are 1, and
      // the loops below run to the compile-time MT (fully unrolled)
#pragma unroll
      for (int i = 0; i < MT; ++i)
#pragma unroll
        for (int j = 0; j < MT; ++j) WT(i, j) = make_float2(i == j && i >= m ? 1.0f : 0.0f, 0.0f);
      for (int i = 0; i < m; ++i)
        for (int q = v.rowptr[i]; q < v.rowptr[i + 1]; ++q) {
          const int j = v.col[q];
          const uint64_t h = splitmix64_mix(tkey ^ ((uint64_t)(i * m + j) * K_ENTRY));
          const int w = (int)(((h >> 32) * 3ull) >> 32);
          WT(i, j) = cube_root((uint32_t)w);
        }
      float pm = 1.0f;
      int pe = 0;
      bool singular = false;
#pragma unroll
      for (int k = 0; k < MT; ++k) {
        if (!singular) {
          int p = k;
          float best = -1.0f;
#pragma unroll
          for (int r = k; r < MT; ++r) {
            const float2 z = WT(r, k);
            const float mg = z.x * z.x + z.y * z.y;
            if (mg > best) {
              best = mg;
              p = r;
            }
          }
          if (!(best > 0.0f)) {
            singular = true;
          } else {
            if (p != k) {
#pragma unroll
              for (int c = k; c < MT; ++c) {
                const float2 a = WT(k, c);
                WT(k, c) = WT(p, c);
                WT(p, c) = a;
              }
            }
            int ex;
            pm = frexpf(pm * best, &ex);
            pe += ex;
            const float2 piv = WT(k, k);
            const float inv = 1.0f / best;
            const float2 ip = make_float2(piv.x * inv, -piv.y * inv);
            // the pivot row's tail in registers; each trailing element is
            // loaded and stored once per step
            float2 pc[MT];
#pragma unroll
            for (int c = k + 1; c < MT; ++c) pc[c] = WT(k, c);
#pragma unroll
            for (int r = k + 1; r < MT; ++r) {
              const float2 a = WT(r, k);
              const float2 f = make_float2(a.x * ip.x - a.y * ip.y, a.x * ip.y + a.y * ip.x);
#pragma unroll
              for (int c = k + 1; c < MT; ++c) {
                float2 z = WT(r, c);
                cfms(z, f, pc[c]);
                WT(r, c) = z;
              }
            }
          }
        }
      }
      if (!singular) acc.add(pm, pe);
    }
#undef WT
    // sum of the warp's 32 trials
    acc.warp_merge(1);
    double lmax, lsum;
    acc.lse(lmax, lsum);
    if (lane == 0) part[item] = make_double2(lmax, lsum);
  }
}

// Register form for jobs of order m <= MT, several rows per lane: a group
// of LPG = MT / RPL lanes runs one trial, lane i holding rows i*RPL ..
// i*RPL+RPL-1 of the trial matrix in registers, so a warp runs 32 / LPG
// trials side by side with no shared memory.  Rows never move: the pivot of
// step k is the row not yet pivoted with the largest |z|^2, ties (within
// 2^-15 relative) to the row at the lowest position (positions follow the
// row swaps of partial pivoting, so the pivot sequence is that of the
// swapping elimination), and the pivot row is broadcast column by column
// with a shuffle from the lane holding it.  |det W|^2 is the product of the
// pivots' |z|^2.  A warp takes 32 trials of one job (LPG rounds of 32 / LPG
// trials) and writes their sum to part[], which k_kklll_combine merges per
// job.
template <int MT, int RPL>
__global__ void __launch_bounds__(256, 2)
    k_kklll_lanes(JobArrays jobs, int64_t njobs, const uint64_t* __restrict__ arena, int trials, uint64_t seed,
                  int chunks_per_job, double2* __restrict__ part) {
  constexpr int LPG = MT / RPL;   // lanes per trial
  constexpr int TPR = 32 / LPG;   // trials per warp and round
  static_assert(MT % RPL == 0 && 32 % LPG == 0, "rows must tile the lanes");
  const int lane = threadIdx.x & 31;
  const int li = lane % LPG;
  const int grp = lane / LPG;
  const int64_t items = njobs * (int64_t)chunks_per_job;
  const int64_t nwarps = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t item = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); item < items; item += nwarps) {
    const int64_t job = item / chunks_per_job;
    const int chunk = (int)(item % chunks_per_job);
    const int m = jobs.m[job];
    const int T = trials > 0 ? trials : m * m;
    Pow2Sum acc;
    if (m >= 1 && m <= MT) {
      const CsrView v = csr_view(arena, jobs.off[job], m, jobs.nnz[job]);
      uint32_t pat[RPL];
#pragma unroll
      for (int s = 0; s < RPL; ++s) {
        const int r = li * RPL + s;
        uint32_t b = 0;
        if (r < m)
          for (int q = v.rowptr[r]; q < v.rowptr[r + 1]; ++q) b |= 1u << v.col[q];
        pat[s] = b;
      }
      const uint64_t jkey = seed ^ ((uint64_t)job * K_JOB);
      for (int round = 0; round < 32 / TPR; ++round) {
        const int t0 = chunk * 32 + round * TPR;
        if (t0 >= T) break;
        const int t = t0 + grp;
        const bool live = t < T;
        const uint64_t tkey = jkey ^ ((uint64_t)t * K_TRIAL);
        // cube-root indices of the row's nonzeros, two bits per column
        uint32_t code[RPL];
#pragma unroll
        for (int s = 0; s < RPL; ++s) {
          const int r = li * RPL + s;
          uint32_t cd = 0, b = live ? pat[s] : 0u;
          while (b) {
            const int c = __ffs(b) - 1;
            b &= b - 1;
            const uint64_t h = splitmix64_mix(tkey ^ ((uint64_t)(r * m + c) * K_ENTRY));
            cd |= (uint32_t)(((h >> 32) * 3ull) >> 32) << (2 * c);
          }
          code[s] = cd;
        }
        float2 W[RPL][MT];
#pragma unroll
        for (int s = 0; s < RPL; ++s) {
          const uint32_t on = live ? pat[s] : 0u;
#pragma unroll
          for (int c = 0; c < MT; ++c) {
            W[s][c] = ((on >> c) & 1u) ? cube_root((code[s] >> (2 * c)) & 3u) : make_float2(0.0f, 0.0f);
          }
        }
        int pos[RPL];
        bool done[RPL];
#pragma unroll
        for (int s = 0; s < RPL; ++s) {
          pos[s] = li * RPL + s;
          done[s] = pos[s] >= m;
        }
        float pm = 1.0f;
        int pe = 0;
        bool singular = !live;
#pragma unroll
        for (int k = 0; k < MT; ++k) {
          if (k < m) {
            // key: |z|^2 with its low 8 bits replaced by (15 - position,
            // row), so magnitudes within 2^-15 of each other tie and go to
            // the lower position; a non-negative float orders like its bits
            uint32_t key = 0u;
#pragma unroll
            for (int s = 0; s < RPL; ++s) {
              const float mg = W[s][k].x * W[s][k].x + W[s][k].y * W[s][k].y;
              const uint32_t ks = done[s] ? 0u
                                          : (__float_as_uint(mg) & 0xffffff00u) |
                                                ((uint32_t)(15 - pos[s]) << 4) | (uint32_t)(li * RPL + s);
              key = ks > key ? ks : key;
            }
#pragma unroll
            for (int d = LPG / 2; d > 0; d >>= 1) {
              const uint32_t o = __shfl_xor_sync(0xffffffffu, key, d, LPG);
              key = o > key ? o : key;
            }
            const int pr = (int)(key & 0xf);
            const int ppos = 15 - (int)((key >> 4) & 0xf);
            const int plane = pr / RPL, pslot = pr % RPL;
            // the row now at position k moves to the pivot's old position
#pragma unroll
            for (int s = 0; s < RPL; ++s) {
              if (pos[s] == k) pos[s] = ppos;
              if (li * RPL + s == pr) {
                pos[s] = k;
                done[s] = true;
              }
            }
            float2 sel = W[0][k];
#pragma unroll
            for (int s = 1; s < RPL; ++s)
              if (pslot == s) sel = W[s][k];
            const float2 piv = make_float2(__shfl_sync(0xffffffffu, sel.x, plane, LPG),
                                           __shfl_sync(0xffffffffu, sel.y, plane, LPG));
            const float pmag = piv.x * piv.x + piv.y * piv.y;
            if (!(pmag > 0.0f)) singular = true;
            if (!singular) {
              int ex;
              pm = frexpf(pm * pmag, &ex);
              pe += ex;
            }
            const float inv = singular ? 0.0f : 1.0f / pmag;
            float2 f[RPL];
#pragma unroll
            for (int s = 0; s < RPL; ++s) {
              const float2 a = W[s][k];
              f[s] = done[s] ? make_float2(0.0f, 0.0f)
                             : make_float2((a.x * piv.x + a.y * piv.y) * inv, (a.y * piv.x - a.x * piv.y) * inv);
            }
#pragma unroll
            // (constant bounds, so the loop unrolls with the step loop and
            // every register index stays a constant)
            for (int c = 1; c < MT; ++c) {
              if (c > k) {  // columns >= m are zero in every row
                float2 ps = W[0][c];
#pragma unroll
                for (int s = 1; s < RPL; ++s)
                  if (pslot == s) ps = W[s][c];
                const float2 pc = make_float2(__shfl_sync(0xffffffffu, ps.x, plane, LPG),
                                              __shfl_sync(0xffffffffu, ps.y, plane, LPG));
#pragma unroll
                for (int s = 0; s < RPL; ++s) {
                  cfms(W[s][c], f[s], pc);
                }
              }
            }
          }
        }
        if (!singular) acc.add(pm, pe);
      }
    }
    // the groups' sums (every lane of a group holds its group's), merged
    acc.warp_merge(LPG);
    double lmax, lsum;
    acc.lse(lmax, lsum);
    if (lane == 0) part[item] = make_double2(lmax, lsum);
  }
}

__global__ void k_kklll_combine(JobArrays jobs, int64_t njobs, int trials, int chunks_per_job,
                                const double2* __restrict__ part, float* __restrict__ log_ap) {
  const int64_t job = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (job >= njobs) return;
  const int m = jobs.m[job];
  const int T = trials > 0 ? trials : m * m;
  double lmax = -INFINITY, lsum = 0.0;
  for (int c = 0; c < chunks_per_job; ++c) {
    const double2 p = part[job * chunks_per_job + c];
    if (p.x == -INFINITY) continue;
    if (p.x > lmax) {
      lsum = (lmax > -INFINITY ? lsum * exp(lmax - p.x) : 0.0) + p.y;
      lmax = p.x;
    } else {
      lsum += p.y * exp(p.x - lmax);
    }
  }
  log_ap[job] = m == 0 ? 0.0f : (lmax == -INFINITY ? -INFINITY : (float)(lmax + log(lsum / (double)T)));
}

template <int MT>
cudaError_t launch_thread(const JobArrays& jobs, int64_t njobs, const uint64_t* arena, int trials, uint64_t seed,
                          float* log_ap, double2* part, int chunks, cudaStream_t s) {
  typedef TCfg<MT> C;
  static bool attr_set = false;
  if (!attr_set) {
    cudaError_t e =
        cudaFuncSetAttribute(k_kklll_thread<MT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::SMEM);
    if (e != cudaSuccess) return e;
    attr_set = true;
  }
  const int64_t items = njobs * chunks;
  int64_t blocks = (items + C::WARPS - 1) / C::WARPS;
  if (blocks > 152 * 16) blocks = 152 * 16;
  k_kklll_thread<MT><<<(unsigned)blocks, C::WARPS * 32, C::SMEM, s>>>(jobs, njobs, arena, trials, seed, chunks,
                                                                     part);
  k_kklll_combine<<<(unsigned)((njobs + 255) / 256), 256, 0, s>>>(jobs, njobs, trials, chunks, part, log_ap);
  return cudaGetLastError();
}

template <int MT, int RPL>
cudaError_t launch_lanes(const JobArrays& jobs, int64_t njobs, const uint64_t* arena, int trials, uint64_t seed,
                         float* log_ap, double2* part, int chunks, cudaStream_t s) {
  const int64_t items = njobs * chunks;
  int64_t blocks = (items + 7) / 8;
  if (blocks > 152 * 8) blocks = 152 * 8;
  k_kklll_lanes<MT, RPL><<<(unsigned)blocks, 256, 0, s>>>(jobs, njobs, arena, trials, seed, chunks, part);
  k_kklll_combine<<<(unsigned)((njobs + 255) / 256), 256, 0, s>>>(jobs, njobs, trials, chunks, part, log_ap);
  return cudaGetLastError();
}

static size_t tile_warp_bytes(int mmax) {
  return ((size_t)mmax * tile_stride(mmax) * sizeof(float2) + 2 * TileCfg<64>::LIST + 15) / 16 * 16;
}

template <int MT>
cudaError_t launch_tile(const JobArrays& jobs, int64_t njobs, const uint64_t* arena, int trials, uint64_t seed,
                        float* log_ap, double2* part, int chunks, int chunk_trials, int max_order, cudaStream_t s) {
  typedef TileCfg<MT> C;
  static bool attr_set = false;
  if (!attr_set) {
    cudaError_t e = cudaFuncSetAttribute(k_kklll_tile<MT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)(C::WARPS * tile_warp_bytes(MT)));
    if (e != cudaSuccess) return e;
    attr_set = true;
  }
  const int wb = (int)tile_warp_bytes(max_order);
  const int smem = C::WARPS * wb;
  const int64_t items = njobs * chunks;
  int64_t blocks = (items + C::WARPS - 1) / C::WARPS;
  if (blocks > 152 * 64) blocks = 152 * 64;
  k_kklll_tile<MT><<<(unsigned)blocks, C::WARPS * 32, smem, s>>>(jobs, njobs, arena, trials, seed, chunks,
                                                                  chunk_trials, tile_stride(max_order), max_order,
                                                                  wb, part);
  k_kklll_combine<<<(unsigned)((njobs + 255) / 256), 256, 0, s>>>(jobs, njobs, trials, chunks, part, log_ap);
  return cudaGetLastError();
}


}  // namespace

// Trials per part: 32 (one per lane, or per lane group, of a warp) up to
// order 16; for the tile form 32 doubled until the parts number at most
// 2^23 (128 MB).
static int kklll_chunk_trials(int64_t njobs, int max_order, int trials) {
  if (max_order <= 16 || max_order > 64) return 32;
  const int64_t T = trials > 0 ? trials : (int64_t)max_order * max_order;
  int ct = 32;
  while ((T + ct - 1) / ct * (njobs > 0 ? njobs : 1) > (1ll << 23) && ct < (1 << 20)) ct *= 2;
  return ct;
}

static int kklll_chunks(int64_t njobs, int max_order, int trials) {
  const int64_t T = trials > 0 ? trials : (int64_t)max_order * max_order;
  const int ct = kklll_chunk_trials(njobs, max_order, trials);
  return (int)((T + ct - 1) / ct);
}

static bool kklll_uses_parts(int max_order) { return max_order <= 64; }

size_t kklll_scratch_bytes(int64_t njobs, int max_order, int trials) {
  if (!kklll_uses_parts(max_order)) return 16;
  return sizeof(double2) * (size_t)(njobs > 0 ? njobs : 1) * (size_t)kklll_chunks(njobs, max_order, trials);
}

cudaError_t launch_kklll(const JobArrays& jobs, int64_t njobs, const uint64_t* arena, int trials, uint64_t seed,
                         float* log_ap, int max_order, void* scratch, cudaStream_t s) {
  if (njobs <= 0) return cudaSuccess;
  double2* part = reinterpret_cast<double2*>(scratch);
  const int chunks = kklll_chunks(njobs, max_order, trials);
  if (max_order <= 8) return launch_thread<8>(jobs, njobs, arena, trials, seed, log_ap, part, chunks, s);
  // jobs of order 9-12 padded to the next of 10, 11, 12 (less padding: fewer
  // flops and more warps per SM)
  if (max_order <= 10) return launch_thread<10>(jobs, njobs, arena, trials, seed, log_ap, part, chunks, s);
  if (max_order <= 11) return launch_thread<11>(jobs, njobs, arena, trials, seed, log_ap, part, chunks, s);
  if (max_order <= 12) return launch_thread<12>(jobs, njobs, arena, trials, seed, log_ap, part, chunks, s);
  if (max_order <= 16) return launch_lanes<16, 2>(jobs, njobs, arena, trials, seed, log_ap, part, chunks, s);
  const int ct = kklll_chunk_trials(njobs, max_order, trials);
  if (max_order <= 24) return launch_tile<24>(jobs, njobs, arena, trials, seed, log_ap, part, chunks, ct, max_order, s);
  if (max_order <= 32) return launch_tile<32>(jobs, njobs, arena, trials, seed, log_ap, part, chunks, ct, max_order, s);
  if (max_order <= 40) return launch_tile<40>(jobs, njobs, arena, trials, seed, log_ap, part, chunks, ct, max_order, s);
  if (max_order <= 48) return launch_tile<48>(jobs, njobs, arena, trials, seed, log_ap, part, chunks, ct, max_order, s);
  if (max_order <= 56) return launch_tile<56>(jobs, njobs, arena, trials, seed, log_ap, part, chunks, ct, max_order, s);
  if (max_order <= 64) return launch_tile<64>(jobs, njobs, arena, trials, seed, log_ap, part, chunks, ct, max_order, s);
  return launch_k<128>(jobs, njobs, arena, trials, seed, log_ap, s);
}
