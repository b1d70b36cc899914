// K3: persistent evaluator.  Warps pull jobs from the ordered queue through
// one atomic counter (Algorithm PH, Step 3: the next job goes to the next
// free worker) and evaluate each by Algorithm H_per (Section 2.1): Eq. 2
// depth first while the order exceeds max(L, 2) and s < 5, Ryser /
// Nijenhuis-Wilf (ryser.cuh) at the leaves.
//
// The job lives in a dense int64 tile in shared memory.  Lines are never
// moved: deleting a row or column clears a bit of the active masks R and C,
// so "lowest index" keeps the meaning it has in the compacted matrices of
// the oracle.  A merge overwrites one line in place after saving it to the
// warp's undo stack in global memory; backtracking restores it.  Nonzero
// patterns are kept as bit masks per row (rowbits) and per column (colbits),
// so a line count is one popcount against the active masks.
#include <cuda_runtime.h>

#include <cstdint>

#include "internal.h"
#include "ryser.cuh"
#include "wide.cuh"

namespace {

template <int TILE>
struct DfsCfg {
  static constexpr int STRIDE = TILE + 1;
  static constexpr int WARPS = TILE <= 32 ? 8 : 4;
  static constexpr size_t TILE_BYTES = sizeof(int64_t) * TILE * STRIDE;
  static constexpr size_t MASK_BYTES = 2 * sizeof(uint64_t) * TILE;
  static constexpr size_t LEAF_BYTES = sizeof(int32_t) * ((PERM_MAX_LEAF - 1) * 32 + 32);
  static constexpr size_t WARP_BYTES = TILE_BYTES + MASK_BYTES + LEAF_BYTES;
  static constexpr size_t SMEM = WARPS * WARP_BYTES;
  // undo stack words per level: meta (8 x int32 = 4 words), pv[4], coef[4], saved mask, line[TILE]
  static constexpr int FRAME_WORDS = 4 + 4 + 4 + 1 + TILE;
  static constexpr int64_t UNDO_WORDS = (int64_t)FRAME_WORDS * TILE;
};

struct Frame {
  int32_t is_col, idx, k, child;
  int32_t pos[4];
};

__device__ __forceinline__ unsigned long long warp_min_u64(unsigned long long v) {
#pragma unroll
  for (int d = 16; d > 0; d >>= 1) {
    unsigned long long o = __shfl_xor_sync(0xffffffffu, v, d);
    v = o < v ? o : v;
  }
  return v;
}

__device__ __forceinline__ bool mad2_checked(int64_t a, int64_t x, int64_t b, int64_t y, int64_t& out) {
  __int128 r = (__int128)a * x + (__int128)b * y;
  out = (int64_t)r;
  return r == (__int128)out;
}

// index of the (n+1)-th set bit of a 64-bit mask
__device__ __forceinline__ int nth_bit(uint64_t mask, int n) {
  const uint32_t lo = (uint32_t)mask;
  const int plo = __popc(lo);
  if (n < plo) return __fns(lo, 0, n + 1);
  return 32 + __fns((uint32_t)(mask >> 32), 0, n - plo + 1);
}

__device__ __forceinline__ uint64_t bit64(int i) { return 1ull << i; }

template <int TILE>
struct Dfs {
  static constexpr int S = DfsCfg<TILE>::STRIDE;
  static constexpr int RPL = TILE / 32;  // lines per lane
  int64_t* T;
  uint64_t* rowbits;
  uint64_t* colbits;
  int32_t* delta;
  int32_t* rho0;
  int64_t* undo;
  int lane;
  uint64_t R, C;
  u256 coef;

  __device__ int64_t* frame_words(int lv) { return undo + (int64_t)lv * DfsCfg<TILE>::FRAME_WORDS; }

  __device__ void store_frame(int lv, const Frame& f, const int64_t* pv, const u256& c) {
    int64_t* w = frame_words(lv);
    if (lane == 0) {
      int32_t* m = reinterpret_cast<int32_t*>(w);
      m[0] = f.is_col;
      m[1] = f.idx;
      m[2] = f.k;
      m[3] = f.child;
      for (int t = 0; t < 4; ++t) m[4 + t] = f.pos[t];
      for (int t = 0; t < 4; ++t) w[4 + t] = pv[t];
      for (int t = 0; t < 4; ++t) w[8 + t] = (int64_t)c.w[t];
    }
  }
  __device__ void load_frame(int lv, Frame& f, int64_t* pv, u256& c) {
    const int64_t* w = frame_words(lv);
    const int32_t* m = reinterpret_cast<const int32_t*>(w);
    f.is_col = m[0];
    f.idx = m[1];
    f.k = m[2];
    f.child = m[3];
    for (int t = 0; t < 4; ++t) f.pos[t] = m[4 + t];
    for (int t = 0; t < 4; ++t) pv[t] = w[4 + t];
    for (int t = 0; t < 4; ++t) c.w[t] = (uint64_t)w[8 + t];
  }
  __device__ void set_child(int lv, int child) {
    if (lane == 0) reinterpret_cast<int32_t*>(frame_words(lv))[3] = child;
  }

  // child c of a frame: kind 1 = merge(pos[x], pos[x+1]), 2 = minor(pos[x])
  __device__ static void child_kind(int k, int c, int& kind, int& x) {
    if (c == 0) {
      kind = k == 1 ? 2 : 1;
      x = 0;
    } else {
      kind = k == 3 ? 2 : 1;
      x = 2;
    }
  }
  __device__ static int nchildren(int k) { return (k == 3 || k == 4) ? 2 : 1; }

  // Apply child c; returns false on int64 overflow of a merged entry.
  __device__ bool apply(int lv, const Frame& f, const int64_t* pv, int c) {
    int kind, x;
    child_kind(f.k, c, kind, x);
    int64_t* saved = frame_words(lv) + 13;
    bool ok = true;
    if (!f.is_col) {
      const int i = f.idx;
      if (kind == 2) {
        R &= ~bit64(i);
        C &= ~bit64(f.pos[x]);
        coef = u256_mul_s64(coef, pv[x]);
        return true;
      }
      const int p = f.pos[x], q = f.pos[x + 1];
      const int64_t a = pv[x], b = pv[x + 1];
      R &= ~bit64(i);
      C &= ~bit64(q);
      uint64_t nzbits = 0;
#pragma unroll
      for (int t = 0; t < RPL; ++t) {
        const int r = lane + 32 * t;
        bool nz = false;
        if ((R >> r) & 1) {
          const int64_t old = T[r * S + p];
          int64_t nv;
          if (!mad2_checked(a, T[r * S + q], b, old, nv)) ok = false;
          saved[r] = old;
          T[r * S + p] = nv;
          nz = nv != 0;
          if (nz) rowbits[r] |= bit64(p); else rowbits[r] &= ~bit64(p);
        }
        const uint32_t bal = __ballot_sync(0xffffffffu, nz);
        nzbits |= (uint64_t)bal << (32 * t);
      }
      if (lane == 0) {
        saved[-1] = (int64_t)colbits[p];
        colbits[p] = nzbits;
      }
    } else {
      const int j = f.idx;
      if (kind == 2) {
        C &= ~bit64(j);
        R &= ~bit64(f.pos[x]);
        coef = u256_mul_s64(coef, pv[x]);
        return true;
      }
      const int p = f.pos[x], q = f.pos[x + 1];
      const int64_t a = pv[x], b = pv[x + 1];
      C &= ~bit64(j);
      R &= ~bit64(q);
      uint64_t nzbits = 0;
#pragma unroll
      for (int t = 0; t < RPL; ++t) {
        const int cc = lane + 32 * t;
        bool nz = false;
        if ((C >> cc) & 1) {
          const int64_t old = T[p * S + cc];
          int64_t nv;
          if (!mad2_checked(a, T[q * S + cc], b, old, nv)) ok = false;
          saved[cc] = old;
          T[p * S + cc] = nv;
          nz = nv != 0;
          if (nz) colbits[cc] |= bit64(p); else colbits[cc] &= ~bit64(p);
        }
        const uint32_t bal = __ballot_sync(0xffffffffu, nz);
        nzbits |= (uint64_t)bal << (32 * t);
      }
      if (lane == 0) {
        saved[-1] = (int64_t)rowbits[p];
        rowbits[p] = nzbits;
      }
    }
    __syncwarp();
    return __all_sync(0xffffffffu, ok);
  }

  __device__ void undo_child(int lv, const Frame& f, const int64_t* pv, const u256& pcoef, int c) {
    int kind, x;
    child_kind(f.k, c, kind, x);
    const int64_t* saved = frame_words(lv) + 13;
    coef = pcoef;
    if (!f.is_col) {
      const int i = f.idx;
      R |= bit64(i);
      if (kind == 2) {
        C |= bit64(f.pos[x]);
        return;
      }
      const int p = f.pos[x], q = f.pos[x + 1];
      C |= bit64(q);
#pragma unroll
      for (int t = 0; t < RPL; ++t) {
        const int r = lane + 32 * t;
        if (r != i && ((R >> r) & 1)) {
          const int64_t old = saved[r];
          T[r * S + p] = old;
          if (old != 0) rowbits[r] |= bit64(p); else rowbits[r] &= ~bit64(p);
        }
      }
      if (lane == 0) colbits[p] = (uint64_t)saved[-1];
    } else {
      const int j = f.idx;
      C |= bit64(j);
      if (kind == 2) {
        R |= bit64(f.pos[x]);
        return;
      }
      const int p = f.pos[x], q = f.pos[x + 1];
      R |= bit64(q);
#pragma unroll
      for (int t = 0; t < RPL; ++t) {
        const int cc = lane + 32 * t;
        if (cc != j && ((C >> cc) & 1)) {
          const int64_t old = saved[cc];
          T[p * S + cc] = old;
          if (old != 0) colbits[cc] |= bit64(p); else colbits[cc] &= ~bit64(p);
        }
      }
      if (lane == 0) rowbits[p] = (uint64_t)saved[-1];
    }
    __syncwarp();
  }

  // smallest line count over the active lines: (s << 17) | (is_col << 16) | index
  __device__ unsigned long long pivot_key() {
    unsigned long long key = ~0ull;
#pragma unroll
    for (int t = 0; t < RPL; ++t) {
      const int r = lane + 32 * t;
      if ((R >> r) & 1) key = min(key, ((unsigned long long)__popcll(rowbits[r] & C) << 17) | (unsigned long long)r);
      if ((C >> r) & 1)
        key = min(key, ((unsigned long long)__popcll(colbits[r] & R) << 17) | (1ull << 16) | (unsigned long long)r);
    }
    return warp_min_u64(key);
  }

  // Ryser on the active sub-matrix; adds coef * per into acc (lane 0).
  __device__ bool leaf(int W, u256& acc) {
    const int m = __popcll(R);
    const int nmax = nmax_for(m);
    bool ok = true;
    if (m == 1) {
      const int r = __ffsll((long long)R) - 1, c = __ffsll((long long)C) - 1;
      if (lane == 0) acc = u256_add(acc, u256_mul_s64(coef, T[r * S + c]));
      return true;
    }
    if (m > PERM_MAX_LEAF) return false;
    const int cols = m - 1;
    for (int k = lane; k < cols * nmax; k += 32) delta[k] = 0;
    __syncwarp();
    int64_t rmax = 0;
    for (int ii = lane; ii < nmax; ii += 32) {
      if (ii >= m) {
        rho0[ii] = 1;
        continue;
      }
      const int r = nth_bit(R, ii);
      int64_t rs = 0, ra = 0, last = 0;
      uint64_t cm = C;
      int jj = 0;
      while (cm) {
        const int c = __ffsll((long long)cm) - 1;
        cm &= cm - 1;
        const int64_t a = T[r * S + c];
        if (a >= (1ll << 30) || a <= -(1ll << 30)) ok = false;
        rs += a;
        ra += a < 0 ? -a : a;
        if (jj < cols) delta[jj * nmax + ii] = (int32_t)(2 * a); else last = a;
        ++jj;
      }
      if (ra >= (1ll << 31)) ok = false;
      rmax = ra > rmax ? ra : rmax;
      rho0[ii] = (int32_t)(2 * last - rs);
    }
    ok = __all_sync(0xffffffffu, ok);
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) {
      int64_t o = __shfl_xor_sync(0xffffffffu, rmax, d);
      rmax = o > rmax ? o : rmax;
    }
    __syncwarp();
    if (!ok) return false;
    const int bc = bit_class(rmax);
    const int e = m - 1;
    int lanes;
    uint64_t cnt;
    if (e <= 5) {
      lanes = 1 << (e - 1);
      cnt = 2;
    } else {
      lanes = 32;
      cnt = 1ull << (e - 5);
    }
    uint64_t words[4] = {0, 0, 0, 0};
    const uint64_t gb = (uint64_t)lane * cnt;
    dispatch_lane(nmax, W, bc, delta, rho0, m, gb, lane < lanes ? cnt : 0, words);
    if (lane == 0) {
      u256 s;
      for (int k = 0; k < 4; ++k) s.w[k] = words[k];
      s = u256_shr(s, m - 1);
      if ((m - 1) & 1) s = u256_neg(s);
      acc = u256_add(acc, u256_mul(s, coef));
    }
    __syncwarp();
    return true;
  }
};

template <int TILE>
__global__ void __launch_bounds__(DfsCfg<TILE>::WARPS * 32) k_dfs(DfsArgs A) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  typedef DfsCfg<TILE> Cfg;
  constexpr int S = Cfg::STRIDE;
  const int lane = threadIdx.x & 31;
  const int wib = threadIdx.x >> 5;
  unsigned char* base = smem_raw + (size_t)wib * Cfg::WARP_BYTES;
  Dfs<TILE> D;
  D.T = reinterpret_cast<int64_t*>(base);
  D.rowbits = reinterpret_cast<uint64_t*>(base + Cfg::TILE_BYTES);
  D.colbits = D.rowbits + TILE;
  D.delta = reinterpret_cast<int32_t*>(base + Cfg::TILE_BYTES + Cfg::MASK_BYTES);
  D.rho0 = D.delta + (PERM_MAX_LEAF - 1) * 32;
  const int64_t gwarp = (int64_t)blockIdx.x * Cfg::WARPS + wib;
  D.undo = A.undo + gwarp * A.undo_words_per_warp;
  D.lane = lane;
  const int cut = A.leaf_size > 2 ? A.leaf_size : 2;

  for (;;) {
    unsigned long long qi = 0;
    if (lane == 0) qi = atomicAdd(A.job_counter, 1ull);
    qi = __shfl_sync(0xffffffffu, qi, 0);
    if (qi >= (unsigned long long)A.nq) break;
    const uint32_t job = A.queue[qi];
    const uint64_t t0 = globaltimer_ns();
    const int m = A.jobs.m[job];
    const int nnz = A.jobs.nnz[job];
    const int W = A.mat_w[A.jobs.mat[job]];
    int status = 0;
    u256 acc = u256_zero();
    unsigned long long nodes = 0, leaves = 0;
    if (m > TILE) {
      status = PERM_EINVAL;
    } else {
      // load the job into the tile and its masks
      CsrView v = csr_view(A.arena, A.jobs.off[job], m, nnz);
      for (int k = lane; k < TILE * S; k += 32) D.T[k] = 0;
      for (int k = lane; k < TILE; k += 32) D.rowbits[k] = D.colbits[k] = 0;
      __syncwarp();
      for (int r = lane; r < m; r += 32) {
        uint64_t rb = 0;
        for (int q = v.rowptr[r]; q < v.rowptr[r + 1]; ++q) {
          const int c = v.col[q];
          D.T[r * S + c] = v.val[q];
          rb |= bit64(c);
          atomicOr((unsigned long long*)&D.colbits[c], (unsigned long long)bit64(r));
        }
        D.rowbits[r] = rb;
      }
      __syncwarp();
      D.R = D.C = (m == 64) ? ~0ull : (bit64(m) - 1);
      for (int t = 0; t < 4; ++t) D.coef.w[t] = A.jobs.coef[4ll * job + t];
      int depth = 0;
      bool done = false;
      while (!done) {
        // ---- visit the current node
        ++nodes;
        if ((nodes & 4095) == 0 && A.timeout_ns > 0 && (int64_t)(globaltimer_ns() - t0) > A.timeout_ns) {
          status = PERM_ETIMEOUT;
          break;
        }
        const unsigned long long key = D.pivot_key();
        const int s = (int)(key >> 17);
        const int mact = __popcll(D.R);
        bool descend = false;
        if (s > 0) {
          if (mact <= cut || s >= 5) {
            ++leaves;
            if (!D.leaf(W, acc)) {
              status = mact > PERM_MAX_LEAF ? PERM_EINVAL : PERM_EOVERFLOW;
              break;
            }
          } else if (depth >= TILE - 1) {
            status = PERM_EINVAL;
            break;
          } else {
            Frame f;
            f.is_col = (int)((key >> 16) & 1);
            f.idx = (int)(key & 0xffff);
            f.k = s;
            f.child = 0;
            int64_t pv[4] = {0, 0, 0, 0};
            uint64_t line = f.is_col ? (D.colbits[f.idx] & D.R) : (D.rowbits[f.idx] & D.C);
            for (int t = 0; t < 4; ++t) {
              if (line) {
                const int c = __ffsll((long long)line) - 1;
                line &= line - 1;
                f.pos[t] = c;
                pv[t] = f.is_col ? D.T[c * S + f.idx] : D.T[f.idx * S + c];
              } else {
                f.pos[t] = 0;
              }
            }
            D.store_frame(depth, f, pv, D.coef);
            __syncwarp();
            if (!D.apply(depth, f, pv, 0)) {
              status = PERM_EOVERFLOW;
              break;
            }
            ++depth;
            descend = true;
          }
        }
        if (descend) continue;
        // ---- backtrack to the next unvisited child
        for (;;) {
          if (depth == 0) {
            done = true;
            break;
          }
          Frame f;
          int64_t pv[4];
          u256 pc;
          D.load_frame(depth - 1, f, pv, pc);
          D.undo_child(depth - 1, f, pv, pc, f.child);
          if (f.child + 1 < Dfs<TILE>::nchildren(f.k)) {
            f.child += 1;
            D.set_child(depth - 1, f.child);
            __syncwarp();
            if (!D.apply(depth - 1, f, pv, f.child)) {
              status = PERM_EOVERFLOW;
              done = true;
            }
            break;
          }
          --depth;
        }
      }
    }
    if (lane == 0) {
      const uint64_t t1 = globaltimer_ns();
      A.out.status[job] = status;
      A.out.t_start[job] = t0;
      A.out.t_end[job] = t1;
      A.out.sm[job] = (int32_t)smid();
      A.out.leaves[job] = leaves;
      A.out.nodes[job] = nodes;
      for (int t = 0; t < 4; ++t) A.out.acc[4ll * job + t] = acc.w[t];
      if (status == 0) atomic_add_words(A.mat_acc + 4ll * A.jobs.mat[job], acc.w, 4);
    }
    __syncwarp();
  }
}

template <int TILE>
cudaError_t launch_dfs_tile(const DfsArgs& a, int num_sms, int warps_per_sm, cudaStream_t s) {
  typedef DfsCfg<TILE> C;
  static bool attr_set = false;
  if (!attr_set) {
    cudaError_t e = cudaFuncSetAttribute(k_dfs<TILE>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::SMEM);
    if (e != cudaSuccess) return e;
    attr_set = true;
  }
  int blocks_per_sm = (warps_per_sm + C::WARPS - 1) / C::WARPS;
  if (blocks_per_sm < 1) blocks_per_sm = 1;
  k_dfs<TILE><<<num_sms * blocks_per_sm, C::WARPS * 32, C::SMEM, s>>>(a);
  return cudaGetLastError();
}

}  // namespace

size_t dfs_smem_bytes(int tile) { return tile <= 32 ? DfsCfg<32>::SMEM : DfsCfg<64>::SMEM; }
int dfs_warps_per_block(int tile) { return tile <= 32 ? DfsCfg<32>::WARPS : DfsCfg<64>::WARPS; }
int64_t dfs_undo_words(int tile) { return tile <= 32 ? DfsCfg<32>::UNDO_WORDS : DfsCfg<64>::UNDO_WORDS; }

cudaError_t launch_dfs(const DfsArgs& a, int tile, int num_sms, int warps_per_sm, cudaStream_t s) {
  if (a.nq <= 0) return cudaSuccess;
  if (tile <= 32) return launch_dfs_tile<32>(a, num_sms, warps_per_sm, s);
  return launch_dfs_tile<64>(a, num_sms, warps_per_sm, s);
}
