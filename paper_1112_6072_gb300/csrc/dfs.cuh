// The depth-first evaluator's node machinery on a warp's tile (Algorithm
// H_per, Section 2.1): its configuration, the leaf evaluation and the walk
// of one job.  Shared by the depth-first kernels (dfs.cu) and the
// single-launch evaluator (persist.cu).
#pragma once
#include <cuda_runtime.h>

#include <cstdint>

#include "internal.h"
#include "ryser.cuh"
#include "ryser4.cuh"
#include "ryser_mod.cuh"
#include "tile.cuh"
#include "wide.cuh"

namespace {

template <int TILE, typename E>
struct DfsCfg {
  static constexpr int STRIDE = TileCfg<TILE, E>::STRIDE;
  static constexpr int WARPS = sizeof(E) == 4 ? (TILE <= 32 ? 8 : 5) : (TILE <= 32 ? 8 : 4);
  // blocks per SM the register budget is sized for (shared memory allows this many)
  static constexpr int MINB = (sizeof(E) == 4 && TILE <= 32) ? 2 : 1;
  static constexpr size_t TILE_BYTES = TileCfg<TILE, E>::TILE_BYTES;
  static constexpr size_t MASK_BYTES = TileCfg<TILE, E>::MASK_BYTES;
  // delta, rho0, column masks of the leaf
  static constexpr size_t LEAF_BYTES = sizeof(int32_t) * ((PERM_MAX_LEAF - 1) * 32 + 32 + 32);
  static constexpr size_t WARP_BYTES = TILE_BYTES + MASK_BYTES + LEAF_BYTES;
  static constexpr size_t SMEM = WARPS * WARP_BYTES;
  static constexpr int FRAME_WORDS = TileCfg<TILE, E>::FRAME_WORDS;
};

// One leaf walk per (NMAX, W, path), inlined (measured 2-3 % faster than
// out of line: the walk keeps the registers it needs).
// path: 0/1/2 plain walk with bit class 7/15/31, 3 blocked NN=8, 4 blocked NN=16
template <int NM, int W, int PATH>
__device__ __forceinline__ void leaf_walk(const int32_t* delta, const int32_t* rho0, int m, uint64_t gb, uint64_t cnt,
                                       uint64_t* words) {
  if constexpr (PATH == 3) {
    run_lane4<NM, 8, W, false, false>(delta, rho0, m, gb, cnt, words);
  } else if constexpr (PATH == 4) {
    run_lane4<NM, 16, W, false, false>(delta, rho0, m, gb, cnt, words);
  } else {
    typename WideT<W>::type s =
        ryser_lane<NM, W, PATH == 0 ? 7 : (PATH == 1 ? 15 : 31), false>(delta, rho0, m, gb, cnt);
    s = warp_sum(s);
    to_words(s, words);
  }
}

template <int NM, int W>
__device__ __forceinline__ void leaf_paths(int path, const int32_t* delta, const int32_t* rho0, int m, uint64_t gb,
                                           uint64_t cnt, uint64_t* words) {
  switch (path) {
    case 0: leaf_walk<NM, W, 0>(delta, rho0, m, gb, cnt, words); break;
    case 1: leaf_walk<NM, W, 1>(delta, rho0, m, gb, cnt, words); break;
    case 2: leaf_walk<NM, W, 2>(delta, rho0, m, gb, cnt, words); break;
    case 3: leaf_walk<NM, W, 3>(delta, rho0, m, gb, cnt, words); break;
    default:
      if constexpr (NM >= 16) leaf_walk<NM, W, 4>(delta, rho0, m, gb, cnt, words);
      break;
  }
}

// Lane shares of one leaf, summed over the warp into lane 0's words.  The
// narrow variant (LN = 16) holds every leaf in 16 register rows.
template <int LN, int W>
__device__ __forceinline__ void leaf_dispatch(int nmax, int path, const int32_t* delta, const int32_t* rho0,
                                              int m, uint64_t gb, uint64_t cnt, uint64_t* words) {
  if constexpr (LN <= 16) {
    leaf_paths<16, W>(path, delta, rho0, m, gb, cnt, words);
  } else {
    if (nmax == 8) leaf_paths<8, W>(path, delta, rho0, m, gb, cnt, words);
    else if (nmax == 16) leaf_paths<16, W>(path, delta, rho0, m, gb, cnt, words);
    else if (nmax == 24) leaf_paths<24, W>(path, delta, rho0, m, gb, cnt, words);
    else leaf_paths<32, W>(path, delta, rho0, m, gb, cnt, words);
  }
}

template <int TILE, typename E, int LN, int W>
struct Dfs : Eq2Tile<TILE, E> {
  typedef Eq2Tile<TILE, E> Base;
  using Base::S;
  using Base::T;
  using Base::rowbits;
  using Base::colbits;
  using Base::lane;
  using Base::R;
  using Base::C;
  using Base::coef;
  int32_t* delta;
  int32_t* rho0;
  uint32_t* cmask;
  ModP mod;

  // Ryser on the active sub-matrix; adds coef * per into acc (lane 0).
  // Returns a status: 0, PERM_EOVERFLOW, PERM_EINVAL, or DFS_RETRY.
  __device__ int leaf(u256& acc) {
    if constexpr (W == 0)
      return leaf_mod(acc);
    else
      return leaf_ring(acc);
  }

  // The residue path: acc.w[0] = (acc.w[0] + coef * per) mod p.
  __device__ int leaf_mod(u256& acc) {
    const uint32_t p = mod.p;
    const int m = __popcll(R);
    if (m == 1) {
      const int r = __ffsll((long long)R) - 1, c = __ffsll((long long)C) - 1;
      if (lane == 0) acc.w[0] = (acc.w[0] + coef.w[0] % p * (uint64_t)(uint32_t)T[r * S + c]) % p;
      return 0;
    }
    if (m > PERM_MAX_LEAF) return PERM_EINVAL;
    if (m > LN) return DFS_RETRY;
    const int nmax = LN <= 16 ? 16 : nmax_for(m);
    uint32_t* d = reinterpret_cast<uint32_t*>(delta);
    uint32_t* r0 = reinterpret_cast<uint32_t*>(rho0);
    const int cols = m - 1;
    for (int k = lane; k < cols * nmax; k += 32) d[k] = 0;
    __syncwarp();
    if (lane < m) {
      const int myrow = nth_bit(R, lane);
      uint64_t cm = rowbits[myrow] & C;
      uint32_t rs = 0, last = 0;
      while (cm) {
        const int c = __ffsll((long long)cm) - 1;
        cm &= cm - 1;
        const int jj = __popcll(C & (bit64(c) - 1));  // leaf column of c
        const uint32_t a = (uint32_t)T[myrow * S + c];
        rs = mod_add(rs, a, p);
        if (jj < cols) d[jj * nmax + lane] = to_mont(mod_add(a, a, p), mod); else last = a;
      }
      r0[lane] = to_mont(mod_sub(mod_add(last, last, p), rs, p), mod);
    }
    for (int i = m + lane; i < nmax; i += 32) r0[i] = to_mont(1u, mod);
    __syncwarp();
    const int e = m - 1;
    const int lanes = e <= 5 ? 1 << (e - 1) : 32;
    const uint64_t cnt = e <= 5 ? 2 : 1ull << (e - 5);
    const uint64_t gb = (uint64_t)lane * cnt, mc = lane < lanes ? cnt : 0;
    uint32_t sg;
    if constexpr (LN <= 16) {
      sg = ryser_lane_mod<16>(d, r0, m, gb, mc, mod);
    } else {
      if (nmax == 8) sg = ryser_lane_mod<8>(d, r0, m, gb, mc, mod);
      else if (nmax == 16) sg = ryser_lane_mod<16>(d, r0, m, gb, mc, mod);
      else if (nmax == 24) sg = ryser_lane_mod<24>(d, r0, m, gb, mc, mod);
      else sg = ryser_lane_mod<32>(d, r0, m, gb, mc, mod);
    }
    sg = warp_sum_mod(sg, p);
    if (lane == 0) {
      const uint32_t per = nw_per_mod(from_mont(sg, mod), m, p);
      acc.w[0] = (acc.w[0] + (uint64_t)per * (coef.w[0] % p)) % p;
    }
    __syncwarp();
    return 0;
  }

  __device__ int leaf_ring(u256& acc) {
    const int m = __popcll(R);
    if (m == 1) {
      const int r = __ffsll((long long)R) - 1, c = __ffsll((long long)C) - 1;
      if (lane == 0) acc = u256_add(acc, u256_mul_s64(coef, (int64_t)T[r * S + c]));
      return 0;
    }
    if (m > PERM_MAX_LEAF) return PERM_EINVAL;
    if (m > LN) return DFS_RETRY;
    const int nmax = LN <= 16 ? 16 : nmax_for(m);
    // row ranges, and per leaf column the leaf rows holding a nonzero
    int64_t rmax = 0;
    bool ok = true;
    int myrow = lane < m ? nth_bit(R, lane) : 0;
    int mycol = lane < m ? nth_bit(C, lane) : 0;
    // the leaf's nonzeros are the set bits of the row and column masks
    // (a lane walks its row's few nonzeros, not every active column)
    const uint64_t rownz = lane < m ? (rowbits[myrow] & C) : 0;
    if (lane < m) {
      int64_t ra = 0;
      uint64_t cm = rownz;
      while (cm) {
        const int c = __ffsll((long long)cm) - 1;
        cm &= cm - 1;
        const int64_t a = (int64_t)T[myrow * S + c];
        if (a >= (1ll << 30) || a <= -(1ll << 30)) ok = false;
        ra += a < 0 ? -a : a;
      }
      if (ra >= (1ll << 31)) ok = false;
      rmax = ra;
      // leaf rows (ranks among the active rows) holding a nonzero in my column
      uint32_t msk = 0;
      uint64_t rm = colbits[mycol] & R;
      while (rm) {
        const int r = __ffsll((long long)rm) - 1;
        rm &= rm - 1;
        msk |= 1u << __popcll(R & (bit64(r) - 1));
      }
      cmask[lane] = msk;
    }
    ok = __all_sync(0xffffffffu, ok);
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) {
      const int64_t o = __shfl_xor_sync(0xffffffffu, rmax, d);
      rmax = o > rmax ? o : rmax;
    }
    __syncwarp();
    if (!ok) return PERM_EOVERFLOW;
    const int bc = bit_class(rmax);
    int path = bc == 7 ? 0 : (bc == 15 ? 1 : 2);
    int ca = 0, cb = 1, clast = m - 1;
    if (bc == 7 && m >= 3) {
      // the leaf-column pair touching the fewest leaf rows, lowest pair on ties
      unsigned key = 0xffffffffu;
      if (lane < m) {
        const uint32_t ma = cmask[lane];
        for (int b = lane + 1; b < m; ++b) {
          const unsigned kk = ((unsigned)__popc(ma | cmask[b]) << 16) | ((unsigned)lane << 8) | (unsigned)b;
          key = kk < key ? kk : key;
        }
      }
#pragma unroll
      for (int d = 16; d > 0; d >>= 1) key = min(key, __shfl_xor_sync(0xffffffffu, key, d));
      const int k = (int)(key >> 16);
      const int ka = (int)((key >> 8) & 0xff), kb = (int)(key & 0xff);
      // 16 N slots: one of the two columns must fit the first 8
      if (k <= 8 || (k <= 16 && nmax >= 16 && min(__popc(cmask[ka]), __popc(cmask[kb])) <= 8)) {
        path = k <= 8 ? 3 : 4;
        // Gray column 0: the one touching at most 8 rows
        const bool a_first = __popc(cmask[ka]) <= 8;
        ca = a_first ? ka : kb;
        cb = a_first ? kb : ka;
        while (clast == ca || clast == cb) --clast;
      }
    }
    // fill delta / rho0 (leaf columns jj, leaf rows ii)
    const int cols = m - 1;
    for (int k = lane; k < cols * nmax; k += 32) delta[k] = 0;
    __syncwarp();
    int slot = lane;
    if (path >= 3) {
      // the rows of Gray column 0 first, then the other rows of column 1, then the rest
      const uint32_t am = cmask[ca];
      const uint32_t tm = am | cmask[cb];
      const uint32_t below = (1u << lane) - 1u;
      const uint32_t valid = m >= 32 ? 0xffffffffu : ((1u << m) - 1u);
      slot = ((am >> lane) & 1) ? __popc(am & below)
             : ((tm >> lane) & 1) ? __popc(am) + __popc(tm & ~am & below)
                                  : __popc(tm) + __popc(~tm & valid & below);
    }
    if (lane < m) {
      int64_t rs = 0, last = 0;
      uint64_t cm = rownz;
      while (cm) {
        const int c = __ffsll((long long)cm) - 1;
        cm &= cm - 1;
        const int jj = __popcll(C & (bit64(c) - 1));  // leaf column of c
        const int64_t a = (int64_t)T[myrow * S + c];
        rs += a;
        int gj;
        if (path >= 3)
          gj = jj == ca ? 0 : (jj == cb ? 1 : (jj == clast ? -1 : 2 + jj - (ca < jj) - (cb < jj) - (clast < jj)));
        else
          gj = jj < cols ? jj : -1;
        if (gj >= 0) delta[gj * nmax + slot] = (int32_t)(2 * a); else last = a;
      }
      rho0[slot] = (int32_t)(2 * last - rs);
    }
    for (int i = m + lane; i < nmax; i += 32) rho0[i] = 1;
    __syncwarp();
    const int e = m - 1;
    int lanes;
    uint64_t cnt;
    if (path >= 3) {
      if (e <= 6) {
        lanes = 1 << (e - 2);
        cnt = 4;
      } else {
        lanes = 32;
        cnt = 1ull << (e - 5);
      }
    } else if (e <= 5) {
      lanes = 1 << (e - 1);
      cnt = 2;
    } else {
      lanes = 32;
      cnt = 1ull << (e - 5);
    }
    uint64_t words[4] = {0, 0, 0, 0};
    const uint64_t gb = (uint64_t)lane * cnt;
    leaf_dispatch<LN, W>(nmax, path, delta, rho0, m, gb, lane < lanes ? cnt : 0, words);
    if (lane == 0) {
      u256 s;
      for (int k = 0; k < 4; ++k) s.w[k] = words[k];
      s = u256_shr(s, m - 1);
      if ((m - 1) & 1) s = u256_neg(s);
      acc = u256_add(acc, u256_mul(s, coef));
    }
    __syncwarp();
    return 0;
  }
};

// Evaluate one job on the warp's tile (every lane takes part): its
// permanent times its coefficient into out.acc[job], its timing, node and
// leaf counts and status, and the sum into its matrix's accumulator.
template <int TILE, typename E, int LN, int W>
__device__ __forceinline__ void dfs_job(Dfs<TILE, E, LN, W>& D, const DfsArgs& A, uint32_t job, int cut) {
  constexpr int S = DfsCfg<TILE, E>::STRIDE;
  const int lane = D.lane;
  const uint64_t t0 = globaltimer_ns();
  const int m = A.jobs.m[job];
  const int nnz = A.jobs.nnz[job];
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
    bool fits = true;
    for (int r = lane; r < m; r += 32) {
      uint64_t rb = 0;
      for (int q = v.rowptr[r]; q < v.rowptr[r + 1]; ++q) {
        const int c = v.col[q];
        const int64_t x = v.val[q];
        if ((int64_t)(E)x != x) fits = false;
        D.T[r * S + c] = (E)x;
        rb |= bit64(c);
        atomicOr((unsigned long long*)&D.colbits[c], (unsigned long long)bit64(r));
      }
      D.rowbits[r] = rb;
    }
    fits = __all_sync(0xffffffffu, fits);
    __syncwarp();
    if (!fits) status = DFS_RETRY;
    D.R = D.C = (m == 64) ? ~0ull : (bit64(m) - 1);
    for (int t = 0; t < 4; ++t) D.coef.w[t] = A.jobs.coef[4ll * job + t];
    int depth = 0;
    bool done = status != 0;
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
        if (mact <= cut || (s >= 5 && !A.three)) {
          ++leaves;
          status = D.leaf(acc);
          if (status != 0) break;
        } else if (depth >= A.max_depth - 1) {
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
              pv[t] = (int64_t)(f.is_col ? D.T[c * S + f.idx] : D.T[f.idx * S + c]);
            } else {
              f.pos[t] = 0;
            }
          }
          D.store_frame(depth, f, pv, D.coef);
          __syncwarp();
          if (!D.apply(depth, f, pv, 0)) {
            status = sizeof(E) == 4 ? DFS_RETRY : PERM_EOVERFLOW;
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
        if (f.child + 1 < Dfs<TILE, E, LN, W>::nchildren(f.k)) {
          f.child += 1;
          D.set_child(depth - 1, f.child);
          __syncwarp();
          if (!D.apply(depth - 1, f, pv, f.child)) {
            status = sizeof(E) == 4 ? DFS_RETRY : PERM_EOVERFLOW;
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
    if (status == DFS_RETRY && A.retry_flag) atomicOr(A.retry_flag, 1ull);
  }
  __syncwarp();
}

}  // namespace
