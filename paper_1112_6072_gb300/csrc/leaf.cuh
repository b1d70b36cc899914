// Leaf jobs (order <= the leaf order) evaluated by Ryser / Nijenhuis-Wilf
// (Section 1): the kernel variants' path codes, the split of a job's Gray
// codes into tasks, the loads of a job into a warp's shared-memory columns,
// and one task's share of the Gray sum.  Shared by the per-variant leaf
// kernels (leaf.cu) and the single-launch evaluator (persist.cu).
#pragma once
#include <cstdint>

#include "jobs.cuh"
#include "ryser.cuh"
#include "ryser4.cuh"
#include "ryser_mod.cuh"

namespace {

// path codes
constexpr int P_G7 = 0, P_G15 = 1, P_G31 = 2, P_F8 = 3, P_F16 = 4, P_MOD = 5, P_F4 = 6, P_BAD = 7;

__host__ __device__ __forceinline__ void leaf_split(int m, int chunk_log2, int& lanes, int& clog,
                                                    uint64_t& tasks) {
  // m >= 2: 2^(m-1) codes, lanes walk aligned blocks of 2^clog codes
  // (clog >= 2 once m >= 3, as the blocked walk needs).
  const int e = m - 1;
  if (e == 1) {
    clog = 1;
    lanes = 1;
    tasks = 1;
    return;
  }
  if (e <= 6) {
    clog = 2;
    lanes = 1 << (e - 2);
    tasks = 1;
    return;
  }
  const int cl = chunk_log2 < 2 ? 2 : chunk_log2;
  lanes = 32;
  clog = e - 5 < cl ? e - 5 : cl;
  tasks = 1ull << (e - 5 - clog);
}

// Load a leaf for the plain walk: rows in order, Gray column j = column j,
// the last column carries the Nijenhuis-Wilf offset.
__device__ void load_plain(const uint64_t* __restrict__ arena, int64_t off, int m, int nnz, int nmax,
                           int32_t* delta, int32_t* rho0, int lane) {
  CsrView v = csr_view(arena, off, m, nnz);
  const int cols = m - 1;
  for (int k = lane; k < cols * nmax; k += 32) delta[k] = 0;
  __syncwarp();
  for (int i = lane; i < nmax; i += 32) {
    if (i >= m) {
      rho0[i] = 1;
      continue;
    }
    int64_t rs = 0, last = 0;
    for (int p = v.rowptr[i]; p < v.rowptr[i + 1]; ++p) {
      const int c = v.col[p];
      const int64_t a = v.val[p];
      rs += a;
      if (c < cols) delta[c * nmax + i] = (int32_t)(2 * a); else last = a;
    }
    rho0[i] = (int32_t)(2 * last - rs);
  }
  __syncwarp();
}

// Load a leaf for the blocked walk: the two sparsest columns become Gray
// columns 0 and 1 (column 0 the one touching at most 8 rows), the rows of
// column 0 come first, then the other rows of column 1, then the rest; the
// highest remaining column carries the offset.
__device__ void load_blocked(const uint64_t* __restrict__ arena, int64_t off, int m, int nnz, int nmax,
                             int32_t* delta, int32_t* rho0, int32_t* colcnt, int lane) {
  CsrView v = csr_view(arena, off, m, nnz);
  const int cols = m - 1;
  for (int k = lane; k < cols * nmax; k += 32) delta[k] = 0;
  colcnt[lane] = 0;
  __syncwarp();
  if (lane < m)
    for (int p = v.rowptr[lane]; p < v.rowptr[lane + 1]; ++p)
      atomicOr(reinterpret_cast<unsigned*>(&colcnt[v.col[p]]), 1u << lane);
  __syncwarp();
  // the column pair: one for the 4 + 4 split (union within 8 rows, one
  // column within 4) if there is one, else the pair touching the fewest
  // rows; fewest rows, then lowest (a, b), on ties (leaf_class's rule)
  unsigned key = 0xffffffffu;
  if (lane < m) {
    const unsigned ma = (unsigned)colcnt[lane];
    const int na = __popc(ma);
    for (int b = lane + 1; b < m; ++b) {
      const unsigned u = (unsigned)__popc(ma | (unsigned)colcnt[b]);
      const bool split = u <= 8 && min(na, __popc((unsigned)colcnt[b])) <= 4;
      const unsigned kk = ((split ? 0u : 1u) << 24) | (u << 16) | ((unsigned)lane << 8) | (unsigned)b;
      key = kk < key ? kk : key;
    }
  }
#pragma unroll
  for (int d = 16; d > 0; d >>= 1) key = min(key, __shfl_xor_sync(0xffffffffu, key, d));
  const int ca = (int)((key >> 8) & 0xff);
  const int cb = (int)(key & 0xff);
  int clast = m - 1;
  while (clast == ca || clast == cb) --clast;
  // Gray column 0: the column of the pair touching fewer rows (at most 8 for
  // the 16-slot form, at most 4 for the 4 + 4 split)
  const bool a_first = __popc((unsigned)colcnt[ca]) <= __popc((unsigned)colcnt[cb]);
  const int g0 = a_first ? ca : cb, g1 = a_first ? cb : ca;  // Gray columns 0 and 1
  const uint32_t am = (uint32_t)colcnt[g0];
  const uint32_t tm = am | (uint32_t)colcnt[g1];
  const uint32_t below = (1u << lane) - 1u;
  const uint32_t valid = m >= 32 ? 0xffffffffu : ((1u << m) - 1u);
  const int slot = ((am >> lane) & 1) ? __popc(am & below)
                   : ((tm >> lane) & 1) ? __popc(am) + __popc(tm & ~am & below)
                                        : __popc(tm) + __popc(~tm & valid & below);
  if (lane < m) {
    int64_t rs = 0, last = 0;
    for (int p = v.rowptr[lane]; p < v.rowptr[lane + 1]; ++p) {
      const int c = v.col[p];
      const int64_t a = v.val[p];
      rs += a;
      // Gray index of physical column c: g0 -> 0, g1 -> 1, clast -> offset, others in order from 2
      const int gj = c == g0 ? 0 : (c == g1 ? 1 : (c == clast ? -1 : 2 + c - (ca < c) - (cb < c) - (clast < c)));
      if (gj >= 0) delta[gj * nmax + slot] = (int32_t)(2 * a); else last = a;
    }
    rho0[slot] = (int32_t)(2 * last - rs);
  }
  for (int i = m + lane; i < nmax; i += 32) rho0[i] = 1;
  __syncwarp();
}

// Load a leaf for the modular walk: as load_plain, with the entries (residues
// in [0, p)) doubled and summed modulo p and stored in Montgomery form.
__device__ void load_mod(const uint64_t* __restrict__ arena, int64_t off, int m, int nnz, int nmax, uint32_t* delta,
                         uint32_t* rho0, int lane, const ModP& M) {
  CsrView v = csr_view(arena, off, m, nnz);
  const int cols = m - 1;
  for (int k = lane; k < cols * nmax; k += 32) delta[k] = 0;
  __syncwarp();
  for (int i = lane; i < nmax; i += 32) {
    if (i >= m) {
      rho0[i] = to_mont(1u, M);
      continue;
    }
    uint32_t rs = 0, last = 0;
    for (int p = v.rowptr[i]; p < v.rowptr[i + 1]; ++p) {
      const int c = v.col[p];
      const uint32_t a = (uint32_t)v.val[p];
      rs = mod_add(rs, a, M.p);
      if (c < cols) delta[c * nmax + i] = to_mont(mod_add(a, a, M.p), M); else last = a;
    }
    rho0[i] = to_mont(mod_sub(mod_add(last, last, M.p), rs, M.p), M);
  }
  __syncwarp();
}

// Gray-code tasks of a leaf job of order m (1 below order 2).
__host__ __device__ __forceinline__ uint64_t leaf_tasks_dev(int m, int chunk_log2) {
  if (m < 2) return 1;
  int lanes, clog;
  uint64_t tasks;
  leaf_split(m, chunk_log2, lanes, clog, tasks);
  return tasks;
}

// Load job (order m >= 2) into the warp's columns for variant PATH.
template <int NMAX, int PATH>
__device__ __forceinline__ void leaf_load(const uint64_t* __restrict__ arena, int64_t off, int m, int nnz,
                                          int32_t* delta, int32_t* rho0, int32_t* colcnt, int lane, const ModP& mod) {
  if constexpr (PATH == P_MOD)
    load_mod(arena, off, m, nnz, NMAX, reinterpret_cast<uint32_t*>(delta), reinterpret_cast<uint32_t*>(rho0), lane,
             mod);
  else if constexpr (PATH == P_F8 || PATH == P_F16 || PATH == P_F4)
    load_blocked(arena, off, m, nnz, NMAX, delta, rho0, colcnt, lane);
  else
    load_plain(arena, off, m, nnz, NMAX, delta, rho0, lane);
}

// Task lt of a loaded leaf job of order m: its Gray codes summed over the
// warp into lane 0's words (the raw Sigma share; a residue in word 0 on the
// residue path).  An order-1 job gives its entry.  Every lane takes part.
template <int NMAX, int W, int PATH>
__device__ __forceinline__ void leaf_task(const uint64_t* __restrict__ arena, int64_t off, int m, int nnz,
                                          uint64_t lt, int chunk_log2, const int32_t* delta, const int32_t* rho0,
                                          int lane, const ModP& mod, uint64_t* words) {
  words[0] = words[1] = words[2] = words[3] = 0;
  if (m == 1) {
    if (lane == 0) {
      CsrView v = csr_view(arena, off, 1, nnz);
      const int64_t a = nnz ? v.val[0] : 0;
      const uint64_t sg = a < 0 ? ~0ull : 0ull;
      words[0] = (uint64_t)a;
      words[1] = words[2] = words[3] = sg;
    }
    return;
  }
  if (m < 2) return;
  int lanes, clog;
  uint64_t tasks;
  leaf_split(m, chunk_log2, lanes, clog, tasks);
  const uint64_t cnt = 1ull << clog;
  const uint64_t gb = (lt * 32 + lane) * cnt;
  const uint64_t mycnt = lane < lanes ? cnt : 0;  // idle lanes of small jobs contribute zero
  if constexpr (PATH == P_MOD) {
    const uint32_t sm_ = ryser_lane_mod<NMAX>(reinterpret_cast<const uint32_t*>(delta),
                                              reinterpret_cast<const uint32_t*>(rho0), m, gb, mycnt, mod);
    words[0] = from_mont(warp_sum_mod(sm_, mod.p), mod);  // Sigma mod p, a plain residue
  } else if constexpr (PATH == P_F4) {
    if (m >= 3) {
      run_lane4<NMAX, 8, W, true>(delta, rho0, m, gb, mycnt, words);
      return;
    }
    typename WideT<W>::type sw = ryser_lane<NMAX, W, 7>(delta, rho0, m, gb, mycnt);
    to_words(warp_sum(sw), words);
  } else if constexpr (PATH == P_F8) {
    if (m >= 3) {
      run_lane4<NMAX, 8, W>(delta, rho0, m, gb, mycnt, words);
      return;
    }
    typename WideT<W>::type sw = ryser_lane<NMAX, W, 7>(delta, rho0, m, gb, mycnt);
    to_words(warp_sum(sw), words);
  } else if constexpr (PATH == P_F16) {
    if constexpr (NMAX >= 16) {
      if (m >= 3) {
        run_lane4<NMAX, 16, W>(delta, rho0, m, gb, mycnt, words);
        return;
      }
    }
    typename WideT<W>::type sw = ryser_lane<NMAX, W, 7>(delta, rho0, m, gb, mycnt);
    to_words(warp_sum(sw), words);
  } else {
    constexpr int BC = PATH == P_G15 ? 15 : (PATH == P_G31 ? 31 : 7);
    typename WideT<W>::type sw = ryser_lane<NMAX, W, BC>(delta, rho0, m, gb, mycnt);
    to_words(warp_sum(sw), words);
  }
}

// Sigma (the job's summed task words) -> coef * per(job), mod 2^256 or
// modulo modp on the residue path.
__device__ __forceinline__ u256 leaf_finish(const uint64_t* sigma, int m, const uint64_t* coef, uint32_t modp) {
  u256 v = u256_zero();
  if (modp) {
    const uint32_t per = nw_per_mod((uint32_t)(sigma[0] % modp), m, modp);
    v.w[0] = (uint64_t)per * (coef[0] % modp) % modp;
    return v;
  }
  u256 s;
  for (int k = 0; k < 4; ++k) s.w[k] = sigma[k];
  if (m >= 2) {
    s = u256_shr(s, m - 1);
    if ((m - 1) & 1) s = u256_neg(s);
  }
  u256 c;
  for (int k = 0; k < 4; ++k) c.w[k] = coef[k];
  return u256_mul(s, c);
}

}  // namespace
