// K1: one level of Algorithm PH, Step 2 (Section 2.2) -- every parent job is
// divided by Eq. 2 into at most two children, written in compact CSR.
//
// One warp per parent.  The parent is scattered into a dense tile in shared
// memory (order <= TILE); lanes own rows and columns.  The pivot is the line
// with the fewest nonzeros (Algorithm H_per, Step 1), lowest row first, else
// lowest column.  With the pivot line's nonzeros at positions j1 < j2 < j3 <
// j4 and values a, b, c, d, the children are, in order:
//   k = 1: a * minor(j1)
//   k = 2: merge(j1, j2)
//   k = 3: merge(j1, j2), c * minor(j3)
//   k = 4: merge(j1, j2), merge(j3, j4)
// where merge(p, q) of a row pivot i deletes row i, replaces column p by
// T[i][p] * col_q + T[i][q] * col_p (Eq. 2's a*y2 + b*y1) and deletes column
// q; a column pivot does the same with rows.  A scalar factor multiplies the
// child's coefficient.  Children holding a zero line are not emitted.  A
// parent of order <= max(L, 2), with s >= 5, or with no levels left is
// carried unchanged to slot 2p.
#include <cuda_runtime.h>

#include <cstdint>

#include "internal.h"
#include "wide.cuh"

namespace {

template <int TILE>
struct ExpandCfg {
  static constexpr int STRIDE = TILE + 1;  // int64 words per tile row (odd: fewer bank conflicts)
  static constexpr int MW = TILE > 64 ? 2 : 1;  // 64-bit mask words per line
  static constexpr int WARPS = TILE >= 128 ? 1 : (TILE >= 64 ? 3 : 8);
  static constexpr size_t TILE_BYTES = sizeof(int64_t) * TILE * STRIDE;
  static constexpr size_t SMEM = WARPS * TILE_BYTES;
};

__device__ __forceinline__ unsigned long long warp_min_u64(unsigned long long v) {
#pragma unroll
  for (int d = 16; d > 0; d >>= 1) {
    unsigned long long o = __shfl_xor_sync(0xffffffffu, v, d);
    v = o < v ? o : v;
  }
  return v;
}

__device__ __forceinline__ int warp_excl_scan(int v, int lane, int& total) {
  int x = v;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    int y = __shfl_up_sync(0xffffffffu, x, d);
    if (lane >= d) x += y;
  }
  total = __shfl_sync(0xffffffffu, x, 31);
  return x - v;
}

// checked a*x + b*y in int64
__device__ __forceinline__ bool mad2_checked(int64_t a, int64_t x, int64_t b, int64_t y, int64_t& out) {
  __int128 r = (__int128)a * x + (__int128)b * y;
  out = (int64_t)r;
  return r == (__int128)out;
}

struct ChildSpec {
  int del_row, del_col;
  int merge;      // 0 none, 1 column p merged (row pivot), 2 row p merged (column pivot)
  int p, q;       // merged line and its partner (deleted)
  int64_t a, b;   // merged line = a * line_q + b * line_p
  int64_t fac;    // scalar factor (minor)
};

template <int TILE>
__device__ void write_child(const int64_t* T, int m, const ChildSpec& cs, int lane, uint64_t* blk,
                            int& nnz_out, bool& keep, int32_t* err) {
  constexpr int S = ExpandCfg<TILE>::STRIDE;
  constexpr int MW = ExpandCfg<TILE>::MW;
  constexpr int RPL = (TILE + 31) / 32;  // child rows per lane
  const int mc = m - 1;
  int cnt[RPL];
  uint64_t colmask[MW];
#pragma unroll
  for (int w = 0; w < MW; ++w) colmask[w] = 0;
  bool ovf = false;
  // pass 1: row lengths and the union of nonzero columns
#pragma unroll
  for (int k = 0; k < RPL; ++k) {
    const int rc = lane + 32 * k;  // child row
    cnt[k] = 0;
    if (rc < mc) {
      const int r = rc + (rc >= cs.del_row);
      int cc = 0;
      for (int c = 0; c < m; ++c) {
        if (c == cs.del_col) continue;
        int64_t v = T[r * S + c];
        if (cs.merge == 1 && c == cs.p) {
          if (!mad2_checked(cs.a, T[r * S + cs.q], cs.b, v, v)) ovf = true;
        } else if (cs.merge == 2 && r == cs.p) {
          if (!mad2_checked(cs.a, T[cs.q * S + c], cs.b, v, v)) ovf = true;
        }
        if (v != 0) {
          cnt[k]++;
          colmask[cc >> 6] |= 1ull << (cc & 63);
        }
        ++cc;
      }
    }
  }
#pragma unroll
  for (int w = 0; w < MW; ++w) {
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) colmask[w] |= __shfl_xor_sync(0xffffffffu, colmask[w], d);
  }
  bool zero_row = false;
#pragma unroll
  for (int k = 0; k < RPL; ++k)
    if (lane + 32 * k < mc && cnt[k] == 0) zero_row = true;
  zero_row = __any_sync(0xffffffffu, zero_row);
  ovf = __any_sync(0xffffffffu, ovf);
  int ncols = 0;
#pragma unroll
  for (int w = 0; w < MW; ++w) ncols += __popcll(colmask[w]);
  if (ovf && lane == 0) atomicCAS(err, 0, PERM_EOVERFLOW);
  keep = !ovf && !zero_row && ncols == mc;
  if (!keep) {
    nnz_out = 0;
    return;
  }
  // row offsets: lanes hold rows lane, lane+32, ...; scan in row order
  int base = 0;
  int offs[RPL];
#pragma unroll
  for (int k = 0; k < RPL; ++k) {
    int tot;
    offs[k] = base + warp_excl_scan(cnt[k], lane, tot);
    base += tot;
  }
  nnz_out = base;
  uint16_t* rowptr = reinterpret_cast<uint16_t*>(blk);
  uint8_t* col = reinterpret_cast<uint8_t*>(blk + blk_rp_words(mc));
  int64_t* val = reinterpret_cast<int64_t*>(blk + blk_rp_words(mc) + blk_col_words(base));
  if (lane == 0) rowptr[mc] = (uint16_t)base;
  // pass 2: write rows
#pragma unroll
  for (int k = 0; k < RPL; ++k) {
    const int rc = lane + 32 * k;
    if (rc < mc) {
      const int r = rc + (rc >= cs.del_row);
      rowptr[rc] = (uint16_t)offs[k];
      int o = offs[k];
      int cc = 0;
      for (int c = 0; c < m; ++c) {
        if (c == cs.del_col) continue;
        int64_t v = T[r * S + c];
        if (cs.merge == 1 && c == cs.p)
          mad2_checked(cs.a, T[r * S + cs.q], cs.b, v, v);
        else if (cs.merge == 2 && r == cs.p)
          mad2_checked(cs.a, T[cs.q * S + c], cs.b, v, v);
        if (v != 0) {
          col[o] = (uint8_t)cc;
          val[o] = v;
          ++o;
        }
        ++cc;
      }
    }
  }
}

__device__ __forceinline__ void copy_words(uint64_t* dst, const uint64_t* src, int64_t words, int lane) {
  // blocks start on 16 bytes and hold an even number of words
  const uint4* s4 = reinterpret_cast<const uint4*>(src);
  uint4* d4 = reinterpret_cast<uint4*>(dst);
  for (int64_t k = lane; k < words / 2; k += 32) d4[k] = s4[k];
}

template <int TILE>
__global__ void __launch_bounds__(ExpandCfg<TILE>::WARPS * 32) k_expand_level(ExpandLevelArgs A) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  constexpr int S = ExpandCfg<TILE>::STRIDE;
  constexpr int MW = ExpandCfg<TILE>::MW;
  constexpr int RPL = (TILE + 31) / 32;
  const int lane = threadIdx.x & 31;
  const int wib = threadIdx.x >> 5;
  int64_t* T = reinterpret_cast<int64_t*>(smem_raw) + (size_t)wib * TILE * S;
  const int64_t nwarps = (int64_t)gridDim.x * ExpandCfg<TILE>::WARPS;
  for (int64_t p = (int64_t)blockIdx.x * ExpandCfg<TILE>::WARPS + wib; p < A.np; p += nwarps) {
    __syncwarp();  // the previous parent's tile reads are done
    const int m = A.parent.m[p];
    const int nnz = A.parent.nnz[p];
    const int64_t off = A.parent.off[p];
    const int dl = A.parent.depth_left[p];
    const int64_t pw = blk_words(m, nnz);
    const int64_t cbase = A.child_off_base[p];
    CsrView v = csr_view(A.arena_in, off, m, nnz);
    // dense tile and line counts
    for (int k = lane; k < m * S; k += 32) T[k] = 0;
    __syncwarp();
    int rcount[RPL];
#pragma unroll
    for (int k = 0; k < RPL; ++k) {
      const int r = lane + 32 * k;
      rcount[k] = 0;
      if (r < m) {
        const int b = v.rowptr[r], e = v.rowptr[r + 1];
        rcount[k] = e - b;
        for (int q = b; q < e; ++q) T[r * S + v.col[q]] = v.val[q];
      }
    }
    __syncwarp();
    unsigned long long key = ~0ull;
#pragma unroll
    for (int k = 0; k < RPL; ++k) {
      const int r = lane + 32 * k;
      if (r < m) key = min(key, ((unsigned long long)rcount[k] << 17) | (unsigned long long)r);
    }
#pragma unroll
    for (int k = 0; k < RPL; ++k) {
      const int c = lane + 32 * k;
      if (c < m) {
        int cnt = 0;
        for (int r = 0; r < m; ++r) cnt += T[r * S + c] != 0;
        key = min(key, ((unsigned long long)cnt << 17) | (1ull << 16) | (unsigned long long)c);
      }
    }
    key = warp_min_u64(key);
    const int s = (int)(key >> 17);
    const bool is_col = (key >> 16) & 1;
    const int idx = (int)(key & 0xffff);
    const int cut = A.leaf_size > 2 ? A.leaf_size : 2;
    uint64_t* out0 = A.arena_out + cbase;
    if (s == 0) {  // zero line: nothing to emit
      if (lane == 0) A.valid[2 * p] = A.valid[2 * p + 1] = 0;
      continue;
    }
    if (dl <= 0 || m <= cut || s >= 5) {
      copy_words(out0, A.arena_in + off, pw, lane);
      if (lane == 0) {
        const int64_t c0 = 2 * p;
        A.child.m[c0] = m;
        A.child.nnz[c0] = nnz;
        A.child.off[c0] = cbase;
        A.child.mat[c0] = A.parent.mat[p];
        A.child.depth_left[c0] = 0;
        for (int w = 0; w < 4; ++w) A.child.coef[4 * c0 + w] = A.parent.coef[4 * p + w];
        A.valid[c0] = 1;
        A.valid[c0 + 1] = 0;
      }
      continue;
    }
    // pivot line's nonzero positions (ascending) and values
    int pos[4];
    int64_t pv[4];
    {
      int k = 0;
      for (int t = 0; t < m && k < 4; ++t) {
        int64_t x = is_col ? T[t * S + idx] : T[idx * S + t];
        if (x != 0) {
          pos[k] = t;
          pv[k] = x;
          ++k;
        }
      }
    }
    u256 pcoef;
    for (int w = 0; w < 4; ++w) pcoef.w[w] = A.parent.coef[4 * p + w];
    for (int c = 0; c < 2; ++c) {
      const int64_t slot = 2 * p + c;
      ChildSpec cs;
      cs.fac = 1;
      cs.merge = 0;
      cs.p = cs.q = 0;
      cs.a = cs.b = 0;
      bool exists = true;
      int kind = 0;  // 1 merge(pos[x], pos[x+1]), 2 minor(pos[x])
      int x = 0;
      if (c == 0) {
        kind = s == 1 ? 2 : 1;
        x = 0;
      } else if (s == 3) {
        kind = 2;
        x = 2;
      } else if (s == 4) {
        kind = 1;
        x = 2;
      } else {
        exists = false;
      }
      bool keep = false;
      int cnnz = 0;
      if (exists) {
        if (!is_col) {
          cs.del_row = idx;
          if (kind == 1) {
            cs.merge = 1;
            cs.p = pos[x];
            cs.q = pos[x + 1];
            cs.a = pv[x];
            cs.b = pv[x + 1];
            cs.del_col = cs.q;
          } else {
            cs.del_col = pos[x];
            cs.fac = pv[x];
          }
        } else {
          cs.del_col = idx;
          if (kind == 1) {
            cs.merge = 2;
            cs.p = pos[x];
            cs.q = pos[x + 1];
            cs.a = pv[x];
            cs.b = pv[x + 1];
            cs.del_row = cs.q;
          } else {
            cs.del_row = pos[x];
            cs.fac = pv[x];
          }
        }
        write_child<TILE>(T, m, cs, lane, out0 + c * pw, cnnz, keep, A.err);
      }
      if (lane == 0) {
        A.valid[slot] = keep ? 1 : 0;
        if (keep) {
          A.child.m[slot] = m - 1;
          A.child.nnz[slot] = cnnz;
          A.child.off[slot] = cbase + c * pw;
          A.child.mat[slot] = A.parent.mat[p];
          A.child.depth_left[slot] = dl - 1;
          u256 cc = cs.fac == 1 ? pcoef : u256_mul_s64(pcoef, cs.fac);
          for (int w = 0; w < 4; ++w) A.child.coef[4 * slot + w] = cc.w[w];
        }
      }
    }
    __syncwarp();
  }
}

__global__ void k_child_capacity(JobArrays parent, int64_t np, int64_t* words) {
  int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (p < np) words[p] = 2 * blk_words(parent.m[p], parent.nnz[p]);
}

// stat[0]: largest kept order, stat[1]: words of the kept blocks, stat[2]:
// kept jobs -- reduced per warp, one atomic per warp.
__global__ void k_compact(JobArrays src, const int32_t* valid, const int32_t* pos, int64_t nslots, JobArrays dst,
                          long long* stat) {
  const int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const bool keep = s < nslots && valid[s];
  unsigned m = 0, words = 0;
  if (keep) {
    const int64_t d = pos[s];
    m = (unsigned)src.m[s];
    words = (unsigned)blk_words(src.m[s], src.nnz[s]);
    dst.m[d] = src.m[s];
    dst.nnz[d] = src.nnz[s];
    dst.off[d] = src.off[s];
    dst.mat[d] = src.mat[s];
    dst.depth_left[d] = src.depth_left[s];
    for (int w = 0; w < 4; ++w) dst.coef[4 * d + w] = src.coef[4 * s + w];
  }
  const unsigned mx = __reduce_max_sync(0xffffffffu, m);
  const unsigned sw = __reduce_add_sync(0xffffffffu, words);
  const unsigned nk = __reduce_add_sync(0xffffffffu, keep ? 1u : 0u);
  if ((threadIdx.x & 31) == 0 && nk) {
    atomicMax(stat, (long long)mx);
    atomicAdd(reinterpret_cast<unsigned long long*>(stat + 1), (unsigned long long)sw);
    atomicAdd(reinterpret_cast<unsigned long long*>(stat + 2), (unsigned long long)nk);
  }
}

template <int TILE>
cudaError_t launch_tile(const ExpandLevelArgs& a, cudaStream_t s) {
  typedef ExpandCfg<TILE> C;
  static bool attr_set = false;
  if (!attr_set) {
    cudaError_t e = cudaFuncSetAttribute(k_expand_level<TILE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)C::SMEM);
    if (e != cudaSuccess) return e;
    attr_set = true;
  }
  int64_t blocks = (a.np + C::WARPS - 1) / C::WARPS;
  if (blocks > 152 * 64) blocks = 152 * 64;
  k_expand_level<TILE><<<(unsigned)blocks, C::WARPS * 32, C::SMEM, s>>>(a);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_expand_level(const ExpandLevelArgs& a, int max_order, cudaStream_t s) {
  if (a.np <= 0) return cudaSuccess;
  if (max_order <= 16) return launch_tile<16>(a, s);
  if (max_order <= 32) return launch_tile<32>(a, s);
  if (max_order <= 64) return launch_tile<64>(a, s);
  return launch_tile<128>(a, s);
}

cudaError_t launch_child_capacity(const JobArrays& parent, int64_t np, int64_t* words, cudaStream_t s) {
  if (np <= 0) return cudaSuccess;
  k_child_capacity<<<(unsigned)((np + 255) / 256), 256, 0, s>>>(parent, np, words);
  return cudaGetLastError();
}

cudaError_t launch_compact_jobs(const JobArrays& src, const int32_t* valid, const int32_t* pos, int64_t nslots,
                                JobArrays dst, long long* stat, cudaStream_t s) {
  if (nslots <= 0) return cudaSuccess;
  k_compact<<<(unsigned)((nslots + 255) / 256), 256, 0, s>>>(src, valid, pos, nslots, dst, stat);
  return cudaGetLastError();
}
