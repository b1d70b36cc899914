// K1: Algorithm PH, Step 2 (Section 2.2) -- every parent job is divided by
// Eq. 2 into at most two children, written in compact CSR.
//
// One warp per parent; lane l owns the parent rows l, l+32, ... and builds
// the child rows from the parent's sparse rows directly (work per child is
// proportional to its nonzeros, not to m^2).  The pivot is the line with the
// fewest nonzeros (Algorithm H_per, Step 1), lowest row first, else lowest
// column.  With the pivot line's nonzeros at positions j1 < j2 < j3 < j4 and
// values a, b, c, d, the children are, in order:
//   k = 1: a * minor(j1)
//   k = 2: merge(j1, j2)
//   k = 3: merge(j1, j2), c * minor(j3)
//   k = 4: merge(j1, j2), merge(j3, j4)
// where merge(p, q) of a row pivot i deletes row i, replaces column p by
// T[i][p] * col_q + T[i][q] * col_p (Eq. 2's a*y2 + b*y1) and deletes column
// q; a column pivot does the same with rows.  A scalar factor multiplies the
// child's coefficient.  Children holding a zero line are not emitted.  A
// parent of order <= max(L, 2), with s >= 5, or with no levels left is
// carried unchanged to slot Kp (K = 2 child slots per parent).  With the
// three-child option (K = 3), a parent with s >= 5 is split by Eq. 2 in
// full: merge(j1, j2), merge(j3, j4), and the parent with the pivot line's
// entries at j1..j4 cleared (same order).  With a split floor (automatic depth), a
// parent still to split whose order is below the floor waits: it is carried
// with its levels left, so the largest jobs of a batch are split first.
//
// Two drivers share the per-parent routine:
//  - k_expand_level: one level per launch; the host reserves two blocks of
//    the parent's size per parent (scan of capacities) and compacts after.
//  - k_expand_front: a cooperative launch that runs consecutive levels while
//    the frontier fits fixed buffers; blocks meet at a bounded grid barrier
//    twice per level, children's blocks are bump-allocated in the arena, and
//    each block compacts its own contiguous range of slots, so the natural
//    (breadth-first) order of the jobs is the same as with k_expand_level.
#include <cuda_runtime.h>

#include <cstdint>

#include "eq2.cuh"
#include "internal.h"
#include "wide.cuh"

namespace {

constexpr int kLevelWarps = 8;   // warps per block, k_expand_level
constexpr int kFrontWarps = 16;  // warps per block, k_expand_front
constexpr int kFrontThreads = kFrontWarps * 32;
constexpr int64_t kBarrierTimeoutNs = 10ll * 1000 * 1000 * 1000;
// words of a warp's shared-memory copy of its parent's CSR block (larger
// blocks are read from global memory)
constexpr int kStageWords = 1024;
constexpr size_t kLevelSmem = sizeof(uint64_t) * kStageWords * kLevelWarps;
constexpr size_t kFrontSmem = sizeof(uint64_t) * kStageWords * kFrontWarps;

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

// A group of LW lanes (the whole warp, or a half warp for parents of order
// <= 16) that works on one parent: every collective takes only its lanes.
template <int LW>
struct Grp {
  unsigned mask;  // lanes of the group
  int base;       // its first lane
  int sub;        // this lane's index in the group
  __device__ explicit Grp(int lane) {
    base = LW == 32 ? 0 : (lane & ~(LW - 1));
    sub = lane - base;
    mask = LW == 32 ? 0xffffffffu : (((1u << (LW & 31)) - 1u) << base);
  }
  __device__ void sync() const { __syncwarp(mask); }
  __device__ unsigned min(unsigned v) const { return __reduce_min_sync(mask, v); }
  __device__ unsigned ballot(bool q) const { return __ballot_sync(mask, q) >> base; }
  __device__ bool any(bool q) const { return __any_sync(mask, q); }
  template <typename T>
  __device__ T shfl(T v, int from) const { return __shfl_sync(mask, v, base + from); }
  __device__ uint64_t or_all(uint64_t v) const {
#pragma unroll
    for (int d = LW / 2; d > 0; d >>= 1) v |= __shfl_xor_sync(mask, v, d);
    return v;
  }
  __device__ int excl_scan(int v, int& total) const {
    int x = v;
#pragma unroll
    for (int d = 1; d < LW; d <<= 1) {
      const int y = __shfl_up_sync(mask, x, d, LW);
      if (sub >= d) x += y;
    }
    total = __shfl_sync(mask, x, base + LW - 1);
    return x - v;
  }
};

// Largest order and largest order still to split among a warp's kept
// children (lane 0), flushed to the level's maxima once per warp.
struct WarpMax {
  int order = 0;
  int open = 0;
};

// Where children's blocks go: reserved (cbase + c * parent words) or
// bump-allocated from a per-level counter.
struct ExpandCtx {
  JobArrays parent;
  const uint64_t* arena_in;
  JobArrays child;  // slots
  uint64_t* arena_out;
  const int64_t* child_off_base;  // reserved mode, else null
  unsigned long long* bump;       // bump mode: words used in arena_out
  int64_t cap_words;              // bump mode: arena_out capacity
  int32_t* valid;
  int32_t leaf_size;
  int32_t split_floor;            // parents of a lower order wait for a later level
  int32_t kslots;                 // child slots per parent: 2, or 3 with the three-child option
  uint32_t mod;                   // 0, or the residue path's modulus
  int32_t* err;
};

__device__ __forceinline__ void copy_words(uint64_t* dst, const uint64_t* src, int64_t words, int sub, int step) {
  // blocks start on 16 bytes and hold an even number of words
  const uint4* s4 = reinterpret_cast<const uint4*>(src);
  uint4* d4 = reinterpret_cast<uint4*>(dst);
  for (int64_t k = sub; k < words / 2; k += step) d4[k] = s4[k];
}

// Offset of a child's block: the group's first lane allocates, the group
// gets it back.  -1 if the arena is full (bump mode; the caller's capacity
// rule excludes it).
template <int LW>
__device__ __forceinline__ int64_t child_block(const ExpandCtx& X, int64_t p, int c, int64_t pw, int64_t words,
                                               const Grp<LW>& G) {
  if (X.child_off_base) return X.child_off_base[p] + c * pw;
  unsigned long long o = 0;
  if (G.sub == 0) o = atomicAdd(X.bump, (unsigned long long)words);
  o = G.shfl(o, 0);
  if ((int64_t)o + words > X.cap_words) {
    if (G.sub == 0) atomicCAS(X.err, 0, PERM_ENOMEM);
    return -1;
  }
  return (int64_t)o;
}

// Parent p unchanged into slot Kp with depth_left dl_out.
template <int LW>
__device__ void carry_parent(const ExpandCtx& X, int64_t p, const uint64_t* src, int64_t pw, int m, int nnz,
                             int dl_out, const Grp<LW>& G, WarpMax& wm) {
  const int64_t o = child_block(X, p, 0, pw, pw, G);
  if (o >= 0) copy_words(X.arena_out + o, src, pw, G.sub, LW);
  if (G.sub == 0) {
    const int64_t c0 = (int64_t)X.kslots * p;
    X.valid[c0] = o >= 0 ? 1 : 0;
    for (int c = 1; c < X.kslots; ++c) X.valid[c0 + c] = 0;
    if (o >= 0) {
      X.child.m[c0] = m;
      X.child.nnz[c0] = nnz;
      X.child.off[c0] = o;
      X.child.mat[c0] = X.parent.mat[p];
      X.child.depth_left[c0] = dl_out;
      for (int w = 0; w < 4; ++w) X.child.coef[4 * c0 + w] = X.parent.coef[4 * p + w];
      wm.order = max(wm.order, m);
      if (dl_out > 0) wm.open = max(wm.open, m);
    }
  }
}

// Divide parent p (one group of LW lanes; lane l of the group owns rows l,
// l + LW, ...).  ccnt: the group's shared-memory column counts (RPL * LW
// entries); stage: its stage_words-word copy of the parent block.
// only_child >= 0: build that child alone (one warp per child when the
// frontier is small; the child-0 warp also writes the carried and dropped
// cases); -1: all.
template <int RPL, int LW>
__device__ void expand_parent(const ExpandCtx& X, int64_t p, const Grp<LW>& G, int32_t* ccnt, uint64_t* stage,
                              int stage_words, WarpMax& wm, int only_child = -1) {
  const int lane = G.sub;
  const int m = X.parent.m[p];
  const int nnz = X.parent.nnz[p];
  const int64_t off = X.parent.off[p];
  const int dl = X.parent.depth_left[p];
  const int64_t pw = blk_words(m, nnz);
  const int cut = X.leaf_size > 2 ? X.leaf_size : 2;
  G.sync();  // the previous parent's reads of stage and ccnt are done
  if (dl > 0 && m > cut && m < X.split_floor) {
    if (only_child <= 0) carry_parent(X, p, X.arena_in + off, pw, m, nnz, dl, G, wm);
    return;
  }
  const uint64_t* src = X.arena_in + off;
  if (pw <= stage_words) {
    copy_words(stage, src, pw, lane, LW);
    src = stage;
  }
  // line counts: rows from rowptr, columns by shared-memory atomics
  for (int c = lane; c < m; c += LW) ccnt[c] = 0;
  G.sync();
  const CsrView v = csr_view(src, 0, m, nnz);
  // (count << 17) | (is_col << 16) | index: count <= 128, index < 128
  unsigned key = 0xffffffffu;
#pragma unroll
  for (int k = 0; k < RPL; ++k) {
    const int r = lane + LW * k;
    if (r < m) {
      const int b = v.rowptr[r], e = v.rowptr[r + 1];
      key = min(key, ((unsigned)(e - b) << 17) | (unsigned)r);
      for (int t = b; t < e; ++t) atomicAdd(&ccnt[v.col[t]], 1);
    }
  }
  G.sync();
#pragma unroll
  for (int k = 0; k < RPL; ++k) {
    const int c = lane + LW * k;
    if (c < m) key = min(key, ((unsigned)ccnt[c] << 17) | (1u << 16) | (unsigned)c);
  }
  G.sync();  // counts read before the next parent clears them
  key = G.min(key);
  const int s = (int)(key >> 17);
  const bool is_col = (key >> 16) & 1;
  const int idx = (int)(key & 0xffff);
  const bool three = X.kslots == 3;
  if (s == 0) {  // zero line: nothing to emit
    if (lane == 0 && only_child <= 0)
      for (int c = 0; c < X.kslots; ++c) X.valid[(int64_t)X.kslots * p + c] = 0;
    return;
  }
  if (dl <= 0 || m <= cut || (s >= 5 && !three)) {
    if (only_child <= 0) carry_parent(X, p, src, pw, m, nnz, 0, G, wm);
    return;
  }
  // pivot line's nonzero positions (ascending) and values
  int pos[4];
  int64_t pv[4];
  if (!is_col) {
    const int b = v.rowptr[idx];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      pos[k] = k < s ? v.col[b + k] : 0;
      pv[k] = k < s ? v.val[b + k] : 0;
    }
  } else {
    int n = 0;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      pos[k] = 0;
      pv[k] = 0;
    }
#pragma unroll
    for (int k = 0; k < RPL; ++k) {
      const int r = lane + LW * k;
      int64_t x = 0;
      if (r < m) {
        const int b = v.rowptr[r], e = v.rowptr[r + 1];
        for (int t = b; t < e; ++t)
          if (v.col[t] == idx) x = v.val[t];
      }
      unsigned bal = G.ballot(x != 0);
      while (bal) {
        const int l = __ffs(bal) - 1;
        bal &= bal - 1;
        const long long xv = G.shfl((long long)x, l);
#pragma unroll
        for (int u = 0; u < 4; ++u)
          if (u == n) {
            pos[u] = l + LW * k;
            pv[u] = xv;
          }
        ++n;
      }
    }
  }
  u256 pcoef;
  for (int w = 0; w < 4; ++w) pcoef.w[w] = X.parent.coef[4 * p + w];
  for (int c = 0; c < X.kslots; ++c) {
    if (only_child >= 0 && c != only_child) continue;
    const int64_t slot = (int64_t)X.kslots * p + c;
    int kind;  // 1 merge(pos[x], pos[x+1]), 2 minor(pos[x]), 3 pivot line's first four entries cleared
    int x = 0;
    if (c == 0) {
      kind = s == 1 ? 2 : 1;
    } else if (c == 1 && s == 3) {
      kind = 2;
      x = 2;
    } else if (c == 1 && s >= 4) {
      kind = 1;
      x = 2;
    } else if (c == 2 && s >= 5) {
      kind = 3;
    } else {
      if (lane == 0) X.valid[slot] = 0;
      continue;
    }
    const int mc = kind == 3 ? m : m - 1;
    ChildSpec cs;
    cs.mod = X.mod;
    cs.fac = 1;
    cs.merge = 0;
    cs.p = cs.q = 0;
    cs.a = cs.b = 0;
    cs.zcol = is_col ? 1 : 0;
    cs.zidx = idx;
#pragma unroll
    for (int u = 0; u < 4; ++u) cs.zp[u] = pos[u];
    const int xp = x == 0 ? pos[0] : pos[2], xq = x == 0 ? pos[1] : pos[3];
    const int64_t va = x == 0 ? pv[0] : pv[2], vb = x == 0 ? pv[1] : pv[3];
    if (kind == 1) {
      cs.merge = is_col ? 2 : 1;
      cs.p = xp;
      cs.q = xq;
      cs.a = va;
      cs.b = vb;
    } else if (kind == 2) {
      cs.fac = va;
    } else {
      cs.merge = 3;
    }
    if (kind == 3) {
      cs.del_row = cs.del_col = kNone;
    } else if (!is_col) {
      cs.del_row = idx;
      cs.del_col = kind == 1 ? xq : xp;
    } else {
      cs.del_col = idx;
      cs.del_row = kind == 1 ? xq : xp;
    }
    // pass 1: row lengths, the union of nonzero columns, overflow
    int cnt[RPL];
    uint64_t cm0 = 0, cm1 = 0;
    bool ovf = false;
#pragma unroll
    for (int k = 0; k < RPL; ++k) {
      const int rc = lane + LW * k;
      int n = 0;
      if (rc < mc) {
        const int r = rc + (rc >= cs.del_row);
        if (!child_row(v, cs, r, [&](int cc, int64_t) {
              ++n;
              if (cc < 64)
                cm0 |= 1ull << cc;
              else
                cm1 |= 1ull << (cc - 64);
            }))
          ovf = true;
      }
      cnt[k] = n;
    }
    cm0 = G.or_all(cm0);
    cm1 = G.or_all(cm1);
    bool zero_row = false;
#pragma unroll
    for (int k = 0; k < RPL; ++k)
      if (lane + LW * k < mc && cnt[k] == 0) zero_row = true;
    zero_row = G.any(zero_row);
    ovf = G.any(ovf);
    if (ovf && lane == 0) atomicCAS(X.err, 0, PERM_EOVERFLOW);
    const int ncols = __popcll(cm0) + __popcll(cm1);
    bool keep = !ovf && !zero_row && ncols == mc;
    int offs[RPL];
    int cnnz = 0;
    int64_t o = -1;
    if (keep) {
#pragma unroll
      for (int k = 0; k < RPL; ++k) {
        int tot;
        offs[k] = cnnz + G.excl_scan(cnt[k], tot);
        cnnz += tot;
      }
      o = child_block(X, p, c, pw, blk_words(mc, cnnz), G);
      keep = o >= 0;
    }
    if (keep) {
      // pass 2: write rows
      uint64_t* blk = X.arena_out + o;
      uint16_t* rowptr = reinterpret_cast<uint16_t*>(blk);
      uint8_t* col = reinterpret_cast<uint8_t*>(blk + blk_rp_words(mc));
      int64_t* val = reinterpret_cast<int64_t*>(blk + blk_rp_words(mc) + blk_col_words(cnnz));
      if (lane == 0) rowptr[mc] = (uint16_t)cnnz;
#pragma unroll
      for (int k = 0; k < RPL; ++k) {
        const int rc = lane + LW * k;
        if (rc < mc) {
          const int r = rc + (rc >= cs.del_row);
          rowptr[rc] = (uint16_t)offs[k];
          int w = offs[k];
          child_row(v, cs, r, [&](int cc, int64_t xv) {
            col[w] = (uint8_t)cc;
            val[w] = xv;
            ++w;
          });
        }
      }
    }
    if (lane == 0) {
      X.valid[slot] = keep ? 1 : 0;
      if (keep) {
        X.child.m[slot] = mc;
        X.child.nnz[slot] = cnnz;
        X.child.off[slot] = o;
        X.child.mat[slot] = X.parent.mat[p];
        X.child.depth_left[slot] = dl - 1;
        u256 cc = pcoef;
        if (cs.fac != 1) {
          if (X.mod)
            cc.w[0] = pcoef.w[0] % X.mod * (uint64_t)cs.fac % X.mod;  // residues: the upper words stay 0
          else
            cc = u256_mul_s64(pcoef, cs.fac);
        }
        for (int w = 0; w < 4; ++w) X.child.coef[4 * slot + w] = cc.w[w];
        wm.order = max(wm.order, mc);
        if (dl - 1 > 0 && mc > cut) wm.open = max(wm.open, mc);
      }
    }
  }
}

template <int RPL>
__global__ void __launch_bounds__(kLevelWarps * 32) k_expand_level(ExpandLevelArgs A) {
  __shared__ int32_t ccnt[kLevelWarps][RPL * 32];
  extern __shared__ __align__(16) uint64_t stage[];
  const int lane = threadIdx.x & 31;
  const int wib = threadIdx.x >> 5;
  ExpandCtx X;
  X.parent = A.parent;
  X.arena_in = A.arena_in;
  X.child = A.child;
  X.arena_out = A.arena_out;
  X.child_off_base = A.child_off_base;
  X.bump = nullptr;
  X.cap_words = 0;
  X.valid = A.valid;
  X.leaf_size = A.leaf_size;
  X.split_floor = A.split_floor;
  X.kslots = A.kslots;
  X.mod = A.mod;
  X.err = A.err;
  const int64_t nwarps = (int64_t)gridDim.x * kLevelWarps;
  WarpMax wm;  // unused: the compaction takes the level's maxima
  const Grp<32> G(lane);
  for (int64_t p = (int64_t)blockIdx.x * kLevelWarps + wib; p < A.np; p += nwarps)
    expand_parent<RPL, 32>(X, p, G, ccnt[wib], stage + wib * kStageWords, kStageWords, wm);
}

// ---- multi-level driver ---------------------------------------------------------

__device__ __forceinline__ long long ld_cg(const long long* p) { return __ldcg(p); }

// Sum over the block; every thread gets the total.  red: kFrontWarps entries.
__device__ __forceinline__ long long block_sum(long long v, long long* red) {
#pragma unroll
  for (int d = 16; d > 0; d >>= 1) v += __shfl_xor_sync(0xffffffffu, v, d);
  __syncthreads();
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  long long t = 0;
#pragma unroll
  for (int w = 0; w < kFrontWarps; ++w) t += red[w];
  return t;
}

// Exclusive scan of 0/1 flags over the block; total in *tot.  red:
// kFrontWarps entries.
__device__ __forceinline__ int block_excl_scan(int v, int* red, int& tot) {
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  int wt;
  const int x = warp_excl_scan(v, lane, wt);
  __syncthreads();
  if (lane == 0) red[wib] = wt;
  __syncthreads();
  int before = 0, all = 0;
#pragma unroll
  for (int w = 0; w < kFrontWarps; ++w) {
    if (w < wib) before += red[w];
    all += red[w];
  }
  tot = all;
  return before + x;
}

// Grid-wide barrier of a cooperative launch: a monotone arrival counter,
// target = (barriers passed) * gridDim.x.  Thread 0 waits with a time
// limit; on expiry the first error becomes PERM_ETIMEOUT and the whole
// block returns false.
__device__ bool grid_barrier(unsigned long long* bar, unsigned long long& target, int32_t* err) {
  __syncthreads();
  int failed = 0;
  if (threadIdx.x == 0) {
    target += gridDim.x;
    __threadfence();
    atomicAdd(bar, 1ull);
    const uint64_t t0 = globaltimer_ns();
    unsigned spins = 0;
    while (*(volatile unsigned long long*)bar < target) {
      __nanosleep(64);
      if ((++spins & 255u) == 0 && globaltimer_ns() - t0 > (uint64_t)kBarrierTimeoutNs) {
        atomicCAS(err, 0, PERM_ETIMEOUT);
        failed = 1;
        break;
      }
    }
    __threadfence();
  }
  return __syncthreads_or(failed) == 0;
}

template <int RPL, int LW>
__global__ void __launch_bounds__(kFrontThreads) k_expand_front(ExpandFrontArgs F) {
  // groups of LW lanes, one parent (or child) each
  constexpr int GPW = 32 / LW;
  constexpr int NG = kFrontWarps * GPW;
  constexpr int SW = kStageWords / GPW;  // stage words per group
  __shared__ int32_t ccnt[NG][RPL * LW];
  extern __shared__ __align__(16) uint64_t stage[];
  __shared__ long long red64[kFrontWarps];
  __shared__ int red32[kFrontWarps];
  const int lane = threadIdx.x & 31;
  const int wib = threadIdx.x >> 5;
  const int64_t G = gridDim.x, b = blockIdx.x;
  const Grp<LW> grp(lane);
  const int gid = wib * GPW + lane / LW;
  unsigned long long target = 0;
  ExpandFrontState S = *F.state;
  bool failed = false;  // an error flag raised during the last level
  for (;;) {
    // the same decision in every block: S and the error flag were read
    // between the same two barriers (the flag is only raised while
    // children are built, before the first barrier of a level)
    const int K = F.kslots;
    // also stop when every order fits the next narrower variant (fewer rows
    // per lane): the host launches that one for the remaining levels
    constexpr int narrower = LW == 16 ? 0 : (RPL > 1 ? RPL * 16 : 16);
    bool stop = failed || S.level >= F.max_levels || S.ncur <= 0 || S.max_order > RPL * LW ||
                S.max_order <= narrower || K * S.ncur > F.cap_jobs || K * S.used_words > F.cap_words;
    if (!stop && F.adaptive) {
      const bool big = S.max_open > F.big_order;
      const bool soft = S.max_open > F.soft_order && S.ncur < F.soft_cap_jobs;
      const bool more = S.ncur < F.target_jobs && S.max_open > 0;
      stop = !big && !soft && !more;
    }
    if (stop) break;
    const int cb = S.cb;
    ExpandCtx X;
    X.parent = F.buf[cb];
    X.arena_in = F.arena[cb];
    X.child = F.slots;
    X.arena_out = F.arena[cb ^ 1];
    X.child_off_base = nullptr;
    X.bump = F.lvl_words + S.level;
    X.cap_words = F.cap_words;
    X.valid = F.valid;
    X.leaf_size = F.leaf_size;
    X.split_floor = F.adaptive ? S.max_open - F.band : 0;
    X.kslots = F.kslots;
    X.mod = F.mod;
    X.err = F.err;
    const int64_t p0 = S.ncur * b / G, p1 = S.ncur * (b + 1) / G;
    WarpMax wm;
    if (K * S.ncur <= G * NG) {
      // small frontier: a group per child, cutting the level's latency
      for (int64_t t = K * p0 + gid; t < K * p1; t += NG)
        expand_parent<RPL, LW>(X, t / K, grp, ccnt[gid], stage + gid * SW, SW, wm, (int)(t % K));
    } else {
      for (int64_t p = p0 + gid; p < p1; p += NG)
        expand_parent<RPL, LW>(X, p, grp, ccnt[gid], stage + gid * SW, SW, wm);
    }
    if (grp.sub == 0) {  // one update of the level's maxima per group
      if (wm.order > 0) atomicMax(F.lvl_maxo + S.level, wm.order);
      if (wm.open > 0) atomicMax(F.lvl_maxopen + S.level, wm.open);
    }
    __syncthreads();
    long long kept = 0;
    for (int64_t t = K * p0 + threadIdx.x; t < K * p1; t += kFrontThreads) kept += F.valid[t];
    kept = block_sum(kept, red64);
    if (threadIdx.x == 0) __stcg(F.partial + b, kept);
    if (!grid_barrier(F.bar, target, F.err)) return;
    failed = __syncthreads_or(threadIdx.x == 0 && __ldcg(F.err) != 0) != 0;
    long long before = 0, total = 0;
    for (int64_t t = threadIdx.x; t < G; t += kFrontThreads) {
      const long long x = ld_cg(F.partial + t);
      total += x;
      if (t < b) before += x;
    }
    before = block_sum(before, red64);
    total = block_sum(total, red64);
    // compaction of this block's slots, natural order kept
    const JobArrays src = F.slots, dst = F.buf[cb ^ 1];
    int64_t base = before;
    for (int64_t t0 = K * p0; t0 < K * p1; t0 += kFrontThreads) {
      const int64_t t = t0 + threadIdx.x;
      const int keep = t < K * p1 ? F.valid[t] : 0;
      int tot;
      const int64_t d = base + block_excl_scan(keep, red32, tot);
      if (keep) {
        dst.m[d] = src.m[t];
        dst.nnz[d] = src.nnz[t];
        dst.off[d] = src.off[t];
        dst.mat[d] = src.mat[t];
        dst.depth_left[d] = src.depth_left[t];
        for (int w = 0; w < 4; ++w) dst.coef[4 * d + w] = src.coef[4 * t + w];
      }
      base += tot;
    }
    if (!grid_barrier(F.bar, target, F.err)) return;
    S.ncur = total;
    S.used_words = (int64_t)__ldcg(F.lvl_words + S.level);
    S.max_order = __ldcg(F.lvl_maxo + S.level);
    S.max_open = __ldcg(F.lvl_maxopen + S.level);
    S.cb ^= 1;
    S.level += 1;
  }
  if (b == 0 && threadIdx.x == 0) *F.state = S;
}

template <int RPL>
cudaError_t launch_level_rpl(const ExpandLevelArgs& a, cudaStream_t s) {
  int64_t blocks = (a.np + kLevelWarps - 1) / kLevelWarps;
  if (blocks > 152 * 32) blocks = 152 * 32;
  static bool attr_set = false;
  if (!attr_set) {
    cudaError_t e = cudaFuncSetAttribute(k_expand_level<RPL>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)kLevelSmem);
    if (e != cudaSuccess) return e;
    attr_set = true;
  }
  k_expand_level<RPL><<<(unsigned)blocks, kLevelWarps * 32, kLevelSmem, s>>>(a);
  return cudaGetLastError();
}

template <int RPL, int LW>
cudaError_t launch_front_rpl(ExpandFrontArgs a, int* grid, cudaStream_t s) {
  int dev = 0, sms = 0, coop = 0, per_sm = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_expand_front<RPL, LW>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)kFrontSmem);
  if (e == cudaSuccess)
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_expand_front<RPL, LW>, kFrontThreads,
                                                      kFrontSmem);
  if (e != cudaSuccess) return e;
  *grid = 0;
  if (!coop || per_sm <= 0) return cudaSuccess;  // not available: per-level launches only
  int g = sms * (per_sm < 2 ? per_sm : 2);
  if (g > PERM_FRONT_MAX_BLOCKS) g = PERM_FRONT_MAX_BLOCKS;
  void* args[] = {&a};
  e = cudaLaunchCooperativeKernel((const void*)k_expand_front<RPL, LW>, dim3((unsigned)g), dim3(kFrontThreads),
                                  args, kFrontSmem, s);
  if (e == cudaSuccess) *grid = g;
  return e;
}

}  // namespace

cudaError_t launch_expand_level(const ExpandLevelArgs& a, int max_order, cudaStream_t s) {
  if (a.np <= 0) return cudaSuccess;
  if (max_order <= 32) return launch_level_rpl<1>(a, s);
  if (max_order <= 64) return launch_level_rpl<2>(a, s);
  return launch_level_rpl<4>(a, s);
}

cudaError_t launch_expand_front(const ExpandFrontArgs& a, int max_order, int* grid, cudaStream_t s) {
  if (max_order <= 16) return launch_front_rpl<1, 16>(a, grid, s);
  if (max_order <= 32) return launch_front_rpl<1, 32>(a, grid, s);
  if (max_order <= 64) return launch_front_rpl<2, 32>(a, grid, s);
  return launch_front_rpl<4, 32>(a, grid, s);
}

__global__ void k_child_capacity(JobArrays parent, int64_t np, int kslots, int64_t* words) {
  int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (p < np) words[p] = kslots * blk_words(parent.m[p], parent.nnz[p]);
}

// stat[0]: largest kept order, stat[1]: words of the kept blocks, stat[2]:
// kept jobs, stat[3]: largest order of a kept job still to split (depth
// left and order above cut) -- reduced per warp, one atomic per warp.
__global__ void k_compact(JobArrays src, const int32_t* valid, const int32_t* pos, int64_t nslots, JobArrays dst,
                          int cut, long long* stat) {
  const int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const bool keep = s < nslots && valid[s];
  unsigned m = 0, words = 0, mo = 0;
  if (keep) {
    const int64_t d = pos[s];
    m = (unsigned)src.m[s];
    mo = src.depth_left[s] > 0 && src.m[s] > cut ? m : 0u;
    words = (unsigned)blk_words(src.m[s], src.nnz[s]);
    dst.m[d] = src.m[s];
    dst.nnz[d] = src.nnz[s];
    dst.off[d] = src.off[s];
    dst.mat[d] = src.mat[s];
    dst.depth_left[d] = src.depth_left[s];
    for (int w = 0; w < 4; ++w) dst.coef[4 * d + w] = src.coef[4 * s + w];
  }
  const unsigned mx = __reduce_max_sync(0xffffffffu, m);
  const unsigned mox = __reduce_max_sync(0xffffffffu, mo);
  const unsigned sw = __reduce_add_sync(0xffffffffu, words);
  const unsigned nk = __reduce_add_sync(0xffffffffu, keep ? 1u : 0u);
  if ((threadIdx.x & 31) == 0 && nk) {
    atomicMax(stat, (long long)mx);
    atomicAdd(reinterpret_cast<unsigned long long*>(stat + 1), (unsigned long long)sw);
    atomicAdd(reinterpret_cast<unsigned long long*>(stat + 2), (unsigned long long)nk);
    atomicMax(stat + 3, (long long)mox);
  }
}

cudaError_t launch_child_capacity(const JobArrays& parent, int64_t np, int kslots, int64_t* words, cudaStream_t s) {
  if (np <= 0) return cudaSuccess;
  k_child_capacity<<<(unsigned)((np + 255) / 256), 256, 0, s>>>(parent, np, kslots, words);
  return cudaGetLastError();
}

cudaError_t launch_compact_jobs(const JobArrays& src, const int32_t* valid, const int32_t* pos, int64_t nslots,
                                JobArrays dst, int cut, long long* stat, cudaStream_t s) {
  if (nslots <= 0) return cudaSuccess;
  k_compact<<<(unsigned)((nslots + 255) / 256), 256, 0, s>>>(src, valid, pos, nslots, dst, cut, stat);
  return cudaGetLastError();
}
