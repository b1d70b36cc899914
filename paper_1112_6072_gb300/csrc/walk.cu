// K1, traversal driver: Algorithm PH, Step 2 (Section 2.2) without a grid
// barrier per level.
//
// The level-by-level driver (expand.cu) pays one grid-wide synchronisation
// per level of Eq. 2, and a sparse 3-regular matrix of order n needs n - L
// levels whose first half holds only a few nodes.  Here every warp walks a
// subtree of the expansion depth first, in place, on a dense tile in shared
// memory (tile.cuh: the depth-first evaluator's node machinery -- the same
// pivot and the same children as expand.cu, undone on the way back).  Only
// the jobs -- the nodes that are not split further -- are compacted back to
// CSR blocks, each with the path of child indices that led to it.  A warp
// that runs dry takes a ticket from a global queue; a warp about to split a
// node while other warps wait hands them the node's other children
// (compacted to CSR) and goes on with child 0.  The natural (breadth-first)
// order of Algorithm PH is the lexicographic order of the paths (a node
// carried unchanged through the last levels sits where its child 0 would),
// so one sort of the path keys gives the job list of the level-by-level
// driver.
//
// Rule per node (the level-by-level driver's rule without its waiting band):
// a node is a job when it has no levels left, its order is at most
// max(L, 2), or its sparsest line has s >= 5 nonzeros (unless Eq. 2's third
// child is enabled); a node holding a zero line is dropped.  Per-depth
// counts of nodes, of jobs and the largest order still to split let the host
// replay the automatic depth rule and check that it reaches the same depth.
//
// Tile entries are int32: a merge whose entry leaves int32, like a full
// buffer, stops the walk with an internal status, and the host runs the
// level-by-level driver (int64 entries) instead.  Every wait is bounded: a
// warp waiting for a ticket gives up after the deadline (PERM_ETIMEOUT).
#include <cuda_runtime.h>

#include <cstdint>

#include "internal.h"
#include "tile.cuh"
#include "wide.cuh"

namespace {

typedef int32_t WE;              // tile entries
constexpr int kOutChunk = 16;    // output slots a warp reserves at a time (as api.cu sizes them)
constexpr int kCheckEvery = 16;   // nodes between looks at the error flag and the waiting warps while none wait
constexpr int kCheckWaiting = 4;  // the same while warps wait

template <int TILE>
struct WalkCfg {
  static constexpr int WARPS = TILE <= 32 ? 8 : 4;  // warps per block
  static constexpr int MINB = TILE <= 32 ? 3 : 2;   // blocks per SM the registers are sized for
  // tile, masks and a scratch line (the in-place children's saved line); the staging copy follows
  static constexpr size_t FIXED_BYTES =
      TileCfg<TILE, WE>::TILE_BYTES + TileCfg<TILE, WE>::MASK_BYTES + sizeof(int64_t) * (TILE + 2);
};

__host__ __device__ __forceinline__ size_t walk_warp_bytes(int tile, int stage_words) {
  return (tile <= 32 ? WalkCfg<32>::FIXED_BYTES : WalkCfg<64>::FIXED_BYTES) + sizeof(uint64_t) * (size_t)stage_words;
}

__device__ __forceinline__ int volatile_ld(const int32_t* p) { return *(const volatile int32_t*)p; }
__device__ __forceinline__ unsigned long long volatile_ld(const unsigned long long* p) {
  return *(const volatile unsigned long long*)p;
}

struct WarpCtx {
  int lane;
  int64_t a_pos, a_end;  // arena chunk of this warp
  int64_t o_pos, o_end;  // output chunk of this warp
  unsigned long long emitted;
};

// Arena words for a block (lane-uniform result; -1 when the arena is full).
__device__ __forceinline__ int64_t walk_alloc(const WalkArgs& A, WarpCtx& W, int64_t words) {
  if (W.a_pos + words > W.a_end) {
    unsigned long long b = 0;
    if (W.lane == 0) b = atomicAdd(A.arena_used, (unsigned long long)A.arena_chunk);
    b = __shfl_sync(0xffffffffu, b, 0);
    if ((int64_t)b + A.arena_chunk > A.cap_words) {
      if (W.lane == 0) atomicCAS(A.err, 0, WALK_FULL);
      return -1;
    }
    W.a_pos = (int64_t)b;
    W.a_end = (int64_t)b + A.arena_chunk;
  }
  const int64_t o = W.a_pos;
  W.a_pos += words;
  return o;
}

// The active sub-matrix of the tile (rows R, columns C, in index order) as a
// CSR block in the arena; returns its offset (-1 when the arena is full),
// its order and its nonzeros.
template <int TILE>
__device__ __noinline__ int64_t compact_tile(const WalkArgs& A, WarpCtx& W, const WE* __restrict__ T,
                                             const uint64_t* __restrict__ rowbits, uint64_t R, uint64_t C,
                                             int& m_out, int& nnz_out) {
  constexpr int S = TileCfg<TILE, WE>::STRIDE;
  constexpr int RPL = TILE / 32;
  const int lane = W.lane;
  const int m = __popcll(R);
  int cnt[RPL], row[RPL];
#pragma unroll
  for (int t = 0; t < RPL; ++t) {
    const int k = lane + 32 * t;
    row[t] = k < m ? nth_bit(R, k) : 0;
    cnt[t] = k < m ? __popcll(rowbits[row[t]] & C) : 0;
  }
  int offs[RPL];
  int nnz = 0;
#pragma unroll
  for (int t = 0; t < RPL; ++t) {
    int x = cnt[t];
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, x, d);
      if (lane >= d) x += y;
    }
    offs[t] = nnz + x - cnt[t];
    nnz += __shfl_sync(0xffffffffu, x, 31);
  }
  m_out = m;
  nnz_out = nnz;
  const int64_t o = walk_alloc(A, W, blk_words(m, nnz));
  if (o < 0) {
    __syncwarp();
    return -1;
  }
  uint64_t* blk = A.arena + o;
  uint16_t* rowptr = reinterpret_cast<uint16_t*>(blk);
  uint8_t* colp = reinterpret_cast<uint8_t*>(blk + blk_rp_words(m));
  int64_t* valp = reinterpret_cast<int64_t*>(blk + blk_rp_words(m) + blk_col_words(nnz));
  if (lane == 0) rowptr[m] = (uint16_t)nnz;
#pragma unroll
  for (int t = 0; t < RPL; ++t) {
    const int k = lane + 32 * t;
    if (k < m) {
      rowptr[k] = (uint16_t)offs[t];
      const int r = row[t];
      uint64_t cm = rowbits[r] & C;
      int w = offs[t];
      while (cm) {
        const int c = __ffsll((long long)cm) - 1;
        cm &= cm - 1;
        colp[w] = (uint8_t)__popcll(C & (bit64(c) - 1));
        valp[w] = (int64_t)T[r * S + c];
        ++w;
      }
    }
  }
  // a lane read rows other lanes own: every read done before any lane
  // changes the tile again (an undo writes each lane's own rows)
  __syncwarp();
  return o;
}

// Write a job's header and path key; its block is at off.
__device__ __noinline__ void walk_emit(const WalkArgs& A, WarpCtx& W, int m, int nnz, int64_t off, int mat, int depth,
                          const u256& coef, uint64_t key_lo, uint64_t key_hi, unsigned* h_term) {
  if (W.o_pos >= W.o_end) {
    unsigned long long b = 0;
    if (W.lane == 0) b = atomicAdd(A.out_used, (unsigned long long)kOutChunk);
    b = __shfl_sync(0xffffffffu, b, 0);
    W.o_pos = (int64_t)b;
    W.o_end = (int64_t)b + kOutChunk;
  }
  const int64_t s = W.o_pos++;
  if (s >= A.cap_out) {
    if (W.lane == 0) atomicCAS(A.err, 0, WALK_FULL);
    return;
  }
  if (W.lane == 0) {
    A.out.m[s] = m;
    A.out.nnz[s] = nnz;
    A.out.off[s] = off;
    A.out.mat[s] = mat;
    A.out.depth_left[s] = 0;
    A.out_key[2 * s] = key_lo;
    A.out_key[2 * s + 1] = key_hi;
    if (depth < A.hist_len) atomicAdd(h_term + depth, 1u);
  }
  if (W.lane < 4) A.out.coef[4 * s + W.lane] = coef.w[W.lane];
  W.emitted += 1;
}

// Append a node (block at off, written by this warp) to queue Q; counted as
// outstanding work when Q is this phase's work queue.
__device__ __noinline__ void walk_push(const WalkArgs& A, const WalkQueue& Q, bool work, int lane, int m, int nnz, int64_t off,
                          int mat, int dl, int depth, const u256& coef, uint64_t key_lo, uint64_t key_hi) {
  __syncwarp();
  __threadfence();  // every lane's part of the block before the slot is published
  __syncwarp();
  if (lane == 0) {
    if (work) atomicAdd(A.outstanding, 1ull);
    const unsigned long long t = atomicAdd(Q.tail, 1ull);
    if ((int64_t)t >= Q.cap) {
      atomicCAS(A.err, 0, WALK_FULL);
    } else {
      Q.m[t] = m;
      Q.nnz[t] = nnz;
      Q.mat[t] = mat;
      Q.dl[t] = dl;
      Q.depth[t] = depth;
      Q.off[t] = off;
      for (int w = 0; w < 4; ++w) Q.coef[4 * t + w] = coef.w[w];
      Q.key[2 * t] = key_lo;
      Q.key[2 * t + 1] = key_hi;
      __threadfence();
      *(volatile int32_t*)(Q.ready + t) = 1;
    }
  }
  __syncwarp();
}

// Child index c at absolute depth t in a path key (bits_per_level bits per
// level, the first level in the highest bits).
__device__ __forceinline__ void key_set(uint64_t& lo, uint64_t& hi, int t, uint64_t c, int bpl, int levels) {
  const int shift = bpl * (levels - t);
  const uint64_t mask = (1ull << bpl) - 1;
  if (shift < 0) return;
  if (shift >= 64)
    hi = (hi & ~(mask << (shift - 64))) | (c << (shift - 64));
  else
    lo = (lo & ~(mask << shift)) | (c << shift);
}

// 64-bit word k of a block another warp wrote (read from L2, never from a
// possibly stale L1 line)
__device__ __forceinline__ uint64_t blk_word(const uint64_t* b, int64_t k) { return __ldcg(b + k); }

template <int TILE>
__global__ void __launch_bounds__(WalkCfg<TILE>::WARPS * 32, WalkCfg<TILE>::MINB) k_expand_walk(WalkArgs A) {
  constexpr int S = TileCfg<TILE, WE>::STRIDE;
  constexpr int NW = WalkCfg<TILE>::WARPS;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int lane = threadIdx.x & 31;
  const int wib = threadIdx.x >> 5;
  const size_t warp_bytes = walk_warp_bytes(TILE, A.stage_words);
  unsigned char* base = smem_raw + (size_t)wib * warp_bytes;
  Eq2Tile<TILE, WE> D;
  D.T = reinterpret_cast<WE*>(base);
  D.rowbits = reinterpret_cast<uint64_t*>(base + TileCfg<TILE, WE>::TILE_BYTES);
  D.colbits = D.rowbits + TILE;
  D.lane = lane;
  D.modp = A.mod;
  // scratch line of the in-place children: mask at [-1], line at [0, TILE)
  int64_t* scratch = reinterpret_cast<int64_t*>(D.colbits + TILE) + 2;
  uint64_t* stage = reinterpret_cast<uint64_t*>(base + WalkCfg<TILE>::FIXED_BYTES);
  const int64_t gwarp = (int64_t)blockIdx.x * NW + wib;
  D.undo = A.undo + gwarp * A.undo_words_per_warp;
  unsigned* h_nodes = reinterpret_cast<unsigned*>(smem_raw + (size_t)NW * warp_bytes);
  unsigned* h_term = h_nodes + A.hist_len;
  int* h_mo = reinterpret_cast<int*>(h_term + A.hist_len);
  for (int k = threadIdx.x; k < A.hist_len; k += blockDim.x) {
    h_nodes[k] = 0;
    h_term[k] = 0;
    h_mo[k] = 0;
  }
  __syncthreads();

  const int cut = A.leaf_size > 2 ? A.leaf_size : 2;
  const bool three = A.kslots == 3;
  const int bpl = A.bits_per_level, levels = A.key_levels;
  const uint64_t t_start = globaltimer_ns();
  WarpCtx W;
  W.lane = lane;
  W.a_pos = W.a_end = 0;
  W.o_pos = W.o_end = 0;
  W.emitted = 0;
  int since_check = 0;
  bool waiting = true;  // other warps wait for work: hand them siblings (looked up every few nodes)

  for (;;) {
    // ---- a subtree root from the work queue
    unsigned long long ticket = 0;
    if (lane == 0) ticket = atomicAdd(A.q.head, 1ull);
    ticket = __shfl_sync(0xffffffffu, ticket, 0);
    int got = 0;
    if (lane == 0) {
      // poll this ticket's own slot, the shared counters only every 8th time,
      // with a growing pause: thousands of idle warps must not hammer one L2 line
      unsigned pause = 64;
      for (unsigned spins = 0;; ++spins) {
        if ((int64_t)ticket < A.q.cap && volatile_ld(A.q.ready + ticket) != 0) {
          got = 1;
          break;
        }
        if ((spins & 7u) == 7u) {
          if ((long long)volatile_ld(A.outstanding) <= 0 || volatile_ld(A.err) != 0) break;
          if (globaltimer_ns() - t_start > (uint64_t)A.timeout_ns) {
            atomicCAS(A.err, 0, PERM_ETIMEOUT);
            break;
          }
        }
        __nanosleep(pause);
        if (pause < 2048) pause *= 2;
      }
      __threadfence();
    }
    got = __shfl_sync(0xffffffffu, got, 0);
    if (!got) break;
    __threadfence();
    const int64_t t = (int64_t)ticket;
    const int m0 = __ldcg(A.q.m + t), nnz0 = __ldcg(A.q.nnz + t), mat = __ldcg(A.q.mat + t);
    const int dl0 = __ldcg(A.q.dl + t), depth0 = __ldcg(A.q.depth + t);
    const int64_t off0 = __ldcg(A.q.off + t);
    for (int w = 0; w < 4; ++w) D.coef.w[w] = __ldcg(A.q.coef + 4 * t + w);
    uint64_t key_lo = __ldcg(A.q.key + 2 * t), key_hi = __ldcg(A.q.key + 2 * t + 1);
    bool stop = m0 > TILE;
    // ---- the node into the tile: its block staged with 16-byte L2 reads,
    // the tile's first m0 rows cleared
    const int64_t bw = blk_words(m0, nnz0);
    const bool staged = bw <= A.stage_words;
    const uint64_t* blk = A.arena + off0;
    if (staged) {
      const uint4* s4 = reinterpret_cast<const uint4*>(blk);
      uint4* d4 = reinterpret_cast<uint4*>(stage);
      for (int64_t k = lane; k < bw / 2; k += 32) d4[k] = __ldcg(s4 + k);
    }
    {
      const int rows = stop ? 0 : m0;
      int4* t4 = reinterpret_cast<int4*>(D.T);
      const int n4 = (int)((sizeof(WE) * (size_t)rows * S + 15) / 16);
      for (int k = lane; k < n4; k += 32) t4[k] = make_int4(0, 0, 0, 0);
      for (int k = lane; k < TILE; k += 32) D.rowbits[k] = D.colbits[k] = 0;
    }
    __syncwarp();
    const int rpw = (int)blk_rp_words(m0), cw = (int)blk_col_words(nnz0);
    const uint16_t* srp = reinterpret_cast<const uint16_t*>(stage);
    const uint8_t* scol = reinterpret_cast<const uint8_t*>(stage + rpw);
    const int64_t* sval = reinterpret_cast<const int64_t*>(stage + rpw + cw);
    bool fits = true;
    for (int r = lane; r < m0 && !stop; r += 32) {
      const int b = staged ? srp[r] : (int)((blk_word(blk, r / 4) >> (16 * (r % 4))) & 0xffff);
      const int e = staged ? srp[r + 1] : (int)((blk_word(blk, (r + 1) / 4) >> (16 * ((r + 1) % 4))) & 0xffff);
      uint64_t rb = 0;
      for (int q = b; q < e; ++q) {
        const int c = staged ? scol[q] : (int)((blk_word(blk, rpw + q / 8) >> (8 * (q % 8))) & 0xff);
        const int64_t x = staged ? sval[q] : (int64_t)blk_word(blk, rpw + cw + q);
        if ((int64_t)(WE)x != x) fits = false;
        D.T[r * S + c] = (WE)x;
        rb |= bit64(c);
        atomicOr((unsigned long long*)&D.colbits[c], (unsigned long long)bit64(r));
      }
      D.rowbits[r] = rb;
    }
    fits = __all_sync(0xffffffffu, fits);
    __syncwarp();
    if (!fits || stop) {
      if (lane == 0) atomicCAS(A.err, 0, WALK_FULL);
      stop = true;
    }
    D.R = D.C = (m0 == 64) ? ~0ull : (bit64(m0) - 1);
    // ---- depth-first walk of the subtree: rel = depth of the current node below its root.
    // One call site per tile operation (the kernel's code stays small enough
    // for the instruction cache): a visit either writes the node out, or
    // splits it -- children that are jobs (or that go to waiting warps)
    // applied and undone with the scratch line -- and then moves into child
    // `next`, or backs up to the next child not yet walked.
    int rel = 0;
    bool done = stop;
    while (!done) {
      const int depth = depth0 + rel;
      // the error flag and the waiting warps: every kCheckWaiting nodes while
      // warps wait, else every kCheckEvery nodes
      const bool check = ++since_check >= (waiting ? kCheckWaiting : kCheckEvery);
      unsigned long long q_h = 0, q_t = 0;
      int e = 0;
      if (check && lane == 0) {
        q_h = __ldcg(A.q.head);
        q_t = __ldcg(A.q.tail);
        e = __ldcg(A.err);
      }
      const unsigned long long key = D.pivot_key();
      const int s = (int)(key >> 17);
      const int mact = __popcll(D.R);
      const int dl = dl0 - rel;
      const bool open = dl > 0 && mact > cut;
      if (check) {
        since_check = 0;
        if (__shfl_sync(0xffffffffu, e, 0) != 0) break;  // another warp failed: abandon the walk
        waiting = __shfl_sync(0xffffffffu, q_h > q_t ? 1 : 0, 0) != 0;
      }
      Frame f;
      int64_t pv[4] = {0, 0, 0, 0};
      u256 pcoef = D.coef;
      int next = -1;
      bool failed = false;
      if (s > 0) {
        const bool handover = open && mact <= A.handover_order;
        if (!handover && lane == 0 && depth < A.hist_len) {
          atomicAdd(h_nodes + depth, 1u);
          if (open) atomicMax(h_mo + depth, mact);
        }
        if (handover || !open || (s >= 5 && !three)) {
          // a job, or a node for the narrower phase (which counts it)
          int mj, nj;
          const int64_t o = compact_tile<TILE>(A, W, D.T, D.rowbits, D.R, D.C, mj, nj);
          if (o >= 0) {
            if (handover)
              walk_push(A, A.hand, false, lane, mj, nj, o, mat, dl, depth, D.coef, key_lo, key_hi);
            else
              walk_emit(A, W, mj, nj, o, mat, depth, D.coef, key_lo, key_hi, h_term);
          }
        } else {
          f.is_col = (int)((key >> 16) & 1);
          f.idx = (int)(key & 0xffff);
          f.k = s;
          f.child = 0;
          uint64_t line = f.is_col ? (D.colbits[f.idx] & D.R) : (D.rowbits[f.idx] & D.C);
          for (int q = 0; q < 4; ++q) {
            f.pos[q] = 0;
            if (line) {
              const int c = __ffsll((long long)line) - 1;
              line &= line - 1;
              f.pos[q] = c;
              pv[q] = (int64_t)(f.is_col ? D.T[c * S + f.idx] : D.T[f.idx * S + c]);
            }
          }
          const int nch = Eq2Tile<TILE, WE>::nchildren(s);
          // every child a job: all of them written out in place; else the
          // children after the first go to waiting warps, if any
          const bool inplace = dl - 1 <= 0 || (mact - 1 <= cut && s < 5);
          if (!inplace) {
            if (rel >= A.max_rel_depth) {
              if (lane == 0) atomicCAS(A.err, 0, WALK_FULL);
              break;
            }
            D.store_frame(rel, f, pv, pcoef);
            __syncwarp();
          }
          const int c1 = inplace || waiting ? nch : 1;
          for (int c = inplace ? 0 : 1; c < c1; ++c) {
            if (!D.apply_to(scratch, f, pv, c)) {
              failed = true;
            } else if (!inplace || (D.pivot_key() >> 17) > 0) {  // a child holding a zero line is dropped
              if (inplace && lane == 0 && depth + 1 < A.hist_len) atomicAdd(h_nodes + depth + 1, 1u);
              int mj, nj;
              const int64_t o = compact_tile<TILE>(A, W, D.T, D.rowbits, D.R, D.C, mj, nj);
              uint64_t klo = key_lo, khi = key_hi;
              key_set(klo, khi, depth + 1, (uint64_t)c, bpl, levels);
              if (o >= 0) {
                if (inplace)
                  walk_emit(A, W, mj, nj, o, mat, depth + 1, D.coef, klo, khi, h_term);
                else
                  walk_push(A, A.q, true, lane, mj, nj, o, mat, dl - 1, depth + 1, D.coef, klo, khi);
              }
            }
            D.undo_from(scratch, f, pv, pcoef, c);
          }
          if (failed) {
            if (lane == 0) atomicCAS(A.err, 0, WALK_FULL);
            break;
          }
          if (!inplace) {
            if (c1 > 1) {
              D.set_child(rel, 1 << 8);  // child 0, the others handed over
              __syncwarp();
            }
            next = 0;
          }
        }
      }
      // ---- the move: into child `next` of this node, or back up to the next child not yet walked
      int lv = rel, c = next;
      if (c < 0) {
        for (;;) {
          if (rel == 0) {
            done = true;
            break;
          }
          D.load_frame(rel - 1, f, pv, pcoef);
          const int cc = f.child & 0xff;
          const bool handed = (f.child >> 8) != 0;
          D.undo_child(rel - 1, f, pv, pcoef, cc);
          key_set(key_lo, key_hi, depth0 + rel, 0, bpl, levels);
          if (!handed && cc + 1 < Eq2Tile<TILE, WE>::nchildren(f.k)) {
            lv = rel - 1;
            c = cc + 1;
            D.set_child(lv, c);
            __syncwarp();
            break;
          }
          --rel;
        }
        if (done) break;
      }
      if (!D.apply(lv, f, pv, c)) {
        if (lane == 0) atomicCAS(A.err, 0, WALK_FULL);
        break;
      }
      key_set(key_lo, key_hi, depth0 + lv + 1, (uint64_t)c, bpl, levels);
      rel = lv + 1;
    }
    // the subtree is done (or abandoned after an error): this warp is idle again
    __syncwarp();
    if (lane == 0) atomicAdd(A.outstanding, ~0ull);  // minus one
  }
  // flush this warp's count and the block's per-depth statistics
  if (lane == 0 && W.emitted) atomicAdd(A.emitted, W.emitted);
  __syncthreads();
  for (int k = threadIdx.x; k < A.hist_len; k += blockDim.x) {
    if (h_nodes[k]) atomicAdd(A.hist_nodes + k, (unsigned long long)h_nodes[k]);
    if (h_term[k]) atomicAdd(A.hist_term + k, (unsigned long long)h_term[k]);
    if (h_mo[k]) atomicMax(A.hist_maxopen + k, h_mo[k]);
  }
}

__global__ void k_walk_gather(const uint32_t* __restrict__ perm, int64_t n, JobArrays src, JobArrays dst) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  const uint32_t s = perm[i];
  dst.m[i] = src.m[s];
  dst.nnz[i] = src.nnz[s];
  dst.off[i] = src.off[s];
  dst.mat[i] = src.mat[s];
  dst.depth_left[i] = src.depth_left[s];
  for (int w = 0; w < 4; ++w) dst.coef[4 * i + w] = src.coef[4 * s + w];
}

__global__ void k_walk_keys(const uint64_t* __restrict__ key2, int64_t n, int word, uint64_t* __restrict__ out,
                            uint32_t* __restrict__ idx) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  out[i] = key2[2 * i + word];
  if (idx) idx[i] = (uint32_t)i;
}

__global__ void k_walk_keys_perm(const uint64_t* __restrict__ key2, const uint32_t* __restrict__ perm, int64_t n,
                                 int word, uint64_t* __restrict__ out) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  out[i] = key2[2 * perm[i] + word];
}

template <int TILE>
cudaError_t walk_blocks_per_sm(int stage_words, int hist_len, int* per_sm) {
  const size_t smem = walk_smem_bytes(TILE, stage_words, hist_len);
  cudaError_t e = cudaFuncSetAttribute(k_expand_walk<TILE>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, k_expand_walk<TILE>, WalkCfg<TILE>::WARPS * 32, smem);
}

template <int TILE>
cudaError_t launch_walk_tile(const WalkArgs& a, int sms, int* grid, cudaStream_t s) {
  int per_sm = 0;
  cudaError_t e = walk_blocks_per_sm<TILE>(a.stage_words, a.hist_len, &per_sm);
  if (e != cudaSuccess) return e;
  *grid = 0;
  // every block resident at once: a waiting warp never waits on a block that has not started
  const int g = sms * per_sm;
  if (per_sm < 1 || (int64_t)g * WalkCfg<TILE>::WARPS > a.warps_cap) return cudaSuccess;
  k_expand_walk<TILE><<<g, WalkCfg<TILE>::WARPS * 32, walk_smem_bytes(TILE, a.stage_words, a.hist_len), s>>>(a);
  e = cudaGetLastError();
  if (e == cudaSuccess) *grid = g;
  return e;
}

}  // namespace

int walk_tile_for(int max_order) { return max_order <= 32 ? 32 : (max_order <= 64 ? 64 : 0); }

size_t walk_smem_bytes(int tile, int stage_words, int hist_len) {
  const int warps = tile <= 32 ? WalkCfg<32>::WARPS : WalkCfg<64>::WARPS;
  return walk_warp_bytes(tile, stage_words) * warps + 3 * sizeof(int32_t) * (size_t)hist_len;
}

int64_t walk_frame_words(int tile) { return tile <= 32 ? TileCfg<32, WE>::FRAME_WORDS : TileCfg<64, WE>::FRAME_WORDS; }

cudaError_t walk_resident_warps(int tile, int stage_words, int hist_len, int sms, int64_t* warps) {
  int per_sm = 0;
  cudaError_t e = tile <= 32 ? walk_blocks_per_sm<32>(stage_words, hist_len, &per_sm)
                             : walk_blocks_per_sm<64>(stage_words, hist_len, &per_sm);
  *warps = (int64_t)sms * per_sm * (tile <= 32 ? WalkCfg<32>::WARPS : WalkCfg<64>::WARPS);
  return e;
}

cudaError_t launch_expand_walk(const WalkArgs& a, int tile, int sms, int* grid, cudaStream_t s) {
  *grid = 0;
  if (tile == 32) return launch_walk_tile<32>(a, sms, grid, s);
  if (tile == 64) return launch_walk_tile<64>(a, sms, grid, s);
  return cudaSuccess;
}

// perm = slots [0, n) in ascending key order; keys use bits [0, key_bits]
// (unused slots hold all ones, above every job's key)
cudaError_t launch_walk_order(const uint64_t* key2, int64_t n, int key_bits, uint64_t* kbuf, uint64_t* kbuf2,
                              uint32_t* ibuf, uint32_t* perm, void* tmp, size_t tmp_bytes, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  const unsigned g = (unsigned)((n + 255) / 256);
  const bool wide = key_bits >= 64;
  // least significant word first, then (stable) the most significant one
  k_walk_keys<<<g, 256, 0, s>>>(key2, n, 0, kbuf, ibuf);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  e = sort_asc_u64(kbuf, kbuf2, ibuf, perm, n, wide ? 64 : key_bits + 1, tmp, tmp_bytes, s);
  if (e != cudaSuccess || !wide) return e;
  k_walk_keys_perm<<<g, 256, 0, s>>>(key2, perm, n, 1, kbuf);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  e = cudaMemcpyAsync(ibuf, perm, 4 * (size_t)n, cudaMemcpyDeviceToDevice, s);
  if (e != cudaSuccess) return e;
  return sort_asc_u64(kbuf, kbuf2, ibuf, perm, n, key_bits + 1 - 64, tmp, tmp_bytes, s);
}

cudaError_t launch_walk_gather(const uint32_t* perm, int64_t n, const JobArrays& src, const JobArrays& dst,
                               cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  k_walk_gather<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(perm, n, src, dst);
  return cudaGetLastError();
}
