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
constexpr int kCheckEvery = 16;  // nodes between looks at the error flag and the waiting warps

template <int TILE>
struct WalkCfg {
  static constexpr int WARPS = TILE <= 32 ? 8 : 4;  // warps per block
  static constexpr size_t WARP_BYTES = TileCfg<TILE, WE>::TILE_BYTES + TileCfg<TILE, WE>::MASK_BYTES;
};

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
__device__ int64_t compact_tile(const WalkArgs& A, WarpCtx& W, const Eq2Tile<TILE, WE>& D, int& m_out,
                                int& nnz_out) {
  constexpr int S = TileCfg<TILE, WE>::STRIDE;
  constexpr int RPL = TILE / 32;
  const int lane = W.lane;
  const int m = __popcll(D.R);
  int cnt[RPL], row[RPL];
#pragma unroll
  for (int t = 0; t < RPL; ++t) {
    const int k = lane + 32 * t;
    row[t] = k < m ? nth_bit(D.R, k) : 0;
    cnt[t] = k < m ? __popcll(D.rowbits[row[t]] & D.C) : 0;
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
  if (o < 0) return -1;
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
      uint64_t cm = D.rowbits[r] & D.C;
      int w = offs[t];
      while (cm) {
        const int c = __ffsll((long long)cm) - 1;
        cm &= cm - 1;
        colp[w] = (uint8_t)__popcll(D.C & (bit64(c) - 1));
        valp[w] = (int64_t)D.T[r * S + c];
        ++w;
      }
    }
  }
  return o;
}

// Write a job's header and path key; its block is at off.
__device__ void walk_emit(const WalkArgs& A, WarpCtx& W, int m, int nnz, int64_t off, int mat, int depth,
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

// Hand a node (block at off, written by this warp) to the global queue.
__device__ void walk_push(const WalkArgs& A, int lane, int m, int nnz, int64_t off, int mat, int dl, int depth,
                          const u256& coef, uint64_t key_lo, uint64_t key_hi) {
  __syncwarp();
  __threadfence();  // every lane's part of the block before the slot is published
  __syncwarp();
  if (lane == 0) {
    atomicAdd(A.outstanding, 1ull);
    const unsigned long long t = atomicAdd(A.q_tail, 1ull);
    if ((int64_t)t >= A.cap_q) {
      atomicCAS(A.err, 0, WALK_FULL);
    } else {
      A.q_m[t] = m;
      A.q_nnz[t] = nnz;
      A.q_mat[t] = mat;
      A.q_dl[t] = dl;
      A.q_depth[t] = depth;
      A.q_off[t] = off;
      for (int w = 0; w < 4; ++w) A.q_coef[4 * t + w] = coef.w[w];
      A.q_key[2 * t] = key_lo;
      A.q_key[2 * t + 1] = key_hi;
      __threadfence();
      *(volatile int32_t*)(A.q_ready + t) = 1;
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
__global__ void __launch_bounds__(WalkCfg<TILE>::WARPS * 32) k_expand_walk(WalkArgs A) {
  constexpr int S = TileCfg<TILE, WE>::STRIDE;
  constexpr int NW = WalkCfg<TILE>::WARPS;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int lane = threadIdx.x & 31;
  const int wib = threadIdx.x >> 5;
  unsigned char* base = smem_raw + (size_t)wib * WalkCfg<TILE>::WARP_BYTES;
  Eq2Tile<TILE, WE> D;
  D.T = reinterpret_cast<WE*>(base);
  D.rowbits = reinterpret_cast<uint64_t*>(base + TileCfg<TILE, WE>::TILE_BYTES);
  D.colbits = D.rowbits + TILE;
  D.lane = lane;
  const int64_t gwarp = (int64_t)blockIdx.x * NW + wib;
  D.undo = A.undo + gwarp * A.undo_words_per_warp;
  unsigned* h_nodes = reinterpret_cast<unsigned*>(smem_raw + (size_t)NW * WalkCfg<TILE>::WARP_BYTES);
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
  bool waiting = true;  // other warps wait for work (looked up every kCheckEvery nodes, or while true)

  for (;;) {
    // ---- a subtree root from the global queue
    unsigned long long ticket = 0;
    if (lane == 0) ticket = atomicAdd(A.q_head, 1ull);
    ticket = __shfl_sync(0xffffffffu, ticket, 0);
    int got = 0;
    if (lane == 0) {
      for (unsigned spins = 0;; ++spins) {
        if ((int64_t)ticket < A.cap_q && volatile_ld(A.q_ready + ticket) != 0) {
          got = 1;
          break;
        }
        if ((long long)volatile_ld(A.outstanding) <= 0 || volatile_ld(A.err) != 0) break;
        if ((spins & 63u) == 63u && globaltimer_ns() - t_start > (uint64_t)A.timeout_ns) {
          atomicCAS(A.err, 0, PERM_ETIMEOUT);
          break;
        }
        __nanosleep(128);
      }
      __threadfence();
    }
    got = __shfl_sync(0xffffffffu, got, 0);
    if (!got) break;
    __threadfence();
    const int64_t t = (int64_t)ticket;
    const int m0 = __ldcg(A.q_m + t), nnz0 = __ldcg(A.q_nnz + t), mat = __ldcg(A.q_mat + t);
    const int dl0 = __ldcg(A.q_dl + t), depth0 = __ldcg(A.q_depth + t);
    const int64_t off0 = __ldcg(A.q_off + t);
    for (int w = 0; w < 4; ++w) D.coef.w[w] = __ldcg(A.q_coef + 4 * t + w);
    uint64_t key_lo = __ldcg(A.q_key + 2 * t), key_hi = __ldcg(A.q_key + 2 * t + 1);
    bool stop = m0 > TILE;
    // ---- the node into the tile
    for (int k = lane; k < TILE * S; k += 32) D.T[k] = 0;
    for (int k = lane; k < TILE; k += 32) D.rowbits[k] = D.colbits[k] = 0;
    __syncwarp();
    const uint64_t* blk = A.arena + off0;
    const int rpw = (int)blk_rp_words(m0), cw = (int)blk_col_words(nnz0);
    bool fits = true;
    for (int r = lane; r < m0 && !stop; r += 32) {
      const int b = (int)((blk_word(blk, r / 4) >> (16 * (r % 4))) & 0xffff);
      const int e = (int)((blk_word(blk, (r + 1) / 4) >> (16 * ((r + 1) % 4))) & 0xffff);
      uint64_t rb = 0;
      for (int q = b; q < e; ++q) {
        const int c = (int)((blk_word(blk, rpw + q / 8) >> (8 * (q % 8))) & 0xff);
        const int64_t x = (int64_t)blk_word(blk, rpw + cw + q);
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
    // ---- depth-first walk of the subtree: rel = depth of the current node below its root
    int rel = 0;
    bool done = stop;
    while (!done) {
      const int depth = depth0 + rel;
      if (++since_check >= kCheckEvery || waiting) {
        since_check = 0;
        int e = 0, wt = 0;
        if (lane == 0) {
          e = volatile_ld(A.err);
          wt = volatile_ld(A.q_head) > volatile_ld(A.q_tail) ? 1 : 0;
        }
        if (__shfl_sync(0xffffffffu, e, 0) != 0) break;  // another warp failed: abandon the walk
        waiting = __shfl_sync(0xffffffffu, wt, 0) != 0;
      }
      if (lane == 0 && depth < A.hist_len) atomicAdd(h_nodes + depth, 1u);
      const unsigned long long key = D.pivot_key();
      const int s = (int)(key >> 17);
      const int mact = __popcll(D.R);
      const int dl = dl0 - rel;
      const bool open = dl > 0 && mact > cut;
      if (open && lane == 0 && depth < A.hist_len) atomicMax(h_mo + depth, mact);
      bool descend = false;
      if (s > 0 && (!open || (s >= 5 && !three))) {
        // a job
        int mj, nj;
        const int64_t o = compact_tile<TILE>(A, W, D, mj, nj);
        if (o >= 0) walk_emit(A, W, mj, nj, o, mat, depth, D.coef, key_lo, key_hi, h_term);
      } else if (s > 0) {
        if (rel >= A.max_rel_depth) {
          if (lane == 0) atomicCAS(A.err, 0, WALK_FULL);
          break;
        }
        Frame f;
        f.is_col = (int)((key >> 16) & 1);
        f.idx = (int)(key & 0xffff);
        f.k = s;
        f.child = 0;
        int64_t pv[4] = {0, 0, 0, 0};
        uint64_t line = f.is_col ? (D.colbits[f.idx] & D.R) : (D.rowbits[f.idx] & D.C);
        for (int q = 0; q < 4; ++q) {
          if (line) {
            const int c = __ffsll((long long)line) - 1;
            line &= line - 1;
            f.pos[q] = c;
            pv[q] = (int64_t)(f.is_col ? D.T[c * S + f.idx] : D.T[f.idx * S + c]);
          } else {
            f.pos[q] = 0;
          }
        }
        const int nch = Eq2Tile<TILE, WE>::nchildren(s);
        const u256 pcoef = D.coef;
        D.store_frame(rel, f, pv, pcoef);
        __syncwarp();
        bool failed = false;
        if (waiting && nch > 1) {
          // hand the other children to the waiting warps, go on with child 0
          for (int c = 1; c < nch && !failed; ++c) {
            if (!D.apply(rel, f, pv, c)) {
              failed = true;
            } else {
              int mj, nj;
              const int64_t o = compact_tile<TILE>(A, W, D, mj, nj);
              uint64_t klo = key_lo, khi = key_hi;
              key_set(klo, khi, depth + 1, (uint64_t)c, bpl, levels);
              if (o >= 0) walk_push(A, lane, mj, nj, o, mat, dl - 1, depth + 1, D.coef, klo, khi);
            }
            D.undo_child(rel, f, pv, pcoef, c);
          }
          D.set_child(rel, 1 << 8);  // child 0, the others handed over
          __syncwarp();
        }
        if (failed || !D.apply(rel, f, pv, 0)) {
          if (lane == 0) atomicCAS(A.err, 0, WALK_FULL);
          break;
        }
        key_set(key_lo, key_hi, depth + 1, 0, bpl, levels);
        ++rel;
        descend = true;
      }
      if (descend) continue;
      // ---- back up to the next child not yet walked
      for (;;) {
        if (rel == 0) {
          done = true;
          break;
        }
        Frame f;
        int64_t pv[4];
        u256 pc;
        D.load_frame(rel - 1, f, pv, pc);
        const int c = f.child & 0xff;
        const bool handed = (f.child >> 8) != 0;
        D.undo_child(rel - 1, f, pv, pc, c);
        if (!handed && c + 1 < Eq2Tile<TILE, WE>::nchildren(f.k)) {
          D.set_child(rel - 1, c + 1);
          __syncwarp();
          if (!D.apply(rel - 1, f, pv, c + 1)) {
            if (lane == 0) atomicCAS(A.err, 0, WALK_FULL);
            done = true;
          }
          key_set(key_lo, key_hi, depth0 + rel, (uint64_t)(c + 1), bpl, levels);
          break;
        }
        key_set(key_lo, key_hi, depth0 + rel, 0, bpl, levels);
        --rel;
      }
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
cudaError_t walk_blocks_per_sm(int hist_len, int* per_sm) {
  const size_t smem = walk_smem_bytes(TILE, hist_len);
  cudaError_t e = cudaFuncSetAttribute(k_expand_walk<TILE>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, k_expand_walk<TILE>, WalkCfg<TILE>::WARPS * 32, smem);
}

template <int TILE>
cudaError_t launch_walk_tile(const WalkArgs& a, int sms, int* grid, cudaStream_t s) {
  int per_sm = 0;
  cudaError_t e = walk_blocks_per_sm<TILE>(a.hist_len, &per_sm);
  if (e != cudaSuccess) return e;
  *grid = 0;
  // every block resident at once: a waiting warp never waits on a block that has not started
  const int g = sms * per_sm;
  if (per_sm < 1 || (int64_t)g * WalkCfg<TILE>::WARPS > a.warps_cap) return cudaSuccess;
  k_expand_walk<TILE><<<g, WalkCfg<TILE>::WARPS * 32, walk_smem_bytes(TILE, a.hist_len), s>>>(a);
  e = cudaGetLastError();
  if (e == cudaSuccess) *grid = g;
  return e;
}

}  // namespace

int walk_tile_for(int max_order) { return max_order <= 32 ? 32 : (max_order <= 64 ? 64 : 0); }

size_t walk_smem_bytes(int tile, int hist_len) {
  const size_t warp = tile <= 32 ? WalkCfg<32>::WARP_BYTES : WalkCfg<64>::WARP_BYTES;
  const int warps = tile <= 32 ? WalkCfg<32>::WARPS : WalkCfg<64>::WARPS;
  return warp * warps + 3 * sizeof(int32_t) * (size_t)hist_len;
}

int64_t walk_frame_words(int tile) { return tile <= 32 ? TileCfg<32, WE>::FRAME_WORDS : TileCfg<64, WE>::FRAME_WORDS; }

cudaError_t walk_resident_warps(int tile, int hist_len, int sms, int64_t* warps) {
  int per_sm = 0;
  cudaError_t e = tile <= 32 ? walk_blocks_per_sm<32>(hist_len, &per_sm) : walk_blocks_per_sm<64>(hist_len, &per_sm);
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
