// K3: persistent evaluator.  Warps pull jobs from the ordered queue through
// one atomic counter (Algorithm PH, Step 3: the next job goes to the next
// free worker) and evaluate each by Algorithm H_per (Section 2.1): Eq. 2
// depth first while the order exceeds max(L, 2) and s < 5, Ryser /
// Nijenhuis-Wilf (ryser.cuh, ryser4.cuh) at the leaves.
//
// The job lives in a dense tile in shared memory.  Lines are never moved:
// deleting a row or column clears a bit of the active masks R and C, so
// "lowest index" keeps the meaning it has in the compacted matrices of the
// oracle.  A merge overwrites one line in place after saving it to the
// warp's undo stack in global memory; backtracking restores it.  Nonzero
// patterns are kept as bit masks per row (rowbits) and per column
// (colbits), so a line count is one popcount against the active masks.
//
// With the three-child option a node whose sparsest line has s >= 5
// nonzeros is not a leaf: Eq. 2's third child clears the pivot line's first
// four entries in place (the frame holds their values for the undo), so a
// path can hold more levels than the job has rows (max_depth frames).
//
// Variants: tile entries int32 (more warps per SM) or int64, and leaves of
// up to 16 or up to 32 rows.  A job that the narrow variant cannot hold (an
// entry leaving int32, a leaf above 16 rows) reports DFS_RETRY and the host
// runs it again on the int64 / 32-row variant.  On the residue path (W = 0)
// the entries are residues modulo a prime p and the leaves take the modular
// walk of ryser_mod.cuh.
#include <cuda_runtime.h>

#include <cstdint>

#include "dfs.cuh"
#include "internal.h"

namespace {

template <int TILE, typename E, int LN, int W>
__global__ void __launch_bounds__(DfsCfg<TILE, E>::WARPS * 32, DfsCfg<TILE, E>::MINB) k_dfs(DfsArgs A) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  typedef DfsCfg<TILE, E> Cfg;
  const int lane = threadIdx.x & 31;
  const int wib = threadIdx.x >> 5;
  unsigned char* base = smem_raw + (size_t)wib * Cfg::WARP_BYTES;
  Dfs<TILE, E, LN, W> D;
  D.T = reinterpret_cast<E*>(base);
  D.rowbits = reinterpret_cast<uint64_t*>(base + Cfg::TILE_BYTES);
  D.colbits = D.rowbits + TILE;
  D.delta = reinterpret_cast<int32_t*>(base + Cfg::TILE_BYTES + Cfg::MASK_BYTES);
  D.rho0 = D.delta + (PERM_MAX_LEAF - 1) * 32;
  D.cmask = reinterpret_cast<uint32_t*>(D.rho0 + 32);
  const int64_t gwarp = (int64_t)blockIdx.x * Cfg::WARPS + wib;
  D.undo = A.undo + gwarp * A.undo_words_per_warp;
  D.lane = lane;
  D.mod = A.mod;
  D.modp = A.mod.p;
  const int cut = A.leaf_size > 2 ? A.leaf_size : 2;

  for (;;) {
    unsigned long long qi = 0;
    if (lane == 0) qi = atomicAdd(A.job_counter, 1ull);
    qi = __shfl_sync(0xffffffffu, qi, 0);
    if (qi >= (unsigned long long)A.nq) break;
    dfs_job<TILE, E, LN, W>(D, A, A.queue[qi], cut);
  }
}

template <int TILE, typename E, int LN, int W>
cudaError_t launch_dfs_variant(const DfsArgs& a, int num_sms, int warps_per_sm, cudaStream_t s) {
  typedef DfsCfg<TILE, E> C;
  static bool attr_set = false;
  if (!attr_set) {
    cudaError_t e =
        cudaFuncSetAttribute(k_dfs<TILE, E, LN, W>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::SMEM);
    if (e != cudaSuccess) return e;
    attr_set = true;
  }
  int per_sm = 0;
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_dfs<TILE, E, LN, W>, C::WARPS * 32, C::SMEM);
  if (e != cudaSuccess) return e;
  int blocks_per_sm = (warps_per_sm + C::WARPS - 1) / C::WARPS;
  if (blocks_per_sm > per_sm) blocks_per_sm = per_sm;
  if (blocks_per_sm < 1) blocks_per_sm = 1;
  k_dfs<TILE, E, LN, W><<<num_sms * blocks_per_sm, C::WARPS * 32, C::SMEM, s>>>(a);
  return cudaGetLastError();
}

}  // namespace

int dfs_warps_per_block(int tile, bool wide) {
  if (wide) return tile <= 32 ? DfsCfg<32, int64_t>::WARPS : DfsCfg<64, int64_t>::WARPS;
  return tile <= 32 ? DfsCfg<32, int32_t>::WARPS : DfsCfg<64, int32_t>::WARPS;
}
int64_t dfs_undo_words(int tile, int frames) {
  return (int64_t)frames * (tile <= 32 ? DfsCfg<32, int32_t>::FRAME_WORDS : DfsCfg<64, int32_t>::FRAME_WORDS);
}

template <int W>
cudaError_t launch_dfs_w(const DfsArgs& a, int tile, bool wide, int num_sms, int warps_per_sm, cudaStream_t s) {
  if (wide) {
    if (tile <= 32) return launch_dfs_variant<32, int64_t, 32, W>(a, num_sms, warps_per_sm, s);
    return launch_dfs_variant<64, int64_t, 32, W>(a, num_sms, warps_per_sm, s);
  }
  if (tile <= 32) return launch_dfs_variant<32, int32_t, 16, W>(a, num_sms, warps_per_sm, s);
  return launch_dfs_variant<64, int32_t, 16, W>(a, num_sms, warps_per_sm, s);
}

cudaError_t launch_dfs(const DfsArgs& a, int tile, bool wide, int W, int num_sms, int warps_per_sm, cudaStream_t s) {
  if (a.nq <= 0) return cudaSuccess;
  if (a.mod.p) return launch_dfs_w<0>(a, tile, wide, num_sms, warps_per_sm, s);
  if (W == 2) return launch_dfs_w<2>(a, tile, wide, num_sms, warps_per_sm, s);
  return launch_dfs_w<4>(a, tile, wide, num_sms, warps_per_sm, s);
}
