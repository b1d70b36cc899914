// The whole evaluation in one persistent launch (Algorithm PH, Step 3 as
// list scheduling over one queue): warps take queue positions in queue
// order through one atomic counter, so the order the queue was sorted in
// (natural, KKLLL-LPT or learned) holds across every job, and each job runs
// its own evaluator as a device function:
//  - a leaf job (order <= the leaf order) its Ryser / Nijenhuis-Wilf variant
//    (leaf.cuh), split into tasks of 32 lanes x 2^c Gray codes; the warp that
//    takes a job of more than one task posts it on a board, and a warp that
//    finds the board set takes tasks of that job (one atomic per task) before
//    it takes a new queue position, so a large job is spread over many warps
//    as in the per-variant kernels; the warp that finishes a job's last task
//    forms coef * per and adds it into the job's matrix (Step 4);
//  - any other job of order <= 32 the depth-first walk of Algorithm H_per
//    (dfs.cuh) on a 32-wide tile: int64 entries and leaves of up to 32 rows,
//    or (the narrow form) int32 entries and leaves of up to 16 rows, where a
//    job that needs more raises a flag and is run again on the wide kernel.
// Jobs of order above 32 that are not leaves run in the depth-first launch
// before this one.  No warp ever waits on another: helping is opportunistic,
// and every job's tasks are finished by the warp that took it if nobody helps.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>
#include <type_traits>

#include "dfs.cuh"
#include "internal.h"
#include "leaf.cuh"

namespace {


constexpr int kPersistWarps = 8;
// per warp: the 32-wide tile (int32 entries and leaves up to 16 rows when
// NARROW, else int64 and up to 32) and its masks, then the leaf columns
// (delta, rho0, column masks), shared by the leaf tasks and the depth-first leaves
template <bool NARROW>
struct PersistCfg {
  typedef typename std::conditional<NARROW, int32_t, int64_t>::type E;
  static constexpr int LN = NARROW ? 16 : 32;
  typedef DfsCfg<32, E> TC;
  static constexpr size_t LEAF_BYTES = sizeof(int32_t) * ((PERM_MAX_LEAF - 1) * 32 + 32 + 32);
  static constexpr size_t WARP_BYTES = TC::TILE_BYTES + TC::MASK_BYTES + LEAF_BYTES;
  static constexpr size_t SMEM = WARP_BYTES * kPersistWarps;
};

// one leaf task of variant (NMAX, PATH): the job loaded first when `load`
template <int NMAX, int W, int PATH>
__device__ __noinline__ void leaf_unit(const uint64_t* __restrict__ arena, int64_t off, int m, int nnz, bool load,
                                       uint64_t lt, int chunk_log2, int32_t* delta, int32_t* rho0, int32_t* colcnt,
                                       int lane, ModP mod, uint64_t* words) {
  if (load && m >= 2) leaf_load<NMAX, PATH>(arena, off, m, nnz, delta, rho0, colcnt, lane, mod);
  leaf_task<NMAX, W, PATH>(arena, off, m, nnz, lt, chunk_log2, delta, rho0, lane, mod, words);
}

template <int W, int NMAX>
__device__ __forceinline__ void leaf_unit_path(int path, const uint64_t* arena, int64_t off, int m, int nnz, bool load,
                                               uint64_t lt, int chunk_log2, int32_t* delta, int32_t* rho0,
                                               int32_t* colcnt, int lane, const ModP& mod, uint64_t* words) {
#define LEAF_UNIT_ARGS arena, off, m, nnz, load, lt, chunk_log2, delta, rho0, colcnt, lane, mod, words
  if constexpr (W == 0) {
    leaf_unit<NMAX, 2, P_MOD>(LEAF_UNIT_ARGS);
  } else {
    switch (path) {
      case P_G7: leaf_unit<NMAX, W, P_G7>(LEAF_UNIT_ARGS); break;
      case P_G15: leaf_unit<NMAX, W, P_G15>(LEAF_UNIT_ARGS); break;
      case P_G31: leaf_unit<NMAX, W, P_G31>(LEAF_UNIT_ARGS); break;
      case P_F8: leaf_unit<NMAX, W, P_F8>(LEAF_UNIT_ARGS); break;
      case P_F4: leaf_unit<NMAX, W, P_F4>(LEAF_UNIT_ARGS); break;
      default:
        if constexpr (NMAX >= 16) leaf_unit<NMAX, W, P_F16>(LEAF_UNIT_ARGS);
        break;
    }
  }
#undef LEAF_UNIT_ARGS
}

// variant key: nmax index | W bit | path << 3 (the W bit is ignored: the
// kernel's ring is at least as wide)
template <int W>
__device__ __forceinline__ void leaf_unit_key(int key, const uint64_t* arena, int64_t off, int m, int nnz, bool load,
                                              uint64_t lt, int chunk_log2, int32_t* delta, int32_t* rho0,
                                              int32_t* colcnt, int lane, const ModP& mod, uint64_t* words) {
  const int path = key >> 3;
  switch (key & 3) {
    case 0: leaf_unit_path<W, 8>(path, arena, off, m, nnz, load, lt, chunk_log2, delta, rho0, colcnt, lane, mod, words); break;
    case 1: leaf_unit_path<W, 16>(path, arena, off, m, nnz, load, lt, chunk_log2, delta, rho0, colcnt, lane, mod, words); break;
    case 2: leaf_unit_path<W, 24>(path, arena, off, m, nnz, load, lt, chunk_log2, delta, rho0, colcnt, lane, mod, words); break;
    default: leaf_unit_path<W, 32>(path, arena, off, m, nnz, load, lt, chunk_log2, delta, rho0, colcnt, lane, mod, words); break;
  }
}

// A warp's running sum of the leaf jobs it closed for one matrix (lane 0):
// added into the matrix accumulator when the matrix changes and at the end,
// so jobs of one matrix taken one after another cost one atomic sum.
struct MatSum {
  int mat = -1;
  u256 v;
  __device__ void flush(unsigned long long* mat_acc) {
    if (mat >= 0) atomic_add_words(mat_acc + 4ll * mat, v.w, 4);
    mat = -1;
  }
  __device__ void add(unsigned long long* mat_acc, int m2, const u256& x) {
    if (m2 != mat) {
      flush(mat_acc);
      mat = m2;
      v = x;
    } else {
      v = u256_add(v, x);
    }
  }
};

// coef * per of a finished leaf job into out.acc and the warp's matrix sum (lane 0)
__device__ __forceinline__ void leaf_close(const PersistArgs& A, uint32_t job, int m, const uint64_t* sigma,
                                           MatSum& ms) {
  const u256 v = leaf_finish(sigma, m, A.dfs.jobs.coef + 4ll * job, A.dfs.mod.p);
  for (int k = 0; k < 4; ++k) A.dfs.out.acc[4ll * job + k] = v.w[k];
  A.dfs.out.nodes[job] = 1;
  ms.add(A.dfs.mat_acc, A.dfs.jobs.mat[job], v);
}

// Take tasks of the leaf job at queue position q until none is left
// (sole: a one-task job this warp took from the queue, which no other warp
// can reach, so its task needs no counter).
template <int W>
__device__ __forceinline__ void leaf_tasks(const PersistArgs& A, int64_t q, int lane, int32_t* delta, int32_t* rho0,
                                           int32_t* colcnt, MatSum& ms, bool sole) {
  const uint32_t job = A.queue[q];
  const int key = (int)A.keys[q];
  const JobArrays& J = A.dfs.jobs;
  const int m = J.m[job];
  const int nnz = J.nnz[job];
  const int64_t off = J.off[job];
  const uint64_t T = leaf_tasks_dev(m, A.chunk_log2);
  const JobOut& out = A.dfs.out;
  if ((key >> 3) == P_BAD) {  // a row sum beyond the exact leaf's range
    unsigned t = 0;
    if (lane == 0 && !sole) t = atomicAdd(A.task_next + q, 1u);
    t = __shfl_sync(0xffffffffu, t, 0);
    if (lane == 0 && t == 0) out.status[job] = PERM_EOVERFLOW;
    return;
  }
  bool loaded = false;
  for (int it = 0;; ++it) {
    unsigned t = 0;
    if (sole) {
      if (it > 0) break;
    } else {
      if (lane == 0) t = atomicAdd(A.task_next + q, 1u);
      t = __shfl_sync(0xffffffffu, t, 0);
      if ((uint64_t)t >= T) break;
    }
    const uint64_t t0 = globaltimer_ns();
    uint64_t words[4];
    leaf_unit_key<W>(key, A.dfs.arena, off, m, nnz, !loaded, t, A.chunk_log2, delta, rho0, colcnt, lane, A.dfs.mod,
                     words);
    loaded = true;
    if (lane == 0) {
      const uint64_t t1 = globaltimer_ns();
      if (t == 0) out.leaves[job] = 1;
      if (T == 1) {  // the whole job in this warp: plain stores
        out.t_start[job] = t0;
        out.t_end[job] = t1;
        out.sm[job] = (int32_t)smid();
        leaf_close(A, job, m, words, ms);
      } else {
        atomic_add_words(out.acc + 4ll * job, words, 4);
        const unsigned long long prev = atomicMin(out.t_start + job, (unsigned long long)t0);
        if (prev == ~0ull) out.sm[job] = (int32_t)smid();
        atomicMax(out.t_end + job, (unsigned long long)t1);
        __threadfence();  // this task's words before its completion count
        if (atomicAdd(A.task_done + q, 1u) == (unsigned)(T - 1)) {
          __threadfence();
          uint64_t sig[4];
          for (int k = 0; k < 4; ++k) sig[k] = __ldcg(reinterpret_cast<const uint64_t*>(out.acc) + 4ll * job + k);
          leaf_close(A, job, m, sig, ms);
        }
      }
    }
    __syncwarp();
  }
}

template <int W, bool NARROW>
__global__ void __launch_bounds__(kPersistWarps * 32, 2) k_eval_persist(PersistArgs A) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  typedef PersistCfg<NARROW> PC;
  typedef typename PC::E E;
  const int lane = threadIdx.x & 31;
  const int wib = threadIdx.x >> 5;
  unsigned char* base = smem_raw + (size_t)wib * PC::WARP_BYTES;
  Dfs<32, E, PC::LN, W> D;
  D.T = reinterpret_cast<E*>(base);
  D.rowbits = reinterpret_cast<uint64_t*>(base + PC::TC::TILE_BYTES);
  D.colbits = D.rowbits + 32;
  D.delta = reinterpret_cast<int32_t*>(base + PC::TC::TILE_BYTES + PC::TC::MASK_BYTES);
  D.rho0 = D.delta + (PERM_MAX_LEAF - 1) * 32;
  D.cmask = reinterpret_cast<uint32_t*>(D.rho0 + 32);
  const int64_t gwarp = (int64_t)blockIdx.x * kPersistWarps + wib;
  D.undo = A.dfs.undo + gwarp * A.dfs.undo_words_per_warp;
  D.lane = lane;
  D.mod = A.dfs.mod;
  D.modp = A.dfs.mod.p;
  const int cut = A.dfs.leaf_size > 2 ? A.dfs.leaf_size : 2;
  int32_t* colcnt = reinterpret_cast<int32_t*>(D.cmask);
  MatSum ms;
  for (;;) {
    // a posted leaf job with tasks left comes first
    long long b = -1;
    if (lane == 0) b = *(volatile long long*)A.board;
    b = __shfl_sync(0xffffffffu, b, 0);
    if (b >= 0) {
      leaf_tasks<W>(A, b, lane, D.delta, D.rho0, colcnt, ms, false);
      if (lane == 0) atomicCAS(reinterpret_cast<unsigned long long*>(A.board), (unsigned long long)b, ~0ull);
      __syncwarp();
      continue;
    }
    unsigned long long qi = 0;
    if (lane == 0) qi = atomicAdd(A.qctr, 1ull);
    qi = __shfl_sync(0xffffffffu, qi, 0);
    if (qi >= (unsigned long long)A.nq) break;
    const int64_t q = (int64_t)qi;
    const uint32_t key = A.keys[q];
    if (key < EVAL_KEY_DFS) {
      const bool many = leaf_tasks_dev(A.dfs.jobs.m[A.queue[q]], A.chunk_log2) > 1;
      if (lane == 0 && many) atomicExch(reinterpret_cast<unsigned long long*>(A.board), (unsigned long long)q);
      __syncwarp();
      leaf_tasks<W>(A, q, lane, D.delta, D.rho0, colcnt, ms, !many);
    } else if (A.dfs.jobs.m[A.queue[q]] <= 32) {
      dfs_job<32, E, PC::LN, W>(D, A.dfs, A.queue[q], cut);
    }
    // else: a depth-first job of order above 32, evaluated by the launch before this one
  }
  if (lane == 0) ms.flush(A.dfs.mat_acc);
}

template <int W, bool NARROW>
cudaError_t blocks_per_sm(int* per_sm) {
  typedef PersistCfg<NARROW> PC;
  static int cached = 0;
  if (cached == 0) {
    cudaError_t e = cudaFuncSetAttribute(k_eval_persist<W, NARROW>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)PC::SMEM);
    if (e != cudaSuccess) return e;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&cached, k_eval_persist<W, NARROW>, kPersistWarps * 32,
                                                      PC::SMEM);
    if (e != cudaSuccess) return e;
    if (cached < 1) cached = 1;
  }
  *per_sm = cached;
  return cudaSuccess;
}

template <int W, bool NARROW>
cudaError_t launch_w(const PersistArgs& a, int sms, cudaStream_t s) {
  int per_sm = 0;
  cudaError_t e = blocks_per_sm<W, NARROW>(&per_sm);
  if (e != cudaSuccess) return e;
  k_eval_persist<W, NARROW><<<sms * per_sm, kPersistWarps * 32, PersistCfg<NARROW>::SMEM, s>>>(a);
  return cudaGetLastError();
}

// resident warps and the launch for one tile form
template <bool NARROW>
cudaError_t persist_warps_t(int W, int sms, int64_t* warps) {
  int per_sm = 0;
  cudaError_t e = W == 0 ? blocks_per_sm<0, NARROW>(&per_sm)
                         : (W == 2 ? blocks_per_sm<2, NARROW>(&per_sm) : blocks_per_sm<4, NARROW>(&per_sm));
  *warps = (int64_t)sms * per_sm * kPersistWarps;
  return e;
}
template <bool NARROW>
cudaError_t launch_persist_t(const PersistArgs& a, int W, int sms, cudaStream_t s) {
  if (a.nq <= 0) return cudaSuccess;
  if (W == 0) return launch_w<0, NARROW>(a, sms, s);
  if (W == 2) return launch_w<2, NARROW>(a, sms, s);
  return launch_w<4, NARROW>(a, sms, s);
}

}  // namespace
