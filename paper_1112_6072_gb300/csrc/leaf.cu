// K2: batched leaf evaluation by Ryser / Nijenhuis-Wilf (Section 1) for jobs
// whose order is at most the leaf order.  The 2^(m-1) Gray codes of a job
// are cut into tasks of 32 lanes x 2^c codes; a persistent grid of warps
// pulls tasks through one atomic counter in queue order (the job order set
// by the LPT / learned ordering), so big jobs queued first are spread over
// many warps and small jobs fill the tail.
//
// A classification pass gives every job its variant: register width NMAX
// (8/16/24/32 rows), ring width W (2 or 4 words) and path -- the blocked
// walk of ryser4.cuh with 8 or 16 "N" slots when the row sums fit 7 bits
// and the two sparsest columns touch at most 16 rows (the 8 slots split
// 4 + 4 when the sparser column touches at most 4), else the plain walk
// of ryser.cuh with the 7-, 15- or 31-bit product tree.  On the residue
// path every leaf takes the modular walk of ryser_mod.cuh.  Each variant is
// its own kernel, so each gets the registers it needs and no more.
#include <cuda_runtime.h>

#include <cstdint>

#include "internal.h"
#include "jobs.cuh"
#include "leaf.cuh"

namespace {

constexpr int LEAF_WARPS = 8;  // warps per block

struct LeafSmem {
  int32_t delta[LEAF_WARPS][(PERM_MAX_LEAF - 1) * 32];
  int32_t rho0[LEAF_WARPS][32];
  int32_t colcnt[LEAF_WARPS][32];
};

// owner[t] = the grouped leaf queue position whose job holds task t
__global__ void k_task_owner(const uint64_t* __restrict__ prefix, int64_t nq, uint32_t* __restrict__ owner) {
  const int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (q >= nq) return;
  for (uint64_t t = prefix[q]; t < prefix[q + 1]; ++t) owner[t] = (uint32_t)q;
}

__global__ void k_leaf_task_counts(const uint32_t* __restrict__ queue, int64_t nq,
                                   const int32_t* __restrict__ jm, int chunk_log2,
                                   uint64_t* __restrict__ counts) {
  int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (q > nq) return;
  if (q == nq) {  // one trailing zero so the exclusive scan yields the total
    counts[q] = 0;
    return;
  }
  int m = jm[queue[q]];
  uint64_t tasks = 1;
  if (m >= 2) {
    int lanes, clog;
    leaf_split(m, chunk_log2, lanes, clog, tasks);
  }
  counts[q] = tasks;
}

// Kernel variant of a leaf job: nmax index | W (4 -> bit 2) | path << 3.
__device__ int leaf_class(uint32_t job, const JobArrays& jobs, const uint64_t* __restrict__ arena,
                          const int32_t* __restrict__ mat_w, bool modular) {
  const int m = jobs.m[job];
  if (modular) return (m <= 8 ? 0 : (m <= 16 ? 1 : (m <= 24 ? 2 : 3))) | (P_MOD << 3);
  const int nnz = jobs.nnz[job];
  CsrView v = csr_view(arena, jobs.off[job], m, nnz);
  uint32_t cm[PERM_MAX_LEAF];  // rows holding a nonzero, per column
  for (int j = 0; j < PERM_MAX_LEAF; ++j) cm[j] = 0;
  int64_t rmax = 0;
  bool ok = m <= PERM_MAX_LEAF;
  for (int r = 0; r < m && ok; ++r) {
    int64_t ra = 0;
    for (int p = v.rowptr[r]; p < v.rowptr[r + 1]; ++p) {
      const int64_t a = v.val[p];
      if (a >= (1ll << 30) || a <= -(1ll << 30)) ok = false;
      ra += a < 0 ? -a : a;
      cm[v.col[p]] |= 1u << r;
    }
    if (ra >= (1ll << 31)) ok = false;
    rmax = ra > rmax ? ra : rmax;
  }
  const int nmi = m <= 8 ? 0 : (m <= 16 ? 1 : (m <= 24 ? 2 : 3));
  const int W = mat_w[jobs.mat[job]];
  int path = P_BAD;
  if (ok) {
    const int bc = bit_class(rmax);
    path = bc == 7 ? P_G7 : (bc == 15 ? P_G15 : P_G31);
    if (bc == 7 && m >= 3) {
      // the column pair for the blocked walk: a pair for the 4 + 4 split
      // (union within 8 rows, one column within 4) if there is one, else the
      // pair touching the fewest rows; fewest rows, then lowest pair, on ties
      // (the same rule as load_blocked)
      unsigned best = 0xffffffffu;
      for (int a = 0; a < m; ++a)
        for (int b = a + 1; b < m; ++b) {
          const unsigned u = (unsigned)__popc(cm[a] | cm[b]);
          const bool split = u <= 8 && min(__popc(cm[a]), __popc(cm[b])) <= 4;
          const unsigned kk = ((split ? 0u : 1u) << 24) | (u << 16) | ((unsigned)a << 8) | (unsigned)b;
          best = kk < best ? kk : best;
        }
      const int k = (int)((best >> 16) & 0xff), pa = (int)((best >> 8) & 0xff), pb = (int)(best & 0xff);
      // 16 N slots: one of the two columns must fit the first 8; 4 + 4 split:
      // the smaller column within the first 4
      if (k <= 8) path = min(__popc(cm[pa]), __popc(cm[pb])) <= 4 ? P_F4 : P_F8;
      else if (k <= 16 && m > 8 && min(__popc(cm[pa]), __popc(cm[pb])) <= 8) path = P_F16;
    }
  }
  return nmi | ((W == 4) ? 4 : 0) | (path << 3);
}

// One thread per queue position: the sort key of its job -- the leaf
// variant (< 64) for jobs of order <= leaf_max, else the depth-first group
// EVAL_KEY_DFS + 2 * (order <= 32) + (W == 4) -- and a histogram of the keys.
__global__ void k_eval_keys(const uint32_t* __restrict__ queue, int64_t n, JobArrays jobs,
                            const uint64_t* __restrict__ arena, const int32_t* __restrict__ mat_w, int leaf_max,
                            bool modular, uint32_t* __restrict__ keys, uint32_t* __restrict__ vals,
                            unsigned long long* __restrict__ hist) {
  const int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const bool act = q < n;
  uint32_t key = 0xffffffffu;
  if (act) {
    const uint32_t job = queue[q];
    const int m = jobs.m[job];
    if (m <= leaf_max)
      key = (uint32_t)leaf_class(job, jobs, arena, mat_w, modular);
    else
      key = EVAL_KEY_DFS + (m <= 32 ? 2u : 0u) + (mat_w[jobs.mat[job]] == 4 ? 1u : 0u);
    keys[q] = key;
    vals[q] = job;
  }
  // one atomic per distinct key in the warp
  const unsigned peers = __match_any_sync(0xffffffffu, key);
  if (act && (threadIdx.x & 31) == __ffs(peers) - 1) atomicAdd(hist + key, (unsigned long long)__popc(peers));
}

template <int NMAX, int W, int PATH>
__global__ void __launch_bounds__(LEAF_WARPS * 32)
    k_leaf_batch(const uint32_t* __restrict__ queue, int64_t nq, const uint64_t* __restrict__ prefix,
                 const uint32_t* __restrict__ owner, int64_t qbase, JobArrays jobs, const uint64_t* __restrict__ arena, int chunk_log2,
                 unsigned long long* __restrict__ task_counter, JobOut out, ModP mod) {
  __shared__ __align__(16) LeafSmem sm;
  const int lane = threadIdx.x & 31;
  const int wib = threadIdx.x >> 5;
  int32_t* delta = sm.delta[wib];
  int32_t* rho0 = sm.rho0[wib];
  // prefix may be a slice of a longer scan: tasks [prefix[0], prefix[nq])
  const uint64_t base = prefix[0];
  const uint64_t total = prefix[nq] - base;
  int64_t cur_q = -1;
  int m = 0;
  for (;;) {
    unsigned long long t = 0;
    if (lane == 0) t = atomicAdd(task_counter, 1ull);
    t = __shfl_sync(0xffffffffu, t, 0);
    if (t >= total) break;
    t += base;
    // queue entry holding task t, from the task owner map
    const int64_t q = (int64_t)owner[t] - qbase;
    const uint32_t job = queue[q];
    const uint64_t first = prefix[q];
    const uint64_t lt = t - first;
    const bool single = prefix[q + 1] - first == 1;  // this warp holds the whole job
    const uint64_t t0 = globaltimer_ns();
    if (q != cur_q) {
      cur_q = q;
      m = jobs.m[job];
      if (m >= 2) leaf_load<NMAX, PATH>(arena, jobs.off[job], m, jobs.nnz[job], delta, rho0, sm.colcnt[wib], lane, mod);
    }
    uint64_t words[4];
    leaf_task<NMAX, W, PATH>(arena, jobs.off[job], m, jobs.nnz[job], lt, chunk_log2, delta, rho0, lane, mod, words);
    if (lane == 0) {
      const uint64_t t1 = globaltimer_ns();
      if (single) {  // no other warp writes this job: plain stores
        for (int k = 0; k < 4; ++k) out.acc[4ll * job + k] = words[k];
        out.t_start[job] = t0;
        out.t_end[job] = t1;
        out.sm[job] = (int32_t)smid();
      } else {
        atomic_add_words(out.acc + 4ll * job, words, 4);
        unsigned long long prev = atomicMin(out.t_start + job, (unsigned long long)t0);
        if (prev == ~0ull) out.sm[job] = (int32_t)smid();
        atomicMax(out.t_end + job, (unsigned long long)t1);
      }
      if (lt == 0) out.leaves[job] = 1;
    }
  }
}

// Leaf jobs: Sigma -> per(job) = (-1)^(m-1) Sigma / 2^(m-1), times the
// job's coefficient; the result replaces acc[job] and is added into the
// job's matrix accumulator (Algorithm PH, Step 4).
// On the residue path (modp != 0) Sigma is a residue (the sum of the
// tasks' residues in word 0) and so is the result.
__global__ void k_leaf_finalize(const uint32_t* __restrict__ queue, int64_t nq, JobArrays jobs,
                                JobOut out, unsigned long long* __restrict__ mat_acc, uint32_t modp) {
  const int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  u256 v = u256_zero();
  int mat = -1;
  if (q < nq) {
    const uint32_t job = queue[q];
    mat = jobs.mat[job];
    if (out.status[job] == 0) {
      const int m = jobs.m[job];
      uint64_t sig[4];
      for (int k = 0; k < 4; ++k) sig[k] = out.acc[4ll * job + k];
      v = leaf_finish(sig, m, jobs.coef + 4ll * job, modp);
      for (int k = 0; k < 4; ++k) out.acc[4ll * job + k] = v.w[k];
      out.nodes[job] = 1;
    }
  }
  // one accumulator update per warp when the whole warp serves one matrix
  // (failed jobs add zero), else one per job
  if (__match_any_sync(0xffffffffu, mat) == 0xffffffffu) {
    if (mat < 0) return;
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) v = u256_add(v, shfl_down_u256(v, d));
    if ((threadIdx.x & 31) == 0) atomic_add_words(mat_acc + 4ll * mat, v.w, 4);
  } else if (mat >= 0) {
    atomic_add_words(mat_acc + 4ll * mat, v.w, 4);
  }
}

__global__ void k_leaf_reject(const uint32_t* __restrict__ queue, int64_t nq, JobOut out) {
  int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (q < nq) out.status[queue[q]] = PERM_EOVERFLOW;
}

template <int NMAX, int W, int PATH>
cudaError_t launch_variant(const uint32_t* queue, int64_t nq, const uint64_t* prefix, const uint32_t* owner,
                           int64_t qbase, const JobArrays& jobs, const uint64_t* arena, int chunk_log2,
                           unsigned long long* task_counter, const JobOut& out, const ModP& mod, int num_sms,
                           cudaStream_t stream) {
  static int per_sm = 0;
  if (per_sm == 0) {
    cudaError_t e =
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_leaf_batch<NMAX, W, PATH>, LEAF_WARPS * 32, 0);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) per_sm = 1;
  }
  k_leaf_batch<NMAX, W, PATH><<<num_sms * per_sm, LEAF_WARPS * 32, 0, stream>>>(
      queue, nq, prefix, owner, qbase, jobs, arena, chunk_log2, task_counter, out, mod);
  return cudaGetLastError();
}

#define LEAF_ARGS queue, nq, prefix, owner, qbase, jobs, arena, chunk_log2, task_counter, out, mod, num_sms, stream

template <int NMAX, int W>
cudaError_t launch_path(int path, const uint32_t* queue, int64_t nq, const uint64_t* prefix, const uint32_t* owner,
                        int64_t qbase, const JobArrays& jobs, const uint64_t* arena, int chunk_log2,
                        unsigned long long* task_counter, const JobOut& out, const ModP& mod, int num_sms,
                        cudaStream_t stream) {
  switch (path) {
    case P_G7: return launch_variant<NMAX, W, P_G7>(LEAF_ARGS);
    case P_G15: return launch_variant<NMAX, W, P_G15>(LEAF_ARGS);
    case P_G31: return launch_variant<NMAX, W, P_G31>(LEAF_ARGS);
    case P_F8: return launch_variant<NMAX, W, P_F8>(LEAF_ARGS);
    case P_F4: return launch_variant<NMAX, W, P_F4>(LEAF_ARGS);
    case P_F16:
      if constexpr (NMAX >= 16) return launch_variant<NMAX, W, P_F16>(LEAF_ARGS);
      return cudaErrorInvalidValue;
    case P_MOD:  // one ring width: the residues need none
      if constexpr (W == 2) return launch_variant<NMAX, 2, P_MOD>(LEAF_ARGS);
      return cudaErrorInvalidValue;
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace

cudaError_t launch_eval_keys(const uint32_t* queue, int64_t n, const JobArrays& jobs, const uint64_t* arena,
                             const int32_t* mat_w, int leaf_max, bool modular, uint32_t* keys, uint32_t* vals,
                             unsigned long long* hist, cudaStream_t stream) {
  if (n <= 0) return cudaSuccess;
  k_eval_keys<<<(unsigned)((n + 127) / 128), 128, 0, stream>>>(queue, n, jobs, arena, mat_w, leaf_max, modular, keys,
                                                               vals, hist);
  return cudaGetLastError();
}

cudaError_t launch_leaf_tasks(const uint32_t* queue, int64_t nq, const JobArrays& jobs, int chunk_log2,
                              uint64_t* counts_scratch, uint64_t* prefix, uint32_t* owner, void* scan_tmp,
                              size_t scan_tmp_bytes, cudaStream_t stream) {
  if (nq <= 0) return cudaSuccess;
  const int tb = 256;
  k_leaf_task_counts<<<(unsigned)((nq + 1 + tb - 1) / tb), tb, 0, stream>>>(queue, nq, jobs.m, chunk_log2,
                                                                              counts_scratch);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  e = scan_exclusive_u64(counts_scratch, prefix, nq + 1, scan_tmp, scan_tmp_bytes, stream);
  if (e != cudaSuccess) return e;
  k_task_owner<<<(unsigned)((nq + tb - 1) / tb), tb, 0, stream>>>(prefix, nq, owner);
  return cudaGetLastError();
}

uint64_t leaf_tasks_host(int m, int chunk_log2) {
  if (m < 2) return 1;
  int lanes, clog;
  uint64_t tasks;
  leaf_split(m, chunk_log2, lanes, clog, tasks);
  return tasks;
}

cudaError_t launch_leaf_batch(const uint32_t* queue, int64_t nq, int cls, const uint64_t* prefix,
                              const uint32_t* owner, int64_t qbase, const JobArrays& jobs, const uint64_t* arena,
                              int chunk_log2,
                              unsigned long long* task_counter, const JobOut& out, const ModP& mod, int num_sms,
                              cudaStream_t stream) {
  if (nq <= 0) return cudaSuccess;
  const int path = cls >> 3;
  if (path == P_BAD) {
    k_leaf_reject<<<(unsigned)((nq + 255) / 256), 256, 0, stream>>>(queue, nq, out);
    return cudaGetLastError();
  }
  cudaError_t e = cudaMemsetAsync(task_counter, 0, sizeof(unsigned long long), stream);
  if (e != cudaSuccess) return e;
  const int nmi = cls & 3;
  if ((cls & 4) == 0) {
    switch (nmi) {
      case 0: return launch_path<8, 2>(path, LEAF_ARGS);
      case 1: return launch_path<16, 2>(path, LEAF_ARGS);
      case 2: return launch_path<24, 2>(path, LEAF_ARGS);
      default: return launch_path<32, 2>(path, LEAF_ARGS);
    }
  }
  switch (nmi) {
    case 0: return launch_path<8, 4>(path, LEAF_ARGS);
    case 1: return launch_path<16, 4>(path, LEAF_ARGS);
    case 2: return launch_path<24, 4>(path, LEAF_ARGS);
    default: return launch_path<32, 4>(path, LEAF_ARGS);
  }
}

cudaError_t launch_leaf_finalize(const uint32_t* queue, int64_t nq, const JobArrays& jobs, const JobOut& out,
                                 unsigned long long* mat_acc, uint32_t modp, cudaStream_t stream) {
  if (nq <= 0) return cudaSuccess;
  k_leaf_finalize<<<(unsigned)((nq + 255) / 256), 256, 0, stream>>>(queue, nq, jobs, out, mat_acc, modp);
  return cudaGetLastError();
}
