// K2: batched leaf evaluation by Ryser / Nijenhuis-Wilf (Section 1) for jobs
// whose order is at most the leaf order.  The 2^(m-1) Gray codes of a job
// are cut into tasks of 32 lanes x 2^c codes; a persistent grid of warps
// pulls tasks through one atomic counter in queue order (the job order set
// by the LPT / learned ordering), so big jobs queued first are spread over
// many warps and small jobs fill the tail.
#include <cuda_runtime.h>

#include <cstdint>

#include "internal.h"
#include "jobs.cuh"
#include "ryser.cuh"

namespace {

constexpr int LEAF_WARPS = 8;  // warps per block

struct LeafSmem {
  int32_t delta[LEAF_WARPS][(PERM_MAX_LEAF - 1) * 32];
  int32_t rho0[LEAF_WARPS][32];
};

__host__ __device__ __forceinline__ void leaf_split(int m, int chunk_log2, int& lanes, int& clog,
                                                    uint64_t& tasks) {
  // m >= 2: 2^(m-1) codes.  Lanes walk aligned blocks of 2^clog >= 2 codes.
  const int e = m - 1;
  if (e <= 5) {
    clog = 1;
    lanes = 1 << (e - 1);
    tasks = 1;
    return;
  }
  lanes = 32;
  clog = e - 5 < chunk_log2 ? e - 5 : chunk_log2;
  tasks = 1ull << (e - 5 - clog);
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

// Load job `job` into the warp's leaf buffers.  Returns false (and sets the
// job status) when an entry or a row sum leaves the int32 range.
__device__ bool load_leaf(const uint64_t* __restrict__ arena, int64_t off, int m, int nnz, int nmax,
                          int32_t* delta, int32_t* rho0, int lane, int& bc) {
  CsrView v = csr_view(arena, off, m, nnz);
  const int cols = m - 1;
  for (int k = lane; k < cols * nmax; k += 32) delta[k] = 0;
  __syncwarp();
  int64_t rmax = 0;
  bool ok = true;
  for (int i = lane; i < nmax; i += 32) {
    if (i >= m) {
      rho0[i] = 1;
      continue;
    }
    int64_t rs = 0, ra = 0, last = 0;
    for (int p = v.rowptr[i]; p < v.rowptr[i + 1]; ++p) {
      int c = v.col[p];
      int64_t a = v.val[p];
      if (a >= (1ll << 30) || a <= -(1ll << 30)) ok = false;
      rs += a;
      ra += a < 0 ? -a : a;
      if (c < cols)
        delta[c * nmax + i] = (int32_t)(2 * a);
      else
        last = a;
    }
    if (ra >= (1ll << 31)) ok = false;
    rmax = ra > rmax ? ra : rmax;
    rho0[i] = (int32_t)(2 * last - rs);
  }
  ok = __all_sync(0xffffffffu, ok);
#pragma unroll
  for (int d = 16; d > 0; d >>= 1) {
    int64_t o = __shfl_xor_sync(0xffffffffu, rmax, d);
    rmax = o > rmax ? o : rmax;
  }
  bc = bit_class(rmax);
  __syncwarp();
  return ok;
}

// One persistent grid per (NMAX, W) group: every job of the group is held in
// NMAX registers per lane (rows beyond m padded with rho = 1) and summed
// modulo 2^(64W).
template <int NMAX, int W>
__global__ void __launch_bounds__(LEAF_WARPS * 32)
    k_leaf_batch(const uint32_t* __restrict__ queue, int64_t nq, const uint64_t* __restrict__ prefix,
                 JobArrays jobs, const uint64_t* __restrict__ arena, int chunk_log2,
                 unsigned long long* __restrict__ task_counter, JobOut out) {
  __shared__ __align__(16) LeafSmem sm;
  const int lane = threadIdx.x & 31;
  const int wib = threadIdx.x >> 5;
  int32_t* delta = sm.delta[wib];
  int32_t* rho0 = sm.rho0[wib];
  const uint64_t total = prefix[nq];
  int64_t cur_q = -1;
  int m = 0, bc = 31;
  bool ok = false;
  for (;;) {
    unsigned long long t = 0;
    if (lane == 0) t = atomicAdd(task_counter, 1ull);
    t = __shfl_sync(0xffffffffu, t, 0);
    if (t >= total) break;
    // queue entry holding task t: last q with prefix[q] <= t
    int64_t lo = 0, hi = nq - 1;
    while (lo < hi) {
      int64_t mid = (lo + hi + 1) >> 1;
      if (prefix[mid] <= t) lo = mid; else hi = mid - 1;
    }
    const int64_t q = lo;
    const uint32_t job = queue[q];
    const uint64_t lt = t - prefix[q];
    const uint64_t t0 = globaltimer_ns();
    if (q != cur_q) {
      cur_q = q;
      m = jobs.m[job];
      ok = m <= NMAX;
      if (ok && m >= 2) ok = load_leaf(arena, jobs.off[job], m, jobs.nnz[job], NMAX, delta, rho0, lane, bc);
      if (!ok && lane == 0) out.status[job] = PERM_EOVERFLOW;
    }
    uint64_t words[4] = {0, 0, 0, 0};
    if (ok) {
      if (m == 1) {
        if (lane == 0) {
          CsrView v = csr_view(arena, jobs.off[job], 1, jobs.nnz[job]);
          int64_t a = jobs.nnz[job] ? v.val[0] : 0;
          uint64_t s = a < 0 ? ~0ull : 0ull;
          words[0] = (uint64_t)a;
          words[1] = words[2] = words[3] = s;
        }
      } else {
        int lanes, clog;
        uint64_t tasks;
        leaf_split(m, chunk_log2, lanes, clog, tasks);
        const uint64_t cnt = 1ull << clog;
        const uint64_t gb = (lt * 32 + lane) * cnt;
        // idle lanes (small jobs) run an empty range and contribute zero
        const uint64_t mycnt = lane < lanes ? cnt : 0;
        run_lane<NMAX, W>(bc, delta, rho0, m, gb, mycnt, words);
      }
    }
    if (lane == 0) {
      if (ok) atomic_add_words(out.acc + 4ll * job, words, 4);
      const uint64_t t1 = globaltimer_ns();
      unsigned long long prev = atomicMin(out.t_start + job, (unsigned long long)t0);
      if (prev == ~0ull) out.sm[job] = (int32_t)smid();
      atomicMax(out.t_end + job, (unsigned long long)t1);
      if (lt == 0) out.leaves[job] = 1;
    }
  }
}

// Leaf jobs: Sigma -> per(job) = (-1)^(m-1) Sigma / 2^(m-1), times the
// job's coefficient; the result replaces acc[job] and is added into the
// job's matrix accumulator (Algorithm PH, Step 4).
__global__ void k_leaf_finalize(const uint32_t* __restrict__ queue, int64_t nq, JobArrays jobs,
                                JobOut out, unsigned long long* __restrict__ mat_acc) {
  int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (q >= nq) return;
  const uint32_t job = queue[q];
  if (out.status[job] != 0) return;
  const int m = jobs.m[job];
  u256 s;
  for (int k = 0; k < 4; ++k) s.w[k] = out.acc[4ll * job + k];
  if (m >= 2) {
    s = u256_shr(s, m - 1);
    if ((m - 1) & 1) s = u256_neg(s);
  }
  u256 c;
  for (int k = 0; k < 4; ++k) c.w[k] = jobs.coef[4ll * job + k];
  u256 v = u256_mul(s, c);
  for (int k = 0; k < 4; ++k) out.acc[4ll * job + k] = v.w[k];
  out.nodes[job] = 1;
  atomic_add_words(mat_acc + 4ll * jobs.mat[job], v.w, 4);
}


template <int NMAX, int W>
cudaError_t launch_group(const uint32_t* queue, int64_t nq, const uint64_t* prefix, const JobArrays& jobs,
                         const uint64_t* arena, int chunk_log2, unsigned long long* task_counter, const JobOut& out,
                         int num_sms, cudaStream_t stream) {
  int per_sm = 0;
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_leaf_batch<NMAX, W>, LEAF_WARPS * 32, 0);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) per_sm = 1;
  k_leaf_batch<NMAX, W><<<num_sms * per_sm, LEAF_WARPS * 32, 0, stream>>>(queue, nq, prefix, jobs, arena,
                                                                          chunk_log2, task_counter, out);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_leaf_batch(const uint32_t* queue, int64_t nq, int nmax, int W, const JobArrays& jobs,
                              const uint64_t* arena, int chunk_log2, uint64_t* counts_scratch, uint64_t* prefix,
                              void* scan_tmp, size_t scan_tmp_bytes, unsigned long long* task_counter,
                              const JobOut& out, int num_sms, cudaStream_t stream) {
  if (nq <= 0) return cudaSuccess;
  const int tb = 256;
  k_leaf_task_counts<<<(unsigned)((nq + 1 + tb - 1) / tb), tb, 0, stream>>>(queue, nq, jobs.m, chunk_log2,
                                                                              counts_scratch);
  cudaError_t e = scan_exclusive_u64(counts_scratch, prefix, nq + 1, scan_tmp, scan_tmp_bytes, stream);
  if (e != cudaSuccess) return e;
  e = cudaMemsetAsync(task_counter, 0, sizeof(unsigned long long), stream);
  if (e != cudaSuccess) return e;
#define LEAF_CASE(NM, WW) \
  if (nmax == NM && W == WW) return launch_group<NM, WW>(queue, nq, prefix, jobs, arena, chunk_log2, task_counter, out, num_sms, stream);
  LEAF_CASE(8, 2) LEAF_CASE(16, 2) LEAF_CASE(24, 2) LEAF_CASE(32, 2)
  LEAF_CASE(8, 4) LEAF_CASE(16, 4) LEAF_CASE(24, 4) LEAF_CASE(32, 4)
#undef LEAF_CASE
  return cudaErrorInvalidValue;
}

cudaError_t launch_leaf_finalize(const uint32_t* queue, int64_t nq, const JobArrays& jobs, const JobOut& out,
                                 unsigned long long* mat_acc, cudaStream_t stream) {
  if (nq <= 0) return cudaSuccess;
  k_leaf_finalize<<<(unsigned)((nq + 255) / 256), 256, 0, stream>>>(queue, nq, jobs, out, mat_acc);
  return cudaGetLastError();
}
