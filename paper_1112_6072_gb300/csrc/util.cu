// Scans and the stable descending sort used by the expansion and the
// ordering step (CUB from the CUDA toolkit's header sources), plus the
// integer multiply-add throughput probe used for the integer-ALU roofline.
#include <cub/cub.cuh>

#include "internal.h"

cudaError_t scan_exclusive_u64(const uint64_t* in, uint64_t* out, int64_t n, void* tmp, size_t tmp_bytes,
                               cudaStream_t s) {
  return cub::DeviceScan::ExclusiveSum(tmp, tmp_bytes, in, out, n, s);
}
size_t scan_tmp_bytes_u64(int64_t n) {
  size_t b = 0;
  cub::DeviceScan::ExclusiveSum(nullptr, b, (const uint64_t*)nullptr, (uint64_t*)nullptr, n);
  return b;
}
cudaError_t scan_exclusive_i64(const int64_t* in, int64_t* out, int64_t n, void* tmp, size_t tmp_bytes,
                               cudaStream_t s) {
  return cub::DeviceScan::ExclusiveSum(tmp, tmp_bytes, in, out, n, s);
}
size_t scan_tmp_bytes_i64(int64_t n) {
  size_t b = 0;
  cub::DeviceScan::ExclusiveSum(nullptr, b, (const int64_t*)nullptr, (int64_t*)nullptr, n);
  return b;
}
cudaError_t scan_exclusive_i32(const int32_t* in, int32_t* out, int64_t n, void* tmp, size_t tmp_bytes,
                               cudaStream_t s) {
  return cub::DeviceScan::ExclusiveSum(tmp, tmp_bytes, in, out, n, s);
}
size_t scan_tmp_bytes_i32(int64_t n) {
  size_t b = 0;
  cub::DeviceScan::ExclusiveSum(nullptr, b, (const int32_t*)nullptr, (int32_t*)nullptr, n);
  return b;
}

// CUB's radix sort is stable, so equal keys keep their input (natural) order.
cudaError_t sort_desc_f32(const float* keys_in, float* keys_out, const uint32_t* vals_in, uint32_t* vals_out,
                          int64_t n, void* tmp, size_t tmp_bytes, cudaStream_t s) {
  return cub::DeviceRadixSort::SortPairsDescending(tmp, tmp_bytes, keys_in, keys_out, vals_in, vals_out, n, 0,
                                                   32, s);
}
size_t sort_tmp_bytes_f32(int64_t n) {
  size_t b = 0;
  cub::DeviceRadixSort::SortPairsDescending(nullptr, b, (const float*)nullptr, (float*)nullptr,
                                            (const uint32_t*)nullptr, (uint32_t*)nullptr, n);
  return b;
}

cudaError_t sort_asc_u64(const uint64_t* keys_in, uint64_t* keys_out, const uint32_t* vals_in, uint32_t* vals_out,
                         int64_t n, int end_bit, void* tmp, size_t tmp_bytes, cudaStream_t s) {
  return cub::DeviceRadixSort::SortPairs(tmp, tmp_bytes, keys_in, keys_out, vals_in, vals_out, n, 0, end_bit, s);
}
size_t sort_tmp_bytes_u64(int64_t n) {
  size_t b = 0;
  cub::DeviceRadixSort::SortPairs(nullptr, b, (const uint64_t*)nullptr, (uint64_t*)nullptr, (const uint32_t*)nullptr,
                                  (uint32_t*)nullptr, n, 0, 64);
  return b;
}

cudaError_t sort_asc_u32(const uint32_t* keys_in, uint32_t* keys_out, const uint32_t* vals_in, uint32_t* vals_out,
                         int64_t n, int end_bit, void* tmp, size_t tmp_bytes, cudaStream_t s) {
  return cub::DeviceRadixSort::SortPairs(tmp, tmp_bytes, keys_in, keys_out, vals_in, vals_out, n, 0, end_bit, s);
}
size_t sort_tmp_bytes_u32(int64_t n, int end_bit) {
  size_t b = 0;
  cub::DeviceRadixSort::SortPairs(nullptr, b, (const uint32_t*)nullptr, (uint32_t*)nullptr, (const uint32_t*)nullptr,
                                  (uint32_t*)nullptr, n, 0, end_bit);
  return b;
}

// ---- evaluation bookkeeping on the device (no per-job host copies) -----------

__global__ void k_status_summary(const int32_t* __restrict__ status, int64_t n, unsigned long long* out) {
  const int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  unsigned long long key = ~0ull;
  if (j < n) {
    const int32_t s = status[j];
    if (s != 0 && s != DFS_RETRY) key = (unsigned long long)j * 256ull + (unsigned long long)(s & 255);
  }
  // lowest key of the warp, then one atomic per warp
#pragma unroll
  for (int d = 16; d > 0; d >>= 1) {
    const unsigned long long o = __shfl_xor_sync(0xffffffffu, key, d);
    key = o < key ? o : key;
  }
  if ((threadIdx.x & 31) == 0 && key != ~0ull) atomicMin(out, key);
}

__global__ void k_iota_u32(uint32_t* __restrict__ out, int64_t n) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) out[i] = (uint32_t)i;
}

cudaError_t launch_iota_u32(uint32_t* out, int64_t n, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  k_iota_u32<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(out, n);
  return cudaGetLastError();
}

cudaError_t launch_status_summary(const int32_t* status, int64_t n, unsigned long long* out, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  k_status_summary<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(status, n, out);
  return cudaGetLastError();
}

__global__ void k_retry_flags(const uint32_t* __restrict__ dq, int64_t n, const int32_t* __restrict__ status,
                              int32_t* __restrict__ flags) {
  const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (k < n) flags[k] = status[dq[k]] == DFS_RETRY ? 1 : 0;
  if (k == n) flags[k] = 0;  // the scan's last entry is the total
}

__global__ void k_retry_scatter(const uint32_t* __restrict__ dq, int64_t n, RetryBounds bounds,
                                const int32_t* __restrict__ flags, const int32_t* __restrict__ pos,
                                uint32_t* __restrict__ rq, unsigned long long* at) {
  const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (k < n && flags[k]) rq[pos[k]] = dq[k];
  if (k == n) {
    for (int g = 0; g <= EVAL_DFS_GROUPS; ++g) at[g] = (unsigned long long)pos[bounds.b[g]];
  }
}

cudaError_t launch_retry_collect(const uint32_t* dq, int64_t n, RetryBounds bounds, const int32_t* status,
                                 int32_t* flags, int32_t* pos, void* scan_tmp, size_t scan_tmp_bytes, uint32_t* rq,
                                 unsigned long long* at, cudaStream_t s) {
  const unsigned blocks = (unsigned)((n + 1 + 255) / 256);
  k_retry_flags<<<blocks, 256, 0, s>>>(dq, n, status, flags);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  e = scan_exclusive_i32(flags, pos, n + 1, scan_tmp, scan_tmp_bytes, s);
  if (e != cudaSuccess) return e;
  k_retry_scatter<<<blocks, 256, 0, s>>>(dq, n, bounds, flags, pos, rq, at);
  return cudaGetLastError();
}

// 16 independent dependency chains of 32-bit multiply-adds per thread, so
// the issue rate rather than the latency limits the throughput.
__global__ void k_ubench_imad(int iters, uint32_t* sink) {
  uint32_t a[16];
#pragma unroll
  for (int k = 0; k < 16; ++k) a[k] = threadIdx.x * 2654435761u + k;
  const uint32_t b = 0x9E3779B9u ^ blockIdx.x, c = 0x7F4A7C15u;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < 16; ++k) a[k] = a[k] * b + c;
  }
  uint32_t x = 0;
#pragma unroll
  for (int k = 0; k < 16; ++k) x ^= a[k];
  if (x == 0x12345678u) sink[blockIdx.x] = x;  // keeps the chains alive
}

cudaError_t launch_ubench_imad(int blocks, int iters, uint32_t* sink, cudaStream_t s) {
  k_ubench_imad<<<blocks, 256, 0, s>>>(iters, sink);
  return cudaGetLastError();
}
