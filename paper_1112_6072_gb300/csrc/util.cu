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
