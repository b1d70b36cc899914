// Integers from their residues modulo k primes by the Chinese remainder
// theorem: the reconstruction step of the residue path (per(A) mod p_i for
// several primes, each from one run of Algorithm PH modulo p_i, give per(A)).
//
// Garner's algorithm (H. L. Garner, "The residue number system", IRE Trans.
// Electronic Computers EC-8, 1959): mixed-radix digits v_i with
//     x = v_0 + v_1 p_0 + v_2 p_0 p_1 + ... ,   0 <= v_i < p_i,
// computed digit by digit as  t = r_i;  for j < i:  t = (t - v_j) p_j^-1 mod p_i,
// so that x is the unique value in [0, M), M = p_0 ... p_{k-1}, with the
// given residues.  x is formed by Horner's rule in 32-bit limbs, and the
// balanced value (x - M when 2x > M) is returned as a sign and a magnitude:
// every integer of absolute value below M / 2 comes back exactly.
#include <cuda_runtime.h>

#include <cstdint>
#include <vector>

#include "internal.h"

namespace {

constexpr int kMaxPrimes = 64;

// One value per thread: residues r[v * k + i], primes p[i], inverses
// inv[j * k + i] = p_j^-1 mod p_i (j < i), M in k + 1 limbs.  out: k + 1
// limbs of the magnitude per value; sign: -1, 0 or +1.
__global__ void k_crt(const uint32_t* __restrict__ r, const uint32_t* __restrict__ p,
                      const uint32_t* __restrict__ inv, const uint32_t* __restrict__ Mlimbs, int k, int count,
                      uint32_t* __restrict__ out, int32_t* __restrict__ sign) {
  const int v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= count) return;
  uint32_t d[kMaxPrimes];
  for (int i = 0; i < k; ++i) {
    const uint64_t pi = p[i];
    uint64_t t = r[(int64_t)v * k + i];
    for (int j = 0; j < i; ++j) {
      const uint64_t vj = d[j] % pi;
      t = (t + pi - vj) % pi * inv[j * k + i] % pi;
    }
    d[i] = (uint32_t)t;
  }
  // x = d_{k-1};  x = x p_i + d_i for i = k-2 .. 0  (x < M < 2^(31k): k + 1 limbs)
  uint32_t* x = out + (int64_t)v * (k + 1);
  for (int w = 0; w <= k; ++w) x[w] = 0;
  for (int i = k - 1; i >= 0; --i) {
    uint64_t carry = d[i];
    for (int w = 0; w <= k; ++w) {
      const uint64_t t = (uint64_t)x[w] * p[i] + carry;
      x[w] = (uint32_t)t;
      carry = t >> 32;
    }
  }
  // balanced value: compare 2x (k + 2 limbs) with M (k + 1 limbs)
  int cmp = 0;
  for (int w = k + 1; w >= 0 && cmp == 0; --w) {
    const uint32_t y = w == k + 1 ? (x[k] >> 31) : ((x[w] << 1) | (w > 0 ? x[w - 1] >> 31 : 0u));
    const uint32_t mw = w <= k ? Mlimbs[w] : 0u;
    if (y != mw) cmp = y > mw ? 1 : -1;
  }
  bool zero = true;
  for (int w = 0; w <= k; ++w) zero = zero && x[w] == 0;
  if (cmp > 0) {  // x - M < 0: magnitude M - x
    int64_t borrow = 0;
    for (int w = 0; w <= k; ++w) {
      const int64_t t = (int64_t)Mlimbs[w] - (int64_t)x[w] - borrow;
      x[w] = (uint32_t)t;
      borrow = t < 0 ? 1 : 0;
    }
  }
  sign[v] = zero ? 0 : (cmp > 0 ? -1 : 1);
}

}  // namespace

static perm_status perm_crt_impl(const uint32_t* residues, const uint32_t* primes, int32_t k, int32_t count,
                                 uint32_t* limbs, int32_t* signs, void* stream) {
  if (!residues || !primes || !limbs || !signs || k < 1 || k > kMaxPrimes || count < 1) return PERM_EINVAL;
  for (int i = 0; i < k; ++i) {
    if (!modp_is_odd_prime(primes[i])) return PERM_EINVAL;
    for (int j = 0; j < i; ++j)
      if (primes[j] == primes[i]) return PERM_EINVAL;
  }
  for (int64_t v = 0; v < (int64_t)count * k; ++v)
    if (residues[v] >= primes[v % k]) return PERM_EINVAL;
  // p_j^-1 mod p_i (Fermat: p_i is prime) and M = p_0 ... p_{k-1} in k + 1 limbs
  std::vector<uint32_t> inv((size_t)k * k, 0u), M((size_t)k + 1, 0u);
  for (int i = 0; i < k; ++i)
    for (int j = 0; j < i; ++j) inv[(size_t)j * k + i] = mod_pow(primes[j] % primes[i], primes[i] - 2, primes[i]);
  M[0] = 1;
  for (int i = 0; i < k; ++i) {
    uint64_t carry = 0;
    for (int w = 0; w <= k; ++w) {
      const uint64_t t = (uint64_t)M[w] * primes[i] + carry;
      M[w] = (uint32_t)t;
      carry = t >> 32;
    }
  }
  cudaStream_t s = (cudaStream_t)stream;
  const size_t nr = (size_t)count * k, nl = (size_t)count * (k + 1);
  uint32_t *dr = nullptr, *dp = nullptr, *di = nullptr, *dm = nullptr, *dl = nullptr;
  int32_t* ds = nullptr;
  cudaError_t e = cudaMallocAsync(&dr, 4 * nr, s);
  if (e == cudaSuccess) e = cudaMallocAsync(&dp, 4 * (size_t)k, s);
  if (e == cudaSuccess) e = cudaMallocAsync(&di, 4 * inv.size(), s);
  if (e == cudaSuccess) e = cudaMallocAsync(&dm, 4 * M.size(), s);
  if (e == cudaSuccess) e = cudaMallocAsync(&dl, 4 * nl, s);
  if (e == cudaSuccess) e = cudaMallocAsync(&ds, 4 * (size_t)count, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(dr, residues, 4 * nr, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(dp, primes, 4 * (size_t)k, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(di, inv.data(), 4 * inv.size(), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(dm, M.data(), 4 * M.size(), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) {
    k_crt<<<(count + 127) / 128, 128, 0, s>>>(dr, dp, di, dm, k, count, dl, ds);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(limbs, dl, 4 * nl, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(signs, ds, 4 * (size_t)count, cudaMemcpyDeviceToHost, s);
  for (void* q : {(void*)dr, (void*)dp, (void*)di, (void*)dm, (void*)dl, (void*)ds})
    if (q) cudaFreeAsync(q, s);
  const cudaError_t e2 = cudaStreamSynchronize(s);
  if (e == cudaSuccess) e = e2;
  if (e != cudaSuccess) {
    set_last_error("perm_crt", e);
    return e == cudaErrorMemoryAllocation ? PERM_ENOMEM : PERM_ECUDA;
  }
  return PERM_OK;
}
extern "C" perm_status perm_crt(const uint32_t* residues, const uint32_t* primes, int32_t k, int32_t count,
                                uint32_t* limbs, int32_t* signs, void* stream) {
  return guarded([&] { return perm_crt_impl(residues, primes, k, count, limbs, signs, stream); });
}
