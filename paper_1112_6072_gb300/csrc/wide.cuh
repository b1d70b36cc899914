// Wrap-around integer arithmetic modulo 2^128 and 2^256 for the exact paths.
//
// Every permanent computed by the library is an integer; all of its
// arithmetic (Eq. 2's merges and scalar factors, Ryser's sums and products)
// is ring arithmetic, so it is carried out modulo 2^(64*W) and the signed
// result is recovered from a proven magnitude bound.  Signed operands are
// handled as their two's complement residues, which is exact in this ring.
#pragma once
#include <cstdint>

typedef unsigned __int128 u128;

struct u256 {
  uint64_t w[4];
};

__host__ __device__ __forceinline__ u256 u256_zero() {
  u256 r;
  r.w[0] = r.w[1] = r.w[2] = r.w[3] = 0;
  return r;
}

__host__ __device__ __forceinline__ u256 u256_from_s64(int64_t v) {
  u256 r;
  uint64_t s = v < 0 ? ~0ull : 0ull;
  r.w[0] = (uint64_t)v;
  r.w[1] = r.w[2] = r.w[3] = s;
  return r;
}

__host__ __device__ __forceinline__ u256 u256_from_u128(u128 v) {
  u256 r;
  r.w[0] = (uint64_t)v;
  r.w[1] = (uint64_t)(v >> 64);
  r.w[2] = r.w[3] = 0;
  return r;
}

__host__ __device__ __forceinline__ u256 u256_add(const u256& a, const u256& b) {
  u256 r;
  u128 c = 0;
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    c += (u128)a.w[k] + b.w[k];
    r.w[k] = (uint64_t)c;
    c >>= 64;
  }
  return r;
}

__host__ __device__ __forceinline__ u256 u256_neg(const u256& a) {
  u256 r;
  u128 c = 1;
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    c += (u128)(~a.w[k]);
    r.w[k] = (uint64_t)c;
    c >>= 64;
  }
  return r;
}

__host__ __device__ __forceinline__ u256 u256_sub(const u256& a, const u256& b) {
  return u256_add(a, u256_neg(b));
}

// a * b mod 2^256 with b a signed 64-bit value.
__host__ __device__ __forceinline__ u256 u256_mul_s64(const u256& a, int64_t b) {
  uint64_t ub = (uint64_t)b;
  u256 r;
  u128 c = 0;
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    c += (u128)a.w[k] * ub;
    r.w[k] = (uint64_t)c;
    c >>= 64;
  }
  if (b < 0) {  // b = ub - 2^64: subtract a << 64
    u256 sh;
    sh.w[0] = 0;
    sh.w[1] = a.w[0];
    sh.w[2] = a.w[1];
    sh.w[3] = a.w[2];
    r = u256_sub(r, sh);
  }
  return r;
}

// a * b mod 2^256, both as residues.
__host__ __device__ __forceinline__ u256 u256_mul(const u256& a, const u256& b) {
  u256 r = u256_zero();
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    u128 c = 0;
#pragma unroll
    for (int j = 0; j + i < 4; ++j) {
      c += (u128)a.w[i] * b.w[j] + r.w[i + j];
      r.w[i + j] = (uint64_t)c;
      c >>= 64;
    }
  }
  return r;
}

// Logical right shift by s (0 <= s < 64) of a 256-bit residue.
__host__ __device__ __forceinline__ u256 u256_shr(const u256& a, int s) {
  if (s == 0) return a;
  u256 r;
#pragma unroll
  for (int k = 0; k < 3; ++k) r.w[k] = (a.w[k] >> s) | (a.w[k + 1] << (64 - s));
  r.w[3] = a.w[3] >> s;
  return r;
}

// a * b mod 2^128 with b a signed 64-bit value.
__device__ __forceinline__ u128 mul128_s64(u128 a, int64_t b) {
  uint64_t alo = (uint64_t)a, ahi = (uint64_t)(a >> 64);
  uint64_t ub = (uint64_t)b;
  uint64_t lo = alo * ub;
  uint64_t hi = __umul64hi(alo, ub) + ahi * ub;
  if (b < 0) hi -= alo;
  return ((u128)hi << 64) | lo;
}

// Signed 64 x 64 -> 128 product as a residue mod 2^128.
__device__ __forceinline__ u128 mul_s64_s64(int64_t a, int64_t b) {
  uint64_t lo = (uint64_t)a * (uint64_t)b;
  uint64_t hi = (uint64_t)__mul64hi(a, b);
  return ((u128)hi << 64) | lo;
}

// a * b mod 2^128, both residues.
__device__ __forceinline__ u128 mul128(u128 a, u128 b) {
  uint64_t alo = (uint64_t)a, ahi = (uint64_t)(a >> 64);
  uint64_t blo = (uint64_t)b, bhi = (uint64_t)(b >> 64);
  uint64_t lo = alo * blo;
  uint64_t hi = __umul64hi(alo, blo) + alo * bhi + ahi * blo;
  return ((u128)hi << 64) | lo;
}

// Add a W-word value into W words of global memory with carries between
// words, modulo 2^(64W).  Safe against concurrent callers: every wrap of a
// word is returned by its atomicAdd and forwarded to the next word, so the
// final contents equal the sum of all addends modulo 2^(64W).
__device__ __forceinline__ void atomic_add_words(unsigned long long* dst, const uint64_t* v, int W) {
  uint64_t carry = 0;
  for (int k = 0; k < W; ++k) {
    uint64_t x = v[k] + carry;
    uint64_t c1 = x < carry ? 1ull : 0ull;
    carry = c1;
    if (x == 0) continue;
    unsigned long long old = atomicAdd(dst + k, (unsigned long long)x);
    carry += (old + x < old) ? 1ull : 0ull;
  }
}

__device__ __forceinline__ u128 shfl_down_u128(u128 v, int d) {
  uint64_t lo = __shfl_down_sync(0xffffffffu, (unsigned long long)(uint64_t)v, d);
  uint64_t hi = __shfl_down_sync(0xffffffffu, (unsigned long long)(uint64_t)(v >> 64), d);
  return ((u128)hi << 64) | lo;
}

__device__ __forceinline__ u256 shfl_down_u256(const u256& v, int d) {
  u256 r;
#pragma unroll
  for (int k = 0; k < 4; ++k) r.w[k] = __shfl_down_sync(0xffffffffu, (unsigned long long)v.w[k], d);
  return r;
}

__device__ __forceinline__ uint64_t globaltimer_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ uint32_t smid() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%smid;" : "=r"(r));
  return r;
}
