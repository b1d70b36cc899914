// Arithmetic modulo an odd prime p < 2^31, for the residue path.
//
// A permanent is an integer polynomial in the entries, so per(A) mod p can
// be computed with every value -- the entries, Eq. 2's merged entries and
// scalar factors, Ryser's row sums and products -- reduced modulo p.
// Several primes and the Chinese remainder theorem then give per(A) exactly
// whatever its size.  Products use Montgomery's reduction (P. L. Montgomery,
// "Modular multiplication without trial division", Math. Comp. 44, 1985)
// with R = 2^32: a value x is held as x R mod p, and
//     mont_mul(a R, b R) = (a R)(b R) R^-1 = a b R  (mod p),
// two 32 x 32 -> 64-bit products and one 32-bit product per multiplication.
// Sums and differences need no conversion.
#pragma once
#include <cstdint>

struct ModP {
  uint32_t p;     // the modulus: 0 = no modulus (the exact ring path), else an odd prime below 2^31
  uint32_t pneg;  // -p^-1 mod 2^32
  uint32_t r2;    // R^2 mod p, R = 2^32
};

// ModP for p: -p^-1 mod 2^32 by Newton's iteration x <- x (2 - p x) (each
// step doubles the number of correct low bits; x = p is right to three
// bits since p^2 = 1 mod 8), R^2 mod p in 64-bit arithmetic.
__host__ __device__ inline ModP modp_make(uint32_t p) {
  ModP m;
  m.p = p;
  uint32_t x = p;
  for (int i = 0; i < 4; ++i) x *= 2u - p * x;  // 3 -> 6 -> 12 -> 24 -> 48 bits
  m.pneg = 0u - x;
  const uint64_t r = (((uint64_t)1) << 32) % p;
  m.r2 = (uint32_t)((r * r) % p);
  return m;
}

__host__ __device__ __forceinline__ uint32_t mod_add(uint32_t a, uint32_t b, uint32_t p) {
  const uint32_t s = a + b;  // < 2^32 since a, b < p < 2^31
  return s >= p ? s - p : s;
}
__host__ __device__ __forceinline__ uint32_t mod_sub(uint32_t a, uint32_t b, uint32_t p) {
  return a >= b ? a - b : a + p - b;
}

// a b R^-1 mod p for a, b < p: t + q p is divisible by 2^32 and
// (t + q p) / 2^32 < (p^2 + 2^32 p) / 2^32 < 2p
__host__ __device__ __forceinline__ uint32_t mont_mul(uint32_t a, uint32_t b, const ModP& M) {
  const uint64_t t = (uint64_t)a * b;
  const uint32_t q = (uint32_t)t * M.pneg;
  const uint64_t u = (t + (uint64_t)q * M.p) >> 32;
  return u >= M.p ? (uint32_t)(u - M.p) : (uint32_t)u;
}
__host__ __device__ __forceinline__ uint32_t to_mont(uint32_t a, const ModP& M) { return mont_mul(a, M.r2, M); }
__host__ __device__ __forceinline__ uint32_t from_mont(uint32_t a, const ModP& M) { return mont_mul(a, 1u, M); }

// a signed 64-bit integer reduced into [0, p)
__host__ __device__ __forceinline__ uint32_t mod_of(int64_t v, uint32_t p) {
  const int64_t r = v % (int64_t)p;
  return (uint32_t)(r < 0 ? r + (int64_t)p : r);
}

// (a x + b y) mod p for residues a, x, b, y < p < 2^31 (the sum is below 2^63)
__host__ __device__ __forceinline__ uint32_t mod_mad2(uint64_t a, uint64_t x, uint64_t b, uint64_t y, uint32_t p) {
  return (uint32_t)((a * x + b * y) % p);
}

// a^e mod p (plain residues, square and multiply)
__host__ __device__ inline uint32_t mod_pow(uint32_t a, uint64_t e, uint32_t p) {
  uint64_t r = 1 % p, b = a % p;
  while (e) {
    if (e & 1) r = r * b % p;
    b = b * b % p;
    e >>= 1;
  }
  return (uint32_t)r;
}

// A modulus of the residue path is an odd prime below 2^31 (trial division).
__host__ __device__ inline bool modp_is_odd_prime(uint32_t p) {
  if (p < 3 || (p & 1u) == 0 || p >= (1u << 31)) return false;
  for (uint32_t d = 3; (uint64_t)d * d <= p; d += 2)
    if (p % d == 0) return false;
  return true;
}
