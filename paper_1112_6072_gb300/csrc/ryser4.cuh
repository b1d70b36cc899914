// Leaf evaluator, blocked form: the Gray walk of ryser.cuh taken four codes
// at a time, for leaves whose row sums fit the 7-bit class.
//
// The leaf's columns and rows are permuted first (the permanent does not
// change): the two sparsest columns become Gray columns 0 and 1, and the rows
// holding a nonzero in either of them ("N" rows) take the first NN register
// slots; the other rows ("Z" rows) take the remaining NMAX - NN slots.
// Within an aligned block of four codes g, g+1, g+2, g+3 (g = 0 mod 4) only
// Gray columns 0 and 1 flip -- column 0 in, column 1 in or out, column 0
// out -- so only N rows change and, with signs +, -, +, -,
//     sum_{t<4} (-1)^t prod_i rho_i(g+t)
//       = prod_{Z} rho_i(g) * sum_{t<4} (-1)^t prod_{N} rho_i(g+t).
// The Z product and the wide multiply-accumulate happen once per block; the
// four N products stay in 64 bits (NN = 8).  For NN = 16 the rows of Gray
// column 0 sit in slots [0, 8) (N1) and slots [8, 16) hold none (N2), so the
// N2 product only changes when column 1 flips and
//     sum_t (-1)^t P1(t) P2(t) = (P1(0) - P1(1)) P2(0) + (P1(2) - P1(3)) P2(2),
// two 64 x 64 -> wide products per block.  For NN = 8 with Gray column 0
// touching at most 4 rows (SPLIT4: its rows sit in slots [0, 4), so slots
// [4, 8) only change when column 1 flips) the same identity with 4-slot
// halves A and B gives
//     sum_t (-1)^t prod_N = (PA(0) - PA(1)) PB(0) + (PA(2) - PA(3)) PB(2),
// six 32-bit quad products and two widening multiplies per block instead of
// four 8-slot products, and column 0 updates four slots instead of eight.
// Column j >= 2 flips at code g with j = ctz(g) and updates every row from
// shared memory (a broadcast, uniform across the warp).
#pragma once
#include <cstdint>

#include "ryser.cuh"

// product of the 8 slots [b, b+8) for |rho| < 2^7: two int32 quads, one widening multiply
template <int NMAX>
__device__ __forceinline__ int32_t prod4(const int32_t (&r)[NMAX], int b) {
  return r[b] * r[b + 1] * r[b + 2] * r[b + 3];
}

template <int NMAX>
__device__ __forceinline__ int64_t prod8(const int32_t (&r)[NMAX], int b) {
  const int32_t q0 = r[b] * r[b + 1] * r[b + 2] * r[b + 3];
  const int32_t q1 = r[b + 4] * r[b + 5] * r[b + 6] * r[b + 7];
  return (int64_t)q0 * (int64_t)q1;
}

__device__ __forceinline__ u128 wide_mulTT(u128 a, u128 b) { return mul128(a, b); }
__device__ __forceinline__ u256 wide_mulTT(const u256& a, const u256& b) { return u256_mul(a, b); }

// product of slots [B, B + 8*G) in the wide ring (G >= 2)
template <int NMAX, int W, int B, int G>
__device__ __forceinline__ typename WideT<W>::type prod_groups(const int32_t (&r)[NMAX]) {
  typedef typename WideT<W>::type T;
  T p = wide_mul64x64(prod8<NMAX>(r, B), prod8<NMAX>(r, B + 8), (T*)nullptr);
#pragma unroll
  for (int k = 2; k < G; ++k) p = wide_mul64(p, prod8<NMAX>(r, B + 8 * k));
  return p;
}

template <int NMAX, int NN, int W, bool SPLIT4 = false, bool BR = true>
__device__ __forceinline__ typename WideT<W>::type ryser_lane4(const int32_t* __restrict__ delta,
                                                               const int32_t* __restrict__ rho0, int m,
                                                               uint64_t gb, uint64_t cnt) {
  typedef typename WideT<W>::type T;
  static_assert(NN % 8 == 0 && NN <= NMAX && NMAX % 8 == 0, "slot groups of 8");
  static_assert(!SPLIT4 || NN == 8, "the 4 + 4 split is of the 8-slot form");
  constexpr int GN = NN / 8;
  constexpr int GZ = (NMAX - NN) / 8;
  if (cnt == 0) return wide_from64(0, (T*)nullptr);
  // column 0 touches only the first 8 slots (NN = 8, and the N1 group of NN = 16)
  int32_t rho[NMAX], d0[8], d1[NN];
  const int4* r4 = reinterpret_cast<const int4*>(rho0);
  const int4* c0 = reinterpret_cast<const int4*>(delta);
  const int4* c1 = reinterpret_cast<const int4*>(delta + NMAX);
#pragma unroll
  for (int k = 0; k < NMAX / 4; ++k) {
    const int4 v = r4[k];
    rho[4 * k] = v.x;
    rho[4 * k + 1] = v.y;
    rho[4 * k + 2] = v.z;
    rho[4 * k + 3] = v.w;
  }
#pragma unroll
  for (int k = 0; k < 2; ++k) {
    const int4 u = c0[k];
    d0[4 * k] = u.x;
    d0[4 * k + 1] = u.y;
    d0[4 * k + 2] = u.z;
    d0[4 * k + 3] = u.w;
  }
#pragma unroll
  for (int k = 0; k < NN / 4; ++k) {
    const int4 w = c1[k];
    d1[4 * k] = w.x;
    d1[4 * k + 1] = w.y;
    d1[4 * k + 2] = w.z;
    d1[4 * k + 3] = w.w;
  }
  const uint64_t S = gb ^ (gb >> 1);
  for (int j = 0; j < m - 1; ++j) {
    if ((S >> j) & 1) {
      const int4* p = reinterpret_cast<const int4*>(delta + j * NMAX);
#pragma unroll
      for (int k = 0; k < NMAX / 4; ++k) {
        const int4 v = p[k];
        rho[4 * k] += v.x;
        rho[4 * k + 1] += v.y;
        rho[4 * k + 2] += v.z;
        rho[4 * k + 3] += v.w;
      }
    }
  }
  T acc = wide_from64(0, (T*)nullptr);
  const uint64_t ge = gb + cnt;
  for (uint64_t g = gb;;) {
    const int32_t s1 = ((g >> 2) & 1) ? -1 : 1;
    if constexpr (SPLIT4) {
      // |rho| < 2^7: quads below 2^28, their differences below 2^29, sn below 2^58
      const int32_t a0 = prod4<NMAX>(rho, 0), b0 = prod4<NMAX>(rho, 4);
#pragma unroll
      for (int i = 0; i < 4; ++i) rho[i] += d0[i];
      const int32_t a1 = prod4<NMAX>(rho, 0);
      reg_update<8, NMAX, BR>(rho, d1, s1 < 0);
      const int32_t a2 = prod4<NMAX>(rho, 0), b2 = prod4<NMAX>(rho, 4);
#pragma unroll
      for (int i = 0; i < 4; ++i) rho[i] -= d0[i];
      const int32_t a3 = prod4<NMAX>(rho, 0);
      const int64_t sn = (int64_t)(a0 - a1) * b0 + (int64_t)(a2 - a3) * b2;
      if constexpr (GZ == 0) {
        wide_add(acc, wide_from64(sn, (T*)nullptr));
      } else if constexpr (GZ == 1) {
        wide_add(acc, wide_mul64x64(sn, prod8<NMAX>(rho, NN), (T*)nullptr));
      } else {
        wide_add(acc, wide_mul64(prod_groups<NMAX, W, NN, GZ>(rho), sn));
      }
    } else if constexpr (GN == 1) {
      const int64_t n0 = prod8<NMAX>(rho, 0);
#pragma unroll
      for (int i = 0; i < NN; ++i) rho[i] += d0[i];
      const int64_t n1 = prod8<NMAX>(rho, 0);
      reg_update<NN, NMAX, BR>(rho, d1, s1 < 0);
      const int64_t n2 = prod8<NMAX>(rho, 0);
#pragma unroll
      for (int i = 0; i < NN; ++i) rho[i] -= d0[i];
      const int64_t n3 = prod8<NMAX>(rho, 0);
      const int64_t sn = (n0 - n1) + (n2 - n3);  // |n_t| < 2^56
      if constexpr (GZ == 0) {
        wide_add(acc, wide_from64(sn, (T*)nullptr));
      } else if constexpr (GZ == 1) {
        wide_add(acc, wide_mul64x64(sn, prod8<NMAX>(rho, NN), (T*)nullptr));
      } else {
        wide_add(acc, wide_mul64(prod_groups<NMAX, W, NN, GZ>(rho), sn));
      }
    } else {
      static_assert(GN == 2, "N groups of 8 and 8");
      const int64_t a0 = prod8<NMAX>(rho, 0);
      const int64_t b0 = prod8<NMAX>(rho, 8);
#pragma unroll
      for (int i = 0; i < 8; ++i) rho[i] += d0[i];
      const int64_t a1 = prod8<NMAX>(rho, 0);
      reg_update<NN, NMAX, BR>(rho, d1, s1 < 0);
      const int64_t a2 = prod8<NMAX>(rho, 0);
      const int64_t b2 = prod8<NMAX>(rho, 8);
#pragma unroll
      for (int i = 0; i < 8; ++i) rho[i] -= d0[i];
      const int64_t a3 = prod8<NMAX>(rho, 0);
      // |a_t| < 2^56, so the differences fit 64 bits
      T sn = wide_mul64x64(a0 - a1, b0, (T*)nullptr);
      wide_add(sn, wide_mul64x64(a2 - a3, b2, (T*)nullptr));
      if constexpr (GZ == 0) {
        wide_add(acc, sn);
      } else if constexpr (GZ == 1) {
        wide_add(acc, wide_mul64(sn, prod8<NMAX>(rho, NN)));
      } else {
        wide_add(acc, wide_mulTT(sn, prod_groups<NMAX, W, NN, GZ>(rho)));
      }
    }
    g += 4;
    if (g >= ge) break;
    const int j = __ffsll((long long)g) - 1;  // >= 2
    col_update<NMAX, BR>(rho, delta + j * NMAX, (g >> (j + 1)) & 1);
  }
  return acc;
}

// Lane share of the blocked walk, warp-summed into lane 0.
template <int NMAX, int NN, int W, bool SPLIT4 = false, bool BR = true>
__device__ __forceinline__ void run_lane4(const int32_t* delta, const int32_t* rho0, int m, uint64_t gb,
                                          uint64_t cnt, uint64_t* words) {
  typename WideT<W>::type s = ryser_lane4<NMAX, NN, W, SPLIT4, BR>(delta, rho0, m, gb, cnt);
  s = warp_sum(s);
  to_words(s, words);
}
