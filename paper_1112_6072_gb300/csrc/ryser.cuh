// Leaf evaluator: Ryser's formula in the Nijenhuis-Wilf form with a Gray code
// (the R-NW algorithm of Section 1, O(n 2^(n-1))), in exact integers.
//
// For an m x m matrix A, with doubled row sums
//     rho_i(S) = 2 a_{i,m-1} - sum_j a_ij + 2 sum_{j in S} a_ij,
// S ranging over subsets of the first m-1 columns,
//     Sigma = sum_S (-1)^|S| prod_i rho_i(S) = (-1)^(m-1) 2^(m-1) per(A).
// S runs through the binary reflected Gray code: step g flips column ctz(g)
// (in if bit ctz(g)+1 of g is 0, out otherwise) and (-1)^|gray(g)| = (-1)^g.
// A lane walks a contiguous, aligned block of 2^c codes, so every lane of a
// warp flips the same column at the same step: the column is read from
// shared memory as a broadcast, and the direction is uniform except at one
// step per block.  Column 0 flips on every odd step; its values stay in
// registers.
//
// Exactness: |rho_i(S)| <= R_i = sum_j |a_ij| for every S, so rho fits int32
// when R < 2^31.  Products are formed in a tree whose lower levels stay in
// 32 and 64 bits (the bit class BC bounds log2 R) and whose top is modulo
// 2^(64W); the sum over S is taken modulo 2^(64W) as well.
#pragma once
#include <cstdint>

#include "wide.cuh"

template <int W>
struct WideT;
template <>
struct WideT<2> {
  typedef u128 type;
};
template <>
struct WideT<4> {
  typedef u256 type;
};

__device__ __forceinline__ u128 wide_zero2() { return (u128)0; }

__device__ __forceinline__ void wide_add(u128& a, u128 b) { a += b; }
__device__ __forceinline__ void wide_sub(u128& a, u128 b) { a -= b; }
__device__ __forceinline__ void wide_add(u256& a, const u256& b) { a = u256_add(a, b); }
__device__ __forceinline__ void wide_sub(u256& a, const u256& b) { a = u256_sub(a, b); }

__device__ __forceinline__ u128 wide_from64(int64_t v, u128*) { return (u128)(__int128)v; }
__device__ __forceinline__ u256 wide_from64(int64_t v, u256*) { return u256_from_s64(v); }

__device__ __forceinline__ u128 wide_mul64(u128 a, int64_t b) { return mul128_s64(a, b); }
__device__ __forceinline__ u256 wide_mul64(const u256& a, int64_t b) { return u256_mul_s64(a, b); }

// Product of the first two 64-bit factors straight into the wide ring.
__device__ __forceinline__ u128 wide_mul64x64(int64_t a, int64_t b, u128*) { return mul_s64_s64(a, b); }
__device__ __forceinline__ u256 wide_mul64x64(int64_t a, int64_t b, u256*) {
  u128 p = mul_s64_s64(a, b);
  u256 r;
  r.w[0] = (uint64_t)p;
  r.w[1] = (uint64_t)(p >> 64);
  uint64_t s = ((int64_t)r.w[1] < 0) ? ~0ull : 0ull;
  r.w[2] = r.w[3] = s;
  return r;
}

// 64-bit partial products of NMAX row sums for bit class BC:
//   BC = 7 : |rho| < 2^7  -> 4 per int32, 8 per int64
//   BC = 15: |rho| < 2^15 -> 2 per int32, 4 per int64
//   BC = 31: |rho| < 2^31 -> 2 per int64
template <int NMAX, int BC>
struct ProdPlan {
  static constexpr int PER64 = BC == 7 ? 8 : (BC == 15 ? 4 : 2);
  static constexpr int N64 = (NMAX + PER64 - 1) / PER64;
};

template <int NMAX, int BC>
__device__ __forceinline__ void partial64(const int32_t (&r)[NMAX],
                                          int64_t (&o)[ProdPlan<NMAX, BC>::N64]) {
  constexpr int PER64 = ProdPlan<NMAX, BC>::PER64;
  constexpr int N64 = ProdPlan<NMAX, BC>::N64;
#pragma unroll
  for (int k = 0; k < N64; ++k) {
    const int b = k * PER64;
    if (BC == 7) {
      int32_t q0 = r[b] * r[b + 1] * r[b + 2] * r[b + 3];
      int32_t q1 = (b + 4 < NMAX) ? r[b + 4] * r[b + 5] * r[b + 6] * r[b + 7] : 1;
      o[k] = (int64_t)q0 * (int64_t)q1;
    } else if (BC == 15) {
      int32_t p0 = r[b] * r[b + 1];
      int32_t p1 = r[b + 2] * r[b + 3];
      o[k] = (int64_t)p0 * (int64_t)p1;
    } else {
      o[k] = (int64_t)r[b] * (int64_t)r[b + 1];
    }
  }
}

template <int NMAX, int W, int BC>
__device__ __forceinline__ typename WideT<W>::type row_product(const int32_t (&r)[NMAX]) {
  typedef typename WideT<W>::type T;
  constexpr int N64 = ProdPlan<NMAX, BC>::N64;
  int64_t o[N64];
  partial64<NMAX, BC>(r, o);
  T p;
  if (N64 == 1) {
    p = wide_from64(o[0], (T*)nullptr);
  } else {
    p = wide_mul64x64(o[0], o[1], (T*)nullptr);
#pragma unroll
    for (int k = 2; k < N64; ++k) p = wide_mul64(p, o[k]);
  }
  return p;
}

// rho -= col or rho += col over NMAX slots (col 16-byte aligned in shared
// memory).  BR: the direction is a branch, not a multiply by +-1, so the
// updates are plain integer adds on the ALU pipe, leaving the multiply pipe
// to the row products (the direction is uniform across the warp at all but
// one step of a lane's block of codes).  The leaf kernels take the branch;
// the depth-first evaluator, whose leaves sit in a larger kernel, keeps the
// shorter multiply form.
template <int NMAX, bool BR>
__device__ __forceinline__ void col_update(int32_t (&rho)[NMAX], const int32_t* __restrict__ col, bool neg) {
  const int4* p = reinterpret_cast<const int4*>(col);
  if constexpr (!BR) {
    const int32_t s = neg ? -1 : 1;
#pragma unroll
    for (int k = 0; k < NMAX / 4; ++k) {
      const int4 v = p[k];
      rho[4 * k] += s * v.x;
      rho[4 * k + 1] += s * v.y;
      rho[4 * k + 2] += s * v.z;
      rho[4 * k + 3] += s * v.w;
    }
  } else if (neg) {
#pragma unroll
    for (int k = 0; k < NMAX / 4; ++k) {
      const int4 v = p[k];
      rho[4 * k] -= v.x;
      rho[4 * k + 1] -= v.y;
      rho[4 * k + 2] -= v.z;
      rho[4 * k + 3] -= v.w;
    }
  } else {
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

// the same for N register values
template <int N, int NMAX, bool BR>
__device__ __forceinline__ void reg_update(int32_t (&rho)[NMAX], const int32_t* d, bool neg) {
  if constexpr (!BR) {
    const int32_t s = neg ? -1 : 1;
#pragma unroll
    for (int i = 0; i < N; ++i) rho[i] += s * d[i];
  } else if (neg) {
#pragma unroll
    for (int i = 0; i < N; ++i) rho[i] -= d[i];
  } else {
#pragma unroll
    for (int i = 0; i < N; ++i) rho[i] += d[i];
  }
}

// One lane's share of Sigma: codes g in [gb, gb + cnt), gb and cnt even.
// delta: shared memory, column j at delta[j * NMAX + i] = 2 a_ij (j < m-1),
// rows i >= m zero.  rho0: shared, rho_i(empty), rows i >= m equal to 1.
template <int NMAX, int W, int BC, bool BR = true>
__device__ __forceinline__ typename WideT<W>::type ryser_lane(const int32_t* __restrict__ delta,
                                                              const int32_t* __restrict__ rho0, int m,
                                                              uint64_t gb, uint64_t cnt) {
  typedef typename WideT<W>::type T;
  if (cnt == 0) return wide_from64(0, (T*)nullptr);
  int32_t rho[NMAX], d0[NMAX];
  const int4* r4 = reinterpret_cast<const int4*>(rho0);
  const int4* c4 = reinterpret_cast<const int4*>(delta);
#pragma unroll
  for (int k = 0; k < NMAX / 4; ++k) {
    int4 v = r4[k];
    rho[4 * k] = v.x;
    rho[4 * k + 1] = v.y;
    rho[4 * k + 2] = v.z;
    rho[4 * k + 3] = v.w;
    int4 u = c4[k];
    d0[4 * k] = u.x;
    d0[4 * k + 1] = u.y;
    d0[4 * k + 2] = u.z;
    d0[4 * k + 3] = u.w;
  }
  // rho at S = gray(gb)
  const uint64_t S = gb ^ (gb >> 1);
  for (int j = 0; j < m - 1; ++j) {
    if ((S >> j) & 1) {
      const int4* p = reinterpret_cast<const int4*>(delta + j * NMAX);
#pragma unroll
      for (int k = 0; k < NMAX / 4; ++k) {
        int4 v = p[k];
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
    // even code g: +prod
    wide_add(acc, row_product<NMAX, W, BC>(rho));
    // odd code g+1 flips column 0; it enters S iff bit 1 of g+1 is 0
    reg_update<NMAX, NMAX, BR>(rho, d0, (g >> 1) & 1);
    wide_sub(acc, row_product<NMAX, W, BC>(rho));
    g += 2;
    if (g >= ge) break;
    // even code g flips column j = ctz(g) >= 1
    const int j = __ffsll((long long)g) - 1;
    col_update<NMAX, BR>(rho, delta + j * NMAX, (g >> (j + 1)) & 1);
  }
  return acc;
}

// Warp sum of the lanes' residues into lane 0.
__device__ __forceinline__ u128 warp_sum(u128 v) {
#pragma unroll
  for (int d = 16; d > 0; d >>= 1) v += shfl_down_u128(v, d);
  return v;
}
__device__ __forceinline__ u256 warp_sum(u256 v) {
#pragma unroll
  for (int d = 16; d > 0; d >>= 1) v = u256_add(v, shfl_down_u256(v, d));
  return v;
}

__device__ __forceinline__ void to_words(u128 v, uint64_t* w) {
  w[0] = (uint64_t)v;
  w[1] = (uint64_t)(v >> 64);
  w[2] = w[3] = 0;
}
__device__ __forceinline__ void to_words(const u256& v, uint64_t* w) {
  w[0] = v.w[0];
  w[1] = v.w[1];
  w[2] = v.w[2];
  w[3] = v.w[3];
}

// Lane share for (NMAX, W) with the bit class chosen at run time, summed over
// the warp into lane 0 as four little-endian words.
template <int NMAX, int W>
__device__ __forceinline__ void run_lane(int bc, const int32_t* delta, const int32_t* rho0, int m, uint64_t gb,
                                         uint64_t cnt, uint64_t* words) {
  typedef typename WideT<W>::type T;
  T s;
  if (bc == 7)
    s = ryser_lane<NMAX, W, 7>(delta, rho0, m, gb, cnt);
  else if (bc == 15)
    s = ryser_lane<NMAX, W, 15>(delta, rho0, m, gb, cnt);
  else
    s = ryser_lane<NMAX, W, 31>(delta, rho0, m, gb, cnt);
  s = warp_sum(s);
  to_words(s, words);
}

__device__ __forceinline__ void dispatch_lane(int nmax, int W, int bc, const int32_t* delta, const int32_t* rho0,
                                              int m, uint64_t gb, uint64_t cnt, uint64_t* words) {
  if (W == 2) {
    switch (nmax) {
      case 8: run_lane<8, 2>(bc, delta, rho0, m, gb, cnt, words); break;
      case 16: run_lane<16, 2>(bc, delta, rho0, m, gb, cnt, words); break;
      case 24: run_lane<24, 2>(bc, delta, rho0, m, gb, cnt, words); break;
      default: run_lane<32, 2>(bc, delta, rho0, m, gb, cnt, words); break;
    }
  } else {
    switch (nmax) {
      case 8: run_lane<8, 4>(bc, delta, rho0, m, gb, cnt, words); break;
      case 16: run_lane<16, 4>(bc, delta, rho0, m, gb, cnt, words); break;
      case 24: run_lane<24, 4>(bc, delta, rho0, m, gb, cnt, words); break;
      default: run_lane<32, 4>(bc, delta, rho0, m, gb, cnt, words); break;
    }
  }
}

// Bit class of a leaf from its largest absolute row sum R (R < 2^31).
__host__ __device__ __forceinline__ int bit_class(int64_t R) { return R < 128 ? 7 : (R < 32768 ? 15 : 31); }
// Smallest register width (8, 16, 24, 32) holding m rows.
__host__ __device__ __forceinline__ int nmax_for(int m) { return m <= 8 ? 8 : (m <= 16 ? 16 : (m <= 24 ? 24 : 32)); }
