// Leaf evaluator of the residue path: the Gray-code walk of ryser.cuh
// (Ryser's formula in the Nijenhuis-Wilf form, Section 1) with every value
// a residue modulo p in Montgomery form (modp.cuh).
//
// delta[j * NMAX + i] = 2 a_ij R mod p (j < m-1), rho0[i] = rho_i(empty) R
// mod p for i < m and R mod p (the Montgomery 1) for i >= m, so that
//     Sigma = sum_S (-1)^|S| prod_i rho_i(S) = (-1)^(m-1) 2^(m-1) per(A)  (mod p)
// and per(A) = (-1)^(m-1) Sigma (2^-1)^(m-1) mod p, 2 being invertible
// modulo the odd prime p.
#pragma once
#include <cstdint>

#include "modp.cuh"

// product of the NMAX row sums (Montgomery form), as a balanced tree
template <int NMAX>
__device__ __forceinline__ uint32_t row_product_mod(const uint32_t (&r)[NMAX], const ModP& M) {
  uint32_t t[NMAX];
#pragma unroll
  for (int i = 0; i < NMAX; ++i) t[i] = r[i];
#pragma unroll
  for (int w = 1; w < NMAX; w <<= 1)
#pragma unroll
    for (int i = 0; i + w < NMAX; i += 2 * w) t[i] = mont_mul(t[i], t[i + w], M);
  return t[0];
}

template <int NMAX>
__device__ __forceinline__ void rows_step_mod(uint32_t (&rho)[NMAX], const uint32_t* __restrict__ col, bool sub,
                                              uint32_t p) {
  const uint4* c4 = reinterpret_cast<const uint4*>(col);
#pragma unroll
  for (int k = 0; k < NMAX / 4; ++k) {
    const uint4 v = c4[k];
    if (sub) {
      rho[4 * k] = mod_sub(rho[4 * k], v.x, p);
      rho[4 * k + 1] = mod_sub(rho[4 * k + 1], v.y, p);
      rho[4 * k + 2] = mod_sub(rho[4 * k + 2], v.z, p);
      rho[4 * k + 3] = mod_sub(rho[4 * k + 3], v.w, p);
    } else {
      rho[4 * k] = mod_add(rho[4 * k], v.x, p);
      rho[4 * k + 1] = mod_add(rho[4 * k + 1], v.y, p);
      rho[4 * k + 2] = mod_add(rho[4 * k + 2], v.z, p);
      rho[4 * k + 3] = mod_add(rho[4 * k + 3], v.w, p);
    }
  }
}

// One lane's share of Sigma (Montgomery form): codes g in [gb, gb + cnt),
// gb and cnt even, walked as in ryser_lane.
template <int NMAX>
__device__ __forceinline__ uint32_t ryser_lane_mod(const uint32_t* __restrict__ delta,
                                                   const uint32_t* __restrict__ rho0, int m, uint64_t gb,
                                                   uint64_t cnt, const ModP& M) {
  if (cnt == 0) return 0;
  const uint32_t p = M.p;
  uint32_t rho[NMAX], d0[NMAX];
  const uint4* r4 = reinterpret_cast<const uint4*>(rho0);
  const uint4* c4 = reinterpret_cast<const uint4*>(delta);
#pragma unroll
  for (int k = 0; k < NMAX / 4; ++k) {
    const uint4 v = r4[k];
    rho[4 * k] = v.x;
    rho[4 * k + 1] = v.y;
    rho[4 * k + 2] = v.z;
    rho[4 * k + 3] = v.w;
    const uint4 u = c4[k];
    d0[4 * k] = u.x;
    d0[4 * k + 1] = u.y;
    d0[4 * k + 2] = u.z;
    d0[4 * k + 3] = u.w;
  }
  // rho at S = gray(gb)
  const uint64_t S = gb ^ (gb >> 1);
  for (int j = 0; j < m - 1; ++j)
    if ((S >> j) & 1) rows_step_mod<NMAX>(rho, delta + j * NMAX, false, p);
  uint32_t acc = 0;
  const uint64_t ge = gb + cnt;
  for (uint64_t g = gb;;) {
    // even code g: +prod
    acc = mod_add(acc, row_product_mod<NMAX>(rho, M), p);
    // odd code g+1 flips column 0: in iff bit 1 of g+1 is 0
    const bool out0 = (g >> 1) & 1;
#pragma unroll
    for (int i = 0; i < NMAX; ++i) rho[i] = out0 ? mod_sub(rho[i], d0[i], p) : mod_add(rho[i], d0[i], p);
    acc = mod_sub(acc, row_product_mod<NMAX>(rho, M), p);
    g += 2;
    if (g >= ge) break;
    // even code g flips column j = ctz(g) >= 1
    const int j = __ffsll((long long)g) - 1;
    rows_step_mod<NMAX>(rho, delta + j * NMAX, (g >> (j + 1)) & 1, p);
  }
  return acc;
}

// warp sum of the lanes' residues into lane 0
__device__ __forceinline__ uint32_t warp_sum_mod(uint32_t v, uint32_t p) {
#pragma unroll
  for (int d = 16; d > 0; d >>= 1) v = mod_add(v, __shfl_down_sync(0xffffffffu, v, d), p);
  return v;
}

// per = (-1)^(m-1) Sigma (2^-1)^(m-1) mod p, from Sigma (plain residue)
__host__ __device__ __forceinline__ uint32_t nw_per_mod(uint32_t sigma, int m, uint32_t p) {
  if (m < 2) return sigma % p;
  const uint32_t h = mod_pow((p + 1) / 2, (uint64_t)(m - 1), p);
  const uint32_t v = (uint32_t)((uint64_t)(sigma % p) * h % p);
  return ((m - 1) & 1) ? (v == 0 ? 0 : p - v) : v;
}
