// One node of Eq. 2 (Section 2.1): the child specification and the rows of
// a child built from its parent's CSR block.  Shared by the level-by-level
// expansion (expand.cu) and the work-distributing traversal (walk.cu), so
// both produce the same children.
#pragma once
#include <cstdint>

#include "jobs.cuh"
#include "modp.cuh"

// checked a*x + b*y in int64; with a modulus (the residue path, all four
// operands residues) the result reduced modulo it, which cannot overflow
__device__ __forceinline__ bool mad2_checked(int64_t a, int64_t x, int64_t b, int64_t y, int64_t& out,
                                             uint32_t mod = 0) {
  if (mod) {
    out = (int64_t)mod_mad2((uint64_t)a, (uint64_t)x, (uint64_t)b, (uint64_t)y, mod);
    return true;
  }
  __int128 r = (__int128)a * x + (__int128)b * y;
  out = (int64_t)r;
  return r == (__int128)out;
}

struct ChildSpec {
  int del_row, del_col;  // kNone for the cleared child
  int merge;      // 0 none, 1 column p merged (row pivot), 2 row p merged (column pivot),
                  // 3 the pivot line's entries at zp[0..3] cleared (nothing deleted)
  int p, q;       // merged line and its partner (deleted), p < q
  int64_t a, b;   // merged line = a * line_q + b * line_p
  int64_t fac;    // scalar factor (minor)
  int zcol, zidx; // merge 3: pivot is a column (1) or a row (0), and its index
  int zp[4];      // merge 3: the cleared positions along the pivot line
  uint32_t mod;   // 0, or the residue path's modulus (merged entries reduced modulo it)
};

constexpr int kNone = 1 << 30;

// The nonzeros of one child row (parent row r), in ascending child column
// order, passed to emit(col, value).  False on int64 overflow.
template <class F>
__device__ __forceinline__ bool child_row(const CsrView& v, const ChildSpec& cs, int r, F&& emit) {
  const int b = v.rowptr[r], e = v.rowptr[r + 1];
  bool ok = true;
  if (cs.merge == 1) {
    int64_t xp = 0, xq = 0;
    for (int t = b; t < e; ++t) {
      const int c = v.col[t];
      if (c == cs.p) xp = v.val[t];
      if (c == cs.q) xq = v.val[t];
    }
    int64_t mv;
    ok = mad2_checked(cs.a, xq, cs.b, xp, mv, cs.mod);
    bool done = false;
    for (int t = b; t < e; ++t) {
      const int c = v.col[t];
      if (!done && c >= cs.p) {
        if (mv != 0) emit(cs.p, mv);
        done = true;
        if (c == cs.p) continue;
      }
      if (c == cs.q) continue;
      emit(c - (c > cs.q), v.val[t]);
    }
    if (!done && mv != 0) emit(cs.p, mv);
  } else if (cs.merge == 3) {
    // the cleared child: row zidx loses columns zp (row pivot), or rows zp
    // lose column zidx (column pivot)
    const bool rowhit = !cs.zcol && r == cs.zidx;
    const bool colhit = cs.zcol && (r == cs.zp[0] || r == cs.zp[1] || r == cs.zp[2] || r == cs.zp[3]);
    for (int t = b; t < e; ++t) {
      const int c = v.col[t];
      if (rowhit && (c == cs.zp[0] || c == cs.zp[1] || c == cs.zp[2] || c == cs.zp[3])) continue;
      if (colhit && c == cs.zidx) continue;
      emit(c, v.val[t]);
    }
  } else if (cs.merge == 2 && r == cs.p) {
    const int bq = v.rowptr[cs.q], eq = v.rowptr[cs.q + 1];
    int i = b, j = bq;
    while (i < e || j < eq) {
      const int ci = i < e ? v.col[i] : 0x7fffffff;
      const int cj = j < eq ? v.col[j] : 0x7fffffff;
      const int c = ci < cj ? ci : cj;
      const int64_t xp = ci == c ? v.val[i++] : 0;
      const int64_t xq = cj == c ? v.val[j++] : 0;
      if (c == cs.del_col) continue;
      int64_t mv;
      if (!mad2_checked(cs.a, xq, cs.b, xp, mv, cs.mod)) ok = false;
      if (mv != 0) emit(c - (c > cs.del_col), mv);
    }
  } else {
    for (int t = b; t < e; ++t) {
      const int c = v.col[t];
      if (c == cs.del_col) continue;
      emit(c - (c > cs.del_col), v.val[t]);
    }
  }
  return ok;
}

