// Eq. 2 (Section 2.1) in place on a dense tile: the node machinery of the
// depth-first walks (the evaluator dfs.cu and the expansion walk.cu).
//
// A job is loaded once into a dense TILE x TILE tile in shared memory.
// Lines are never moved: deleting a row or column clears a bit of the
// active masks R and C, so "lowest index" keeps the meaning it has in the
// compacted matrices.  A merge overwrites one line in place after saving it
// to a frame of the warp's undo stack in global memory; backtracking
// restores it.  Nonzero patterns are kept as bit masks per row (rowbits) and
// per column (colbits), so a line count is one popcount against the active
// masks.  With the three-child option, Eq. 2's third child clears the pivot
// line's first four entries in place (the frame holds their values).  On
// the residue path (modp != 0) the entries are residues modulo modp and
// merged entries and coefficients are reduced modulo modp.
#pragma once
#include <cstdint>

#include "modp.cuh"
#include "wide.cuh"

template <int TILE, typename E>
struct TileCfg {
  static constexpr int STRIDE = TILE + 1;
  static constexpr size_t TILE_BYTES = (sizeof(E) * TILE * STRIDE + 15) / 16 * 16;
  static constexpr size_t MASK_BYTES = 2 * sizeof(uint64_t) * TILE;
  // undo stack words per level: meta (8 x int32 = 4 words), pv[4], coef[4], saved mask, line[TILE]
  static constexpr int FRAME_WORDS = 4 + 4 + 4 + 1 + TILE;
};

struct Frame {
  int32_t is_col, idx, k, child;
  int32_t pos[4];
};

// a*x + b*y, false when the result leaves E.  In an int32 tile all four
// operands are tile entries (|v| < 2^31), so int64 holds the sum exactly.
template <typename E>
__device__ __forceinline__ bool tile_mad2(int64_t a, int64_t x, int64_t b, int64_t y, E& out) {
  if constexpr (sizeof(E) == 4) {
    const int64_t r = a * x + b * y;
    out = (E)r;
    return r == (int64_t)out;
  } else {
    const __int128 r = (__int128)a * x + (__int128)b * y;
    out = (E)r;
    return r == (__int128)out;
  }
}

// index of the (n+1)-th set bit of a 64-bit mask
__device__ __forceinline__ int nth_bit(uint64_t mask, int n) {
  const uint32_t lo = (uint32_t)mask;
  const int plo = __popc(lo);
  if (n < plo) return __fns(lo, 0, n + 1);
  return 32 + __fns((uint32_t)(mask >> 32), 0, n - plo + 1);
}

__device__ __forceinline__ uint64_t bit64(int i) { return 1ull << i; }

template <int TILE, typename E>
struct Eq2Tile {
  static constexpr int S = TileCfg<TILE, E>::STRIDE;
  static constexpr int RPL = TILE / 32;  // lines per lane
  E* T;
  uint64_t* rowbits;
  uint64_t* colbits;
  int64_t* undo;
  int lane;
  uint64_t R, C;
  u256 coef;
  uint32_t modp = 0;  // 0: exact entries; else residues modulo this prime

  // a*x + b*y into a tile entry (false when it leaves E; never on the residue path)
  __device__ __forceinline__ bool mad2(int64_t a, int64_t x, int64_t b, int64_t y, E& out) const {
    if (modp) {
      out = (E)mod_mad2((uint64_t)a, (uint64_t)x, (uint64_t)b, (uint64_t)y, modp);
      return true;
    }
    return tile_mad2<E>(a, x, b, y, out);
  }
  // coef *= v (Eq. 2's scalar factor of a minor)
  __device__ __forceinline__ void mul_coef(int64_t v) {
    if (modp)
      coef.w[0] = coef.w[0] % modp * (uint64_t)v % modp;
    else
      coef = u256_mul_s64(coef, v);
  }

  __device__ int64_t* frame_words(int lv) { return undo + (int64_t)lv * TileCfg<TILE, E>::FRAME_WORDS; }

  __device__ void store_frame(int lv, const Frame& f, const int64_t* pv, const u256& c) {
    int64_t* w = frame_words(lv);
    if (lane == 0) {
      int32_t* m = reinterpret_cast<int32_t*>(w);
      m[0] = f.is_col;
      m[1] = f.idx;
      m[2] = f.k;
      m[3] = f.child;
      for (int t = 0; t < 4; ++t) m[4 + t] = f.pos[t];
      for (int t = 0; t < 4; ++t) w[4 + t] = pv[t];
      for (int t = 0; t < 4; ++t) w[8 + t] = (int64_t)c.w[t];
    }
  }
  __device__ void load_frame(int lv, Frame& f, int64_t* pv, u256& c) {
    const int64_t* w = frame_words(lv);
    const int32_t* m = reinterpret_cast<const int32_t*>(w);
    f.is_col = m[0];
    f.idx = m[1];
    f.k = m[2];
    f.child = m[3];
    for (int t = 0; t < 4; ++t) f.pos[t] = m[4 + t];
    for (int t = 0; t < 4; ++t) pv[t] = w[4 + t];
    for (int t = 0; t < 4; ++t) c.w[t] = (uint64_t)w[8 + t];
  }
  __device__ void set_child(int lv, int child) {
    if (lane == 0) reinterpret_cast<int32_t*>(frame_words(lv))[3] = child;
  }

  // child c of a frame: kind 1 = merge(pos[x], pos[x+1]), 2 = minor(pos[x]),
  // 3 = the pivot line's entries at pos[0..3] cleared (k >= 5)
  __device__ static void child_kind(int k, int c, int& kind, int& x) {
    if (c == 0) {
      kind = k == 1 ? 2 : 1;
      x = 0;
    } else if (c == 1) {
      kind = k == 3 ? 2 : 1;
      x = 2;
    } else {
      kind = 3;
      x = 0;
    }
  }
  __device__ static int nchildren(int k) { return k >= 5 ? 3 : ((k == 3 || k == 4) ? 2 : 1); }

  // the pivot line's entries at pos[0..3] set to 0 (clear) or back to pv
  __device__ void clear_four(const Frame& f, const int64_t* pv, bool restore) {
    if (lane < 4) {
      const int t = lane;
      const int at = f.pos[t];
      if (!f.is_col) {
        T[f.idx * S + at] = restore ? (E)pv[t] : (E)0;
        if (restore) colbits[at] |= bit64(f.idx); else colbits[at] &= ~bit64(f.idx);
      } else {
        T[at * S + f.idx] = restore ? (E)pv[t] : (E)0;
        if (restore) rowbits[at] |= bit64(f.idx); else rowbits[at] &= ~bit64(f.idx);
      }
    }
    if (lane == 0) {
      const uint64_t m4 = bit64(f.pos[0]) | bit64(f.pos[1]) | bit64(f.pos[2]) | bit64(f.pos[3]);
      uint64_t* line = f.is_col ? &colbits[f.idx] : &rowbits[f.idx];
      *line = restore ? (*line | m4) : (*line & ~m4);
    }
    __syncwarp();
  }

  // Apply child c; returns false when a merged entry leaves E.
  __device__ bool apply(int lv, const Frame& f, const int64_t* pv, int c) {
    return apply_to(frame_words(lv) + 13, f, pv, c);
  }
  // The same with the overwritten line saved at saved[0 .. TILE) and its
  // mask at saved[-1] (a frame of the undo stack, or a scratch line).
  __device__ bool apply_to(int64_t* saved, const Frame& f, const int64_t* pv, int c) {
    int kind, x;
    child_kind(f.k, c, kind, x);
    if (kind == 3) {
      clear_four(f, pv, false);
      return true;
    }
    bool ok = true;
    if (!f.is_col) {
      const int i = f.idx;
      if (kind == 2) {
        R &= ~bit64(i);
        C &= ~bit64(f.pos[x]);
        mul_coef(pv[x]);
        return true;
      }
      const int p = f.pos[x], q = f.pos[x + 1];
      const int64_t a = pv[x], b = pv[x + 1];
      R &= ~bit64(i);
      C &= ~bit64(q);
      uint64_t nzbits = 0;
#pragma unroll
      for (int t = 0; t < RPL; ++t) {
        const int r = lane + 32 * t;
        bool nz = false;
        if ((R >> r) & 1) {
          const E old = T[r * S + p];
          E nv;
          if (!mad2(a, T[r * S + q], b, old, nv)) ok = false;
          saved[r] = old;
          T[r * S + p] = nv;
          nz = nv != 0;
          if (nz) rowbits[r] |= bit64(p); else rowbits[r] &= ~bit64(p);
        }
        const uint32_t bal = __ballot_sync(0xffffffffu, nz);
        nzbits |= (uint64_t)bal << (32 * t);
      }
      if (lane == 0) {
        saved[-1] = (int64_t)colbits[p];
        colbits[p] = nzbits;
      }
    } else {
      const int j = f.idx;
      if (kind == 2) {
        C &= ~bit64(j);
        R &= ~bit64(f.pos[x]);
        mul_coef(pv[x]);
        return true;
      }
      const int p = f.pos[x], q = f.pos[x + 1];
      const int64_t a = pv[x], b = pv[x + 1];
      C &= ~bit64(j);
      R &= ~bit64(q);
      uint64_t nzbits = 0;
#pragma unroll
      for (int t = 0; t < RPL; ++t) {
        const int cc = lane + 32 * t;
        bool nz = false;
        if ((C >> cc) & 1) {
          const E old = T[p * S + cc];
          E nv;
          if (!mad2(a, T[q * S + cc], b, old, nv)) ok = false;
          saved[cc] = old;
          T[p * S + cc] = nv;
          nz = nv != 0;
          if (nz) colbits[cc] |= bit64(p); else colbits[cc] &= ~bit64(p);
        }
        const uint32_t bal = __ballot_sync(0xffffffffu, nz);
        nzbits |= (uint64_t)bal << (32 * t);
      }
      if (lane == 0) {
        saved[-1] = (int64_t)rowbits[p];
        rowbits[p] = nzbits;
      }
    }
    __syncwarp();
    return __all_sync(0xffffffffu, ok);
  }

  __device__ void undo_child(int lv, const Frame& f, const int64_t* pv, const u256& pcoef, int c) {
    undo_from(frame_words(lv) + 13, f, pv, pcoef, c);
  }
  __device__ void undo_from(const int64_t* saved, const Frame& f, const int64_t* pv, const u256& pcoef, int c) {
    int kind, x;
    child_kind(f.k, c, kind, x);
    coef = pcoef;
    if (kind == 3) {
      clear_four(f, pv, true);
      return;
    }
    if (!f.is_col) {
      const int i = f.idx;
      R |= bit64(i);
      if (kind == 2) {
        C |= bit64(f.pos[x]);
        return;
      }
      const int p = f.pos[x], q = f.pos[x + 1];
      C |= bit64(q);
#pragma unroll
      for (int t = 0; t < RPL; ++t) {
        const int r = lane + 32 * t;
        if (r != i && ((R >> r) & 1)) {
          const E old = (E)saved[r];
          T[r * S + p] = old;
          if (old != 0) rowbits[r] |= bit64(p); else rowbits[r] &= ~bit64(p);
        }
      }
      if (lane == 0) colbits[p] = (uint64_t)saved[-1];
    } else {
      const int j = f.idx;
      C |= bit64(j);
      if (kind == 2) {
        R |= bit64(f.pos[x]);
        return;
      }
      const int p = f.pos[x], q = f.pos[x + 1];
      R |= bit64(q);
#pragma unroll
      for (int t = 0; t < RPL; ++t) {
        const int cc = lane + 32 * t;
        if (cc != j && ((C >> cc) & 1)) {
          const E old = (E)saved[cc];
          T[p * S + cc] = old;
          if (old != 0) colbits[cc] |= bit64(p); else colbits[cc] &= ~bit64(p);
        }
      }
      if (lane == 0) rowbits[p] = (uint64_t)saved[-1];
    }
    __syncwarp();
  }

  // smallest line count over the active lines: (s << 17) | (is_col << 16) | index
  // (s <= 64, index < 64: 24 bits), one warp-wide min reduction
  __device__ unsigned long long pivot_key() {
    unsigned key = 0xffffffffu;
#pragma unroll
    for (int t = 0; t < RPL; ++t) {
      const int r = lane + 32 * t;
      if ((R >> r) & 1) key = min(key, ((unsigned)__popcll(rowbits[r] & C) << 17) | (unsigned)r);
      if ((C >> r) & 1) key = min(key, ((unsigned)__popcll(colbits[r] & R) << 17) | (1u << 16) | (unsigned)r);
    }
    return (unsigned long long)__reduce_min_sync(0xffffffffu, key);
  }

};
