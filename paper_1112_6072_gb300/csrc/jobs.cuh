// Device layout of a job set: the sub-matrices produced by Algorithm PH,
// Step 2 (Section 2.2), in natural order, each stored as a compact CSR block
// in one arena of 8-byte words.
//
// Block of a job of order m with nnz nonzeros, starting at word off[j]:
//   words [0, rp)        uint16 rowptr[m+1]            rp  = ceil((m+1)/4)
//   words [rp, rp+cw)    uint8  col[nnz]               cw  = ceil(nnz/8)
//   words [rp+cw, +nnz)  int64  val[nnz]
// rounded up to an even word count, so every block starts on 16 bytes and
// can be moved with 16-byte vector copies.  Rows are in order and the
// columns of a row ascend.
#pragma once
#include <cstdint>

#define PERM_WARPS_MAX 32

__host__ __device__ __forceinline__ int64_t blk_rp_words(int m) { return (m + 1 + 3) / 4; }
__host__ __device__ __forceinline__ int64_t blk_col_words(int nnz) { return (nnz + 7) / 8; }
__host__ __device__ __forceinline__ int64_t blk_words(int m, int nnz) {
  int64_t w = blk_rp_words(m) + blk_col_words(nnz) + nnz;
  return (w + 1) & ~(int64_t)1;
}

struct CsrView {
  const uint16_t* rowptr;
  const uint8_t* col;
  const int64_t* val;
};

__host__ __device__ __forceinline__ CsrView csr_view(const uint64_t* arena, int64_t off, int m, int nnz) {
  CsrView v;
  const uint64_t* b = arena + off;
  v.rowptr = reinterpret_cast<const uint16_t*>(b);
  v.col = reinterpret_cast<const uint8_t*>(b + blk_rp_words(m));
  v.val = reinterpret_cast<const int64_t*>(b + blk_rp_words(m) + blk_col_words(nnz));
  return v;
}

// Per-job arrays (structure of arrays, device memory).
struct JobArrays {
  int32_t* m;           // order
  int32_t* nnz;         // nonzeros
  int64_t* off;         // word offset of the CSR block in the arena
  int32_t* mat;         // source matrix
  int32_t* depth_left;  // levels of Eq. 2 still to apply in the pre-expansion
  uint64_t* coef;       // 4 words per job: scalar factor modulo 2^256
};

// Evaluation outputs, indexed by job.
struct JobOut {
  unsigned long long* acc;        // 4 words per job: Ryser sums or coef*per (mod 2^256)
  unsigned long long* t_start;    // globaltimer of the first worker
  unsigned long long* t_end;      // globaltimer of the last worker
  int32_t* sm;                    // SM of the first worker
  int32_t* status;                // 0 ok, PERM_EOVERFLOW, PERM_ETIMEOUT
  unsigned long long* leaves;     // Ryser leaves
  unsigned long long* nodes;      // Eq. 2 nodes visited
};
