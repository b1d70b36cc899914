// Internal declarations shared by the library's translation units.
#pragma once
#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>
#include <exception>

#include "../../include/perm.h"
#include "jobs.cuh"
#include "modp.cuh"

// Evaluation keys of a queue: leaf jobs (order <= leaf_max) get their kernel
// variant (nmax index | W bit | path << 3, < 64), the others the
// depth-first group EVAL_KEY_DFS + g, g = 2 * (order <= 32) + (ring width
// 4): tile 64 before tile 32; hist[key] counts them.
#define EVAL_KEY_DFS 64
#define EVAL_DFS_GROUPS 4
#define EVAL_KEYS (EVAL_KEY_DFS + EVAL_DFS_GROUPS)

// ---- scans and sorts (CUB, header source) --------------------------------
cudaError_t scan_exclusive_u64(const uint64_t* in, uint64_t* out, int64_t n, void* tmp, size_t tmp_bytes,
                               cudaStream_t s);
size_t scan_tmp_bytes_u64(int64_t n);
cudaError_t scan_exclusive_i64(const int64_t* in, int64_t* out, int64_t n, void* tmp, size_t tmp_bytes,
                               cudaStream_t s);
size_t scan_tmp_bytes_i64(int64_t n);
cudaError_t scan_exclusive_i32(const int32_t* in, int32_t* out, int64_t n, void* tmp, size_t tmp_bytes,
                               cudaStream_t s);
size_t scan_tmp_bytes_i32(int64_t n);
// Stable sort of (key, value) pairs by non-increasing key.
cudaError_t sort_desc_f32(const float* keys_in, float* keys_out, const uint32_t* vals_in, uint32_t* vals_out,
                          int64_t n, void* tmp, size_t tmp_bytes, cudaStream_t s);
size_t sort_tmp_bytes_f32(int64_t n);
// Stable sort of (key, value) pairs by ascending key bits [0, end_bit) of 64-bit keys.
cudaError_t sort_asc_u64(const uint64_t* keys_in, uint64_t* keys_out, const uint32_t* vals_in, uint32_t* vals_out,
                         int64_t n, int end_bit, void* tmp, size_t tmp_bytes, cudaStream_t s);
size_t sort_tmp_bytes_u64(int64_t n);
// Stable sort of (key, value) pairs by ascending key bits [0, end_bit).
cudaError_t sort_asc_u32(const uint32_t* keys_in, uint32_t* keys_out, const uint32_t* vals_in, uint32_t* vals_out,
                         int64_t n, int end_bit, void* tmp, size_t tmp_bytes, cudaStream_t s);
size_t sort_tmp_bytes_u32(int64_t n, int end_bit);
// out[i] = i for i < n (the natural order of a job list)
cudaError_t launch_iota_u32(uint32_t* out, int64_t n, cudaStream_t s);
// *out = min over jobs j < n with status s not in {0, DFS_RETRY} of j * 256 + s
// (unchanged when there is none; set it to ~0 first).
cudaError_t launch_status_summary(const int32_t* status, int64_t n, unsigned long long* out, cudaStream_t s);
// Stable compaction of the depth-first queue's jobs whose status is
// DFS_RETRY into rq; at[g] = retried jobs before queue position bounds.b[g]
// (g <= EVAL_DFS_GROUPS), so the retry queue keeps the queue's groups.
// flags and pos hold n + 1 entries each.
struct RetryBounds {
  int64_t b[EVAL_DFS_GROUPS + 1];
};
cudaError_t launch_retry_collect(const uint32_t* dq, int64_t n, RetryBounds bounds, const int32_t* status,
                                 int32_t* flags, int32_t* pos, void* scan_tmp, size_t scan_tmp_bytes, uint32_t* rq,
                                 unsigned long long* at, cudaStream_t s);

// ---- K2 leaf batch -----------------------------------------------------------
// Evaluation key (see EVAL_KEY_DFS) of every queue position, the queue's
// jobs in vals, and the key histogram (zero it first, EVAL_KEYS entries).
// modular: the residue path (every leaf job takes the modular variant).
cudaError_t launch_eval_keys(const uint32_t* queue, int64_t n, const JobArrays& jobs, const uint64_t* arena,
                             const int32_t* mat_w, int leaf_max, bool modular, uint32_t* keys, uint32_t* vals,
                             unsigned long long* hist, cudaStream_t stream);
// Ryser tasks of every queued leaf job, their exclusive scan (nq + 1
// entries) and the task owner map: owner[t] = queue position of task t's job
// (prefix[nq] entries; leaf_tasks_host(m, chunk_log2) summed over the jobs).
cudaError_t launch_leaf_tasks(const uint32_t* queue, int64_t nq, const JobArrays& jobs, int chunk_log2,
                              uint64_t* counts_scratch, uint64_t* prefix, uint32_t* owner, void* scan_tmp,
                              size_t scan_tmp_bytes, cudaStream_t stream);
uint64_t leaf_tasks_host(int m, int chunk_log2);
// One variant group of leaf jobs in queue order: the group starts at queue
// position qbase of the grouped queue; queue and prefix are its slices (nq
// and nq + 1 entries), owner the whole map.  mod: the modulus of the
// residue path (used by the modular variant only).
cudaError_t launch_leaf_batch(const uint32_t* queue, int64_t nq, int cls, const uint64_t* prefix,
                              const uint32_t* owner, int64_t qbase, const JobArrays& jobs, const uint64_t* arena,
                              int chunk_log2, unsigned long long* task_counter, const JobOut& out, const ModP& mod,
                              int num_sms, cudaStream_t stream);
// Sigma -> coef * per for every leaf job, summed into the matrix accumulators
// (modp != 0: residues modulo modp).
cudaError_t launch_leaf_finalize(const uint32_t* queue, int64_t nq, const JobArrays& jobs, const JobOut& out,
                                 unsigned long long* mat_acc, uint32_t modp, cudaStream_t stream);

// ---- K1 expansion (one level) ---------------------------------------------------
// Parents [0, np) in arena_in.  Children go to slots Kp .. Kp + K - 1 of the
// child arrays (K = kslots: 2, or 3 with Eq. 2's third child for s >= 5);
// child_off_base[p] is the first word of parent p's K child blocks (each of
// the parent's size) in arena_out.  valid[Kp + c] is 1 for an emitted child.
struct ExpandLevelArgs {
  JobArrays parent;
  const uint64_t* arena_in;
  int64_t np;
  JobArrays child;  // K*np slots
  uint64_t* arena_out;
  const int64_t* child_off_base;
  int32_t* valid;   // K*np
  int32_t kslots;
  int32_t leaf_size;
  int32_t split_floor;  // parents of a lower order (with depth left, above the leaf order) wait
  uint32_t mod;     // 0, or the residue path's modulus: entries and coefficients reduced modulo it
  int32_t* err;     // device flag: first error status
};
cudaError_t launch_expand_level(const ExpandLevelArgs& a, int max_order, cudaStream_t s);

// Consecutive levels in one cooperative launch.  The current jobs are
// buf[state.cb] with their blocks in arena[state.cb] (state.used_words
// words).  Runs a level while: level < max_levels, 0 < ncur, 2 * ncur <=
// cap_jobs, K * used_words <= cap_words (K child slots per parent; the
// condition on ncur is K * ncur <= cap_jobs), and (when adaptive) max_open >
// big_order, or max_open > soft_order and ncur < soft_cap_jobs, or (ncur <
// target_jobs and max_open > 0), where max_open is the
// largest order of a job still to split; adaptive levels split only parents
// of order >= max_open - band.  The state is updated in place; the children
// of a level are compacted in natural order into the other buffer.  bar,
// lvl_words, lvl_maxo and lvl_maxopen (max_levels entries) must be zero;
// partial holds PERM_FRONT_MAX_BLOCKS entries.
struct ExpandFrontState {
  int64_t ncur;
  int64_t used_words;
  int32_t level;
  int32_t max_order;
  int32_t max_open;
  int32_t cb;
};
#define PERM_FRONT_MAX_BLOCKS 1024
struct ExpandFrontArgs {
  JobArrays buf[2];
  uint64_t* arena[2];
  int64_t cap_jobs;
  int64_t cap_words;
  JobArrays slots;  // cap_jobs (children of at most cap_jobs / K parents)
  int32_t* valid;   // cap_jobs
  int32_t kslots;
  int32_t leaf_size;
  int32_t max_levels;
  int32_t adaptive;
  int32_t big_order;
  int32_t band;
  int32_t soft_order;
  int64_t soft_cap_jobs;
  int64_t target_jobs;
  ExpandFrontState* state;
  long long* partial;
  unsigned long long* bar;
  unsigned long long* lvl_words;
  int32_t* lvl_maxo;
  int32_t* lvl_maxopen;
  uint32_t mod;     // as in ExpandLevelArgs
  int32_t* err;
};
// *grid = blocks launched, 0 when the device has no cooperative launch (the
// caller then runs every level with launch_expand_level).
cudaError_t launch_expand_front(const ExpandFrontArgs& a, int max_order, int* grid, cudaStream_t s);
// words[p] = kslots * blk_words(parent p) (capacity for its children)
cudaError_t launch_child_capacity(const JobArrays& parent, int64_t np, int kslots, int64_t* words, cudaStream_t s);
// Compact valid slots into dst (natural order kept).  Accumulates into
// stat[0] the largest kept order, stat[1] the kept blocks' words, stat[2]
// the kept job count and stat[3] the largest order of a kept job with depth
// left and order above cut (zero them first).
cudaError_t launch_compact_jobs(const JobArrays& src, const int32_t* valid, const int32_t* pos, int64_t nslots,
                                JobArrays dst, int cut, long long* stat, cudaStream_t s);

// ---- K1 traversal driver (walk.cu) ----------------------------------------------
// The walk's internal status when a buffer (arena, outputs, queue) is full:
// the host then uses the level-by-level driver.
#define WALK_FULL 200
// A queue of subtree roots handed between warps (ticket per waiting warp).
struct WalkQueue {
  int32_t* m;
  int32_t* nnz;
  int32_t* mat;
  int32_t* dl;
  int32_t* depth;
  int64_t* off;
  uint64_t* coef;   // 4 words per node
  uint64_t* key;    // 2 words per node (path key, low word first)
  int32_t* ready;   // 1 once slot t is written (zero it first)
  int64_t cap;
  unsigned long long* head;  // tickets taken
  unsigned long long* tail;  // slots reserved
};
struct WalkArgs {
  WalkQueue q;      // work: the roots (or the nodes handed over by the wider phase) and donated siblings
  WalkQueue hand;   // nodes of order <= handover_order, for the narrower phase
  int32_t handover_order;  // 0: walk every node here
  unsigned long long* outstanding;  // nodes in q not yet taken plus busy warps (two's complement count)
  // blocks: the roots' blocks first, then bump-allocated in chunks
  uint64_t* arena;
  int64_t cap_words;
  int64_t arena_chunk;
  unsigned long long* arena_used;
  // jobs, in slots reserved a few at a time (unused slots keep key ~0)
  JobArrays out;
  uint64_t* out_key;  // 2 words per slot
  int64_t cap_out;
  unsigned long long* out_used;
  unsigned long long* emitted;
  // per depth: nodes, jobs, largest order still to split
  unsigned long long* hist_nodes;
  unsigned long long* hist_term;
  int32_t* hist_maxopen;
  int32_t hist_len;
  int32_t leaf_size;
  int32_t kslots;
  int32_t bits_per_level;
  int32_t key_levels;
  int32_t stage_words;  // words of a warp's staging copy of a block (larger blocks are read from L2)
  // per-warp undo stacks (tile.cuh frames) for warps_cap warps
  int64_t* undo;
  int64_t undo_words_per_warp;
  int32_t max_rel_depth;  // frames per warp
  int64_t warps_cap;
  int64_t timeout_ns;
  uint32_t mod;     // as in ExpandLevelArgs
  int32_t* err;
};
// tile width for roots of this order (0: above the tiles; use the level-by-level driver)
int walk_tile_for(int max_order);
size_t walk_smem_bytes(int tile, int stage_words, int hist_len);
int64_t walk_frame_words(int tile);
// warps of the launch (every block resident)
cudaError_t walk_resident_warps(int tile, int stage_words, int hist_len, int sms, int64_t* warps);
// *grid = blocks launched (0: the kernel does not fit; use the level-by-level driver)
cudaError_t launch_expand_walk(const WalkArgs& a, int tile, int sms, int* grid, cudaStream_t s);
// perm = slots [0, n) in ascending path-key order; keys use bits [0, key_bits]
// (two passes when key_bits >= 64)
cudaError_t launch_walk_order(const uint64_t* key2, int64_t n, int key_bits, uint64_t* kbuf, uint64_t* kbuf2,
                              uint32_t* ibuf, uint32_t* perm, void* tmp, size_t tmp_bytes, cudaStream_t s);
cudaError_t launch_walk_gather(const uint32_t* perm, int64_t n, const JobArrays& src, const JobArrays& dst,
                               cudaStream_t s);

// ---- K3 depth-first evaluator --------------------------------------------------
struct DfsArgs {
  const uint32_t* queue;
  int64_t nq;
  JobArrays jobs;
  const uint64_t* arena;
  const int32_t* mat_w;
  int32_t leaf_size;
  unsigned long long* job_counter;
  JobOut out;
  unsigned long long* mat_acc;
  int64_t* undo;          // per-warp undo stacks
  int64_t undo_words_per_warp;
  int64_t timeout_ns;
  int32_t three;          // s >= 5 nodes split by Eq. 2's three children (else leaves)
  int32_t max_depth;      // undo frames per warp
  unsigned long long* retry_flag;  // nullable: set to 1 when a job reports DFS_RETRY
  ModP mod;               // p = 0: the ring path; else every value modulo p (W is ignored)
};
// Internal job status of the narrow depth-first variant (int32 tile, leaves
// up to 16 rows): the job needs the wide variant (int64 tile, leaves up to 32).
#define DFS_RETRY 100
// All queued jobs must belong to matrices of ring width W (2 or 4 words).
cudaError_t launch_dfs(const DfsArgs& a, int tile, bool wide, int W, int num_sms, int warps_per_sm, cudaStream_t s);
int dfs_warps_per_block(int tile, bool wide);
// undo words per warp for a stack of `frames` levels
int64_t dfs_undo_words(int tile, int frames);

// ---- single-launch evaluation (persist.cu) ------------------------------------
// The whole queue in one persistent launch: leaf jobs by their variant's
// Ryser walk (tasks shared through a board), other jobs of order <= 32 by
// the depth-first walk on a 32-wide int64 tile; jobs of order > 32 that are
// not leaves are skipped (the caller runs them first).  keys: the
// evaluation key of every queue position (launch_eval_keys).  qctr (zero),
// board (-1), task_next and task_done (nq entries, zero) are reset by the
// caller before every launch.  dfs: the depth-first arguments (queue, nq
// and job_counter unused; undo sized for persist_warps warps).
struct PersistArgs {
  const uint32_t* queue;
  const uint32_t* keys;
  int64_t nq;
  int32_t chunk_log2;
  unsigned long long* qctr;
  long long* board;
  uint32_t* task_next;
  uint32_t* task_done;
  DfsArgs dfs;
};
// W: 2 or 4 (ring words; 4 also serves matrices of width 2), 0 = the residue
// path.  narrow: int32 tiles and depth-first leaves up to 16 rows (a job that
// needs more reports DFS_RETRY and sets dfs.retry_flag), else int64 and 32.
cudaError_t launch_persist(const PersistArgs& a, int W, bool narrow, int sms, cudaStream_t s);
cudaError_t persist_warps(int W, bool narrow, int sms, int64_t* warps);
cudaError_t launch_persist_narrow(const PersistArgs& a, int W, int sms, cudaStream_t s);
cudaError_t persist_warps_narrow(int W, int sms, int64_t* warps);

// ---- K4 KKLLL estimator -------------------------------------------------------
// scratch: kklll_scratch_bytes(njobs, max_order, trials) bytes of device memory
cudaError_t launch_kklll(const JobArrays& jobs, int64_t njobs, const uint64_t* arena, int trials, uint64_t seed,
                         float* log_ap, int max_order, void* scratch, cudaStream_t s);
size_t kklll_scratch_bytes(int64_t njobs, int max_order, int trials);

// ---- K5 features and MLP -------------------------------------------------------
cudaError_t launch_features(const JobArrays& jobs, int64_t njobs, const uint64_t* arena, const float* log_ap,
                            float* feats, cudaStream_t s);
cudaError_t mlp_forward_backward(const float* params, const float* feats, const float* target, int32_t count,
                                 float* hidden_scratch, float* grad, float* loss, cudaStream_t s);
cudaError_t mlp_predict(const float* params, const float* feats, int32_t count, float* pred, cudaStream_t s);
cudaError_t mlp_adam_step(float* params, const float* grad, float* m1, float* m2, int32_t step, float lr,
                          cudaStream_t s);

// ---- measurement ----------------------------------------------------------------
cudaError_t launch_ubench_imad(int blocks, int iters, uint32_t* sink, cudaStream_t s);

// ---- errors ----------------------------------------------------------------------
void set_last_error(const char* what, cudaError_t e);
void set_last_error_text(const char* what) noexcept;

// Runs an entry point's body so that a host exception (a failed host
// allocation, or a host thread that could not start) becomes PERM_ENOMEM
// with perm_last_error() set, instead of crossing the C boundary.
template <class F>
static perm_status guarded(F&& body) noexcept {
  try {
    return body();
  } catch (const std::exception& e) {
    set_last_error_text(e.what());
  } catch (...) {
    set_last_error_text("host exception");
  }
  return PERM_ENOMEM;
}
