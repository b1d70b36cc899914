/*
 * perm.h -- C ABI of the GB300 sparse-permanent library (libperm.so).
 *
 * Computes exact permanents (Eq. 1 of Wang, Liang, Bai and Huo, "A load
 * balancing strategy for parallel computation of sparse permanents",
 * arXiv 1112.6072) of sparse integer matrices by the paper's parallel hybrid
 * method:
 *   1. divide: the expansion of Eq. 2, applied level by level (Algorithm PH,
 *      Step 2, Section 2.2), turns each matrix into sub-matrix jobs;
 *   2. order: jobs sorted by non-increasing KKLLL approximate permanent
 *      (Section 3.3, the improved Step 3), or by a learned cost model;
 *   3. evaluate: each job by Algorithm H_per (Section 2.1) -- Eq. 2 depth
 *      first down to a leaf order L, then Ryser's formula with the
 *      Nijenhuis-Wilf Gray-code variant (Section 1) in exact integers;
 *   4. sum: Step 4 of Algorithm PH.
 * Every step runs in CUDA kernels for sm_103a on one GPU.
 *
 * Conventions for every entry point:
 *   - Return value is a perm_status; no entry point aborts or exits.
 *   - Host pointers are caller-owned and only read or written during the
 *     call.  Device memory is owned by the library (plan and job handles)
 *     unless an entry point says otherwise.
 *   - Work is issued on perm_opts.stream (a cudaStream_t; NULL is the legacy
 *     default stream).  Entry points that return host data synchronise that
 *     stream before returning.
 *   - Exactness: results are computed modulo 2^K in wrap-around integer
 *     arithmetic, where K is chosen per matrix from the bound
 *     |per(A)| <= min(prod_i sum_j |a_ij|, prod_j sum_i |a_ij|) so that the
 *     signed value is recovered exactly.  If no supported K proves the
 *     bound, the call fails with PERM_EOVERFLOW instead of returning a
 *     wrong value.
 */
#ifndef PERM_H_
#define PERM_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  PERM_OK = 0,
  PERM_EINVAL = 1,     /* bad argument: n < 0 or n > PERM_MAX_N, null pointer, ld < n ... */
  PERM_EOVERFLOW = 2,  /* a value or bound beyond what the exact paths can prove */
  PERM_ETIMEOUT = 3,   /* a bounded device wait gave up (kernel watchdog) */
  PERM_ECUDA = 4,      /* a CUDA runtime call failed; see perm_last_error() */
  PERM_ESHORTBUF = 5,  /* output buffer too short; the required size is reported */
  PERM_ENOMEM = 6,     /* device or host allocation failed */
  PERM_ESTATE = 7      /* call out of sequence (e.g. evaluate before expand) */
} perm_status;

#define PERM_MAX_N 128       /* largest matrix order accepted */
#define PERM_MAX_JOB_N 64    /* largest job order the depth-first evaluator holds */
#define PERM_MAX_LEAF 32     /* largest order the leaf Ryser kernel evaluates */

typedef enum {
  PERM_ORDER_NATURAL = 0,  /* Algorithm PH, Step 3: natural order of expansion (LS) */
  PERM_ORDER_LPT = 1,      /* Section 3.3: non-increasing KKLLL approximate permanent */
  PERM_ORDER_LEARNED = 2   /* non-increasing predicted job time (MLP); LPT if no model */
} perm_order_kind;

/* A dense integer matrix in host memory, row-major: a[i * ld + j]. */
typedef struct {
  int32_t n;          /* order, 0 <= n <= PERM_MAX_N; n = 0 has per = 1 */
  const int64_t* a;   /* entries; |a_ij| < 2^31 (any int64 on the residue path, opts.modulus) */
  int64_t ld;         /* leading dimension, ld >= n */
} perm_matrix;

/* Optional device allocator: lets a host framework (e.g. PyTorch's caching
 * allocator) own the memory.  Both NULL: stream-ordered allocations on the
 * plan's stream from a memory pool the library creates per device, which
 * keeps up to 4 GiB of freed memory mapped for later plans (released at
 * process exit). */
typedef void* (*perm_alloc_fn)(size_t bytes, void* stream, void* ctx);
typedef void (*perm_free_fn)(void* ptr, void* stream, void* ctx);

typedef struct {
  int32_t split_depth;     /* d of Algorithm PH; -1 = choose: expand while a job has order
                              > PERM_MAX_JOB_N, or order > 32 with fewer than 2^25 jobs, or
                              while there are fewer than 2^17 jobs per matrix (2^21 for batches
                              of 16 or more) and a job above order L; each level then splits
                              only the jobs within 2 orders of the largest one (largest first) */
  int32_t leaf_size;       /* L: a node of order <= L is evaluated by Ryser; 0 = choose */
  int32_t order;           /* perm_order_kind used by perm_eval_batch when no order is given */
  int32_t kklll_trials;    /* KKLLL trials per job; 0 = m^2 for a job of order m (Table T5 note) */
  uint64_t seed;           /* seed of the KKLLL counter-based stream */
  int32_t workers_per_sm;  /* resident evaluator warps per SM; 0 = choose */
  int32_t chunk_log2;      /* leaf Ryser: at most 2^chunk_log2 Gray steps per lane; 0 = choose */
  void* stream;            /* cudaStream_t for all work of the plan */
  perm_alloc_fn alloc;     /* optional allocator (see above) */
  perm_free_fn free;
  void* alloc_ctx;
  int64_t timeout_ns;      /* device watchdog for bounded waits; 0 = 10 s */
  int32_t model_uses_estimate; /* 1: job features include the KKLLL estimate (runs the
                                  estimator); 0: that feature is 0 and the learned order
                                  needs no estimate */
  int32_t fused_levels;    /* expansion: 1 = run consecutive levels in one cooperative launch
                              while the frontier fits its buffers (grown to at most 2^20 jobs and
                              2^26 arena words), then one launch per level; 0 = one launch per
                              level throughout.  The job list is the same either way */
  int32_t dense_split;     /* 0 = Algorithm H_per: a node whose sparsest line has s >= 5 nonzeros
                              is a leaf (Ryser).  1 = such a node is split by Eq. 2 with all three
                              children: merge(j1, j2), merge(j3, j4), and the node with the pivot
                              line's entries at j1..j4 cleared (same order) */
  int32_t expand_walk;     /* expansion driver: 1 = a traversal in which warps walk the tree depth
                              first and hand nodes to idle warps, writing only the jobs, which a
                              sort of their child-index paths puts in natural order (used when
                              every root block fits its shared-memory buffers, with a fixed depth,
                              or with the automatic depth for roots of one order without the
                              three-child split; otherwise, or when its buffers fill, the
                              level-by-level driver runs); 0 = level by level.  The job list is the
                              same either way */
  uint32_t modulus;        /* 0 = exact: results in a 2^K ring proven wide enough (else
                              PERM_EOVERFLOW).  An odd prime p < 2^31 = the residue path: every
                              entry (any int64; reduced first), merged entry, coefficient and
                              Ryser sum is taken modulo p (Eq. 2 and Ryser's formula are
                              identities over any commutative ring, so per(A) mod p is exact
                              however large per(A) is); results are residues in [0, p)
                              (perm_result_words word 0, perm_result a non-negative value,
                              perm_result_bits 0).  Residues for several primes and perm_crt give
                              per(A) itself.  PERM_EINVAL if p is not an odd prime below 2^31 */
  int32_t single_launch;   /* evaluation: 0 = one persistent launch per kernel variant (leaf
                              variants grouped, depth-first jobs by tile width; queue order kept
                              inside each group).  1 = the whole queue in one persistent launch:
                              warps take queue positions in queue order through one counter and
                              run each job's own evaluator as a device function (leaf jobs'
                              Gray-code tasks shared with idle warps; depth-first jobs of order
                              <= 32 on a 32-wide tile), so the queue order holds across all jobs;
                              depth-first jobs of order > 32 run in a launch before it, and a job
                              the int32 tile cannot hold (leaf order <= 16) runs again on the int64
                              kernel after it.  The results are the same either way */
} perm_opts;

/* Fill opts with the defaults above. */
void perm_opts_default(perm_opts* opts);

typedef struct perm_plan perm_plan_t; /* opaque */
typedef struct perm_jobs perm_jobs_t; /* opaque, owned by its plan */

/* Per-job record returned by perm_eval_batch (host memory, caller-owned). */
typedef struct {
  int32_t matrix;      /* index of the input matrix the job belongs to */
  int32_t order;       /* m, the job's order */
  int32_t nnz;         /* nonzeros of the job */
  int32_t status;      /* perm_status of the job */
  uint64_t value[4];   /* coef * per(job) modulo 2^256, two's complement, little-endian
                          words; exact in its low K bits (see perm_result_bits) */
  int64_t t_start_ns;  /* device globaltimer when the first worker took the job */
  int64_t t_end_ns;    /* device globaltimer when the last worker finished it */
  int32_t sm;          /* SM of the worker that took the job first */
  int32_t queue_pos;   /* position of the job in the evaluated queue */
  int64_t leaves;      /* Ryser leaves evaluated for the job */
  int64_t nodes;       /* Eq. 2 nodes visited for the job (leaves included) */
} perm_job_result;

/* a1 -- Validate and canonicalise count matrices (Eq. 1's A; the pattern B
 * of Section 3 is implicit), choose the exact width K per matrix and upload
 * them.  *out is owned by the library; release it with perm_plan_destroy.
 * Errors: PERM_EINVAL (count < 1, null pointers, n out of range, ld < n,
 * |a_ij| >= 2^31 on the exact path, a modulus that is not an odd prime below
 * 2^31), PERM_EOVERFLOW (bound too large for the exact path), PERM_ECUDA,
 * PERM_ENOMEM. */
perm_status perm_plan_create(const perm_matrix* mats, int32_t count, const perm_opts* opts,
                             perm_plan_t** out);
void perm_plan_destroy(perm_plan_t* plan);

/* a2, a3 -- Algorithm PH, Step 2: apply Eq. 2 split_depth times to every
 * matrix, level by level, on the device.  Pivot: the smallest line count s
 * (Algorithm H_per, Step 1), lowest row first, else lowest column; a node of
 * order <= max(L, 2) or with s >= 5 is carried unchanged; children holding a
 * zero line are dropped.  Jobs are kept in natural order (matrix order, then
 * BFS order, children in Eq. 2 order) in a compact CSR arena.
 * *jobs stays owned by the plan (one job set per plan; a second call
 * replaces it).  *njobs receives the job count. */
perm_status perm_expand(perm_plan_t* plan, perm_jobs_t** jobs, int64_t* njobs);

/* Which driver built the plan's job set: 0 = level by level (one launch
 * sequence per level), 1 = consecutive levels per cooperative launch,
 * 2 = the traversal (opts.expand_walk).  PERM_ESTATE before perm_expand. */
perm_status perm_expand_driver(perm_plan_t* plan, int32_t* driver);

/* Device time of the last perm_expand (ms): events on the plan's stream
 * around its uploads, kernels, and (traversal) key sort and gather.
 * PERM_ESTATE before perm_expand. */
perm_status perm_last_expand_ms(perm_plan_t* plan, float* ms);

/* a4 -- Algorithm KKLLL (Section 2.3) on each job's 0/1 pattern (Section 3),
 * jobs of any order up to PERM_MAX_N:
 * log of the mean over trials of |det W|^2, W_ij a cube root of unity drawn
 * from SplitMix64(seed ^ job*0xD1B54A32D192ED03 ^ trial*0xABC98388FB8FAC03 ^
 * (i*m+j)*0x8CB92BA72F3D8DD7).  FP32 on the device; -inf when every trial is
 * singular.  log_ap (host, nullable) receives njobs floats. */
perm_status perm_estimate(perm_jobs_t* jobs, float* log_ap);

/* a5, a6 -- Set the evaluation queue: kind = PERM_ORDER_NATURAL keeps the
 * natural order; PERM_ORDER_LPT sorts by non-increasing KKLLL estimate
 * (runs perm_estimate if needed); PERM_ORDER_LEARNED sorts by non-increasing
 * time predicted by the model attached with perm_mlp_attach (falls back to
 * LPT without one).  Equal keys keep natural order.  order_out (host,
 * nullable) receives the njobs job indices in queue order. */
perm_status perm_order(perm_jobs_t* jobs, int32_t kind, uint32_t* order_out);

/* a7, a8 -- Evaluate every job exactly and sum per matrix (Algorithm PH,
 * Steps 3-4): one persistent launch for jobs above the leaf order (Eq. 2
 * depth first, Ryser at the leaves) and one for leaf-order jobs (Ryser, the
 * Gray range split over warps).  Workers pull jobs through an atomic queue
 * in the order given (host array of njobs job indices, a permutation), or
 * in the order set by perm_order when order is NULL.  results (host,
 * nullable) receives njobs records indexed by job.  Errors: PERM_EINVAL
 * (order not a permutation), PERM_EOVERFLOW (an entry left int64 or a leaf
 * row sum left int32), PERM_ETIMEOUT, PERM_ECUDA. */
perm_status perm_eval_batch(perm_jobs_t* jobs, const uint32_t* order, perm_job_result* results);

/* a7, a8 over part of the queue (Algorithm PH, Step 3, with the jobs dealt
 * to several workers -- e.g. one GPU each -- and Step 4's sum taken over
 * their partial sums).  queue (host) holds count distinct job indices
 * (0 <= count <= njobs; queue may be NULL when count is 0), evaluated in
 * that order as by perm_eval_batch; the other jobs are not evaluated: their
 * records are zero with queue_pos = -1.  Afterwards perm_result,
 * perm_result_words and perm_result_bits give each matrix's sum over the
 * evaluated jobs, modulo 2^K (perm_result_bits): the sums of disjoint
 * sub-queues that together hold every job add up, modulo 2^K, to per(A).  A
 * matrix without jobs (order 0, or a zero line) contributes 0 to every
 * sub-queue sum.  Errors as for perm_eval_batch; PERM_EINVAL for a repeated
 * or out-of-range index. */
perm_status perm_eval_subset(perm_jobs_t* jobs, const uint32_t* queue, int64_t count,
                             perm_job_result* results);

/* a7, a8 again, as a CUDA graph: repeat the last perm_eval_batch of this job
 * set (same queue, same buffers).  The first call captures that
 * evaluation's memsets and launches into a graph (on a stream the library
 * creates), later calls launch the instantiated graph on the plan's stream.
 * results as for perm_eval_batch.  PERM_ESTATE if the job set has not been
 * evaluated yet. */
perm_status perm_eval_replay(perm_jobs_t* jobs, perm_job_result* results);

/* Wall time of the last perm_eval_batch on the device (ms), from events on
 * the plan's stream. */
perm_status perm_last_eval_ms(perm_plan_t* plan, float* ms);

/* Number of kernel launches the last perm_eval_batch issued between its two
 * timing events (scans included). */
perm_status perm_last_eval_launches(perm_plan_t* plan, int32_t* launches);

/* a8 -- per(A) of matrix `index` after perm_eval_batch, as a magnitude in
 * little-endian uint32 limbs and a sign (-1, 0, +1).  cap too small ->
 * PERM_ESHORTBUF with *nlimbs set to the required length. */
perm_status perm_result(perm_plan_t* plan, int32_t index, uint32_t* limbs, int32_t cap,
                        int32_t* nlimbs, int32_t* sign);

/* The number of exact low bits K of matrix `index` (results are exact
 * modulo 2^K and |per(A)| < 2^(K-1) is proven); 0 on the residue path. */
perm_status perm_result_bits(perm_plan_t* plan, int32_t index, int32_t* bits);

/* All results at once: out[i*4 .. i*4+3] = per(A_i) modulo 2^256 (two's
 * complement words, exact in the low perm_result_bits bits); on the residue
 * path per(A_i) mod p in word 0 and zero words above. */
perm_status perm_result_words(perm_plan_t* plan, uint64_t* out, int32_t count);

/* Residue path, reconstruction -- integers from residues by the Chinese
 * remainder theorem (Garner's mixed-radix form), for results taken modulo
 * several primes (opts.modulus).  residues (host) holds count rows of k
 * values, residues[v * k + i] = x_v mod primes[i] (< primes[i]); primes
 * (host): k distinct odd primes below 2^31, 1 <= k <= 64.  Output (host):
 * limbs[v * (k + 1) ..] = |x_v| in k + 1 little-endian uint32 limbs,
 * signs[v] in {-1, 0, +1}.  Every x_v with |x_v| < M / 2, M the product of
 * the primes, comes back exactly (the balanced residue).  Runs on the
 * stream (nullable) and returns when the results are in host memory.
 * Errors: PERM_EINVAL (k or count out of range, a prime repeated or not an
 * odd prime below 2^31, a residue not below its prime), PERM_ECUDA,
 * PERM_ENOMEM. */
perm_status perm_crt(const uint32_t* residues, const uint32_t* primes, int32_t k, int32_t count,
                     uint32_t* limbs, int32_t* signs, void* stream);

/* Export the job list for inspection (two-call protocol: with sizes == NULL
 * only *total_entries is set).  sizes[w] = order, mats receives the dense
 * row-major jobs back to back (int64), coef[w*4..] the coefficient modulo
 * 2^256, matrix[w] the source matrix (nullable). */
perm_status perm_jobs_export(perm_jobs_t* jobs, int64_t* total_entries, int32_t* sizes,
                             int64_t* mats, uint64_t* coef, int32_t* matrix);

/* Export chosen jobs only (a sample of a large job set): idx (host) holds
 * count job indices (repeats allowed).  sizes[k] = order of job idx[k];
 * *entries = the sum of the orders squared; mats (nullable) receives the
 * dense row-major jobs back to back (PERM_ESHORTBUF, with sizes and *entries
 * set, when mats_cap is smaller); coef[k*4..] (nullable) the coefficient
 * modulo 2^256; matrix[k] (nullable) the source matrix.  PERM_EINVAL for an
 * index outside [0, njobs). */
perm_status perm_jobs_select(perm_jobs_t* jobs, const int64_t* idx, int64_t count, int32_t* sizes,
                             int64_t* mats, int64_t mats_cap, uint64_t* coef, int32_t* matrix,
                             int64_t* entries);

/* Convenience: per(A) of one matrix (perm_plan_create, perm_expand,
 * perm_order(opts.order), perm_eval_batch, perm_result, perm_plan_destroy). */
perm_status perm_exact(const perm_matrix* a, const perm_opts* opts, uint32_t* limbs, int32_t cap,
                       int32_t* nlimbs, int32_t* sign);

/* ---- learned cost model (a5, a9): 2 x 64 hidden ReLU MLP, FP32 ---------------
 * Features of a job (PERM_MLP_FEATURES floats): order m/64, nnz/m^2,
 * fraction of rows with 1, 2, 3, 4, 5-6, 7-9, 10-14, >=15 nonzeros, KKLLL
 * log AP / 64, Ryser work log2(m * 2^(m-1)) / 64.  Target: log(job time).
 * Parameters are one float array of PERM_MLP_PARAMS values:
 * W1[64][F], b1[64], W2[64][64], b2[64], w3[64], b3. */
#define PERM_MLP_FEATURES 12
#define PERM_MLP_HIDDEN 64
#define PERM_MLP_PARAMS (64 * 12 + 64 + 64 * 64 + 64 + 64 + 1)

/* Features of every job of the set, computed on the device (a5).  feats
 * (host) receives njobs * PERM_MLP_FEATURES floats.  With
 * opts.model_uses_estimate set, runs perm_estimate if the set has no
 * estimate yet; otherwise the estimate feature is 0. */
perm_status perm_job_features(perm_jobs_t* jobs, float* feats);

/* One forward and backward pass on a batch (device kernels): feats (host,
 * count x F), target (host, count), params (host).  loss receives the mean
 * squared error, grad (host, PERM_MLP_PARAMS) its gradient. */
perm_status perm_mlp_grad(const float* params, const float* feats, const float* target,
                          int32_t count, void* stream, float* loss, float* grad);

/* Train with Adam on the device for `steps` full-batch steps from params
 * (host, in/out), learning rate lr.  final_loss (nullable) receives the
 * last loss. */
perm_status perm_mlp_train(float* params, const float* feats, const float* target, int32_t count,
                           int32_t steps, float lr, void* stream, float* final_loss);

/* Inference (device kernel): pred (host) receives count predictions. */
perm_status perm_mlp_predict(const float* params, const float* feats, int32_t count, void* stream,
                             float* pred);

/* Attach model parameters (host, copied) to a plan for PERM_ORDER_LEARNED. */
perm_status perm_mlp_attach(perm_plan_t* plan, const float* params);

/* ---- allocation-free leaf batch -------------------------------------------------
 * The paper has no counterpart to this entry point.  It is for callers that
 * cannot allocate device memory while they run: a host framework whose own
 * allocator must own every device allocation (so the library may not call
 * cudaMalloc behind its back), a latency-bound loop that may not allocate
 * after start-up (cudaMalloc and cudaFree can synchronise the device and
 * stall it), or a process working inside a fixed device-memory budget.  It
 * evaluates count dense matrices of one order n by the leaf Ryser /
 * Nijenhuis-Wilf kernel and allocates nothing: no cudaMalloc, no cudaFree,
 * no allocating library call.
 *   a      device, count matrices of order n back to back, row-major int64
 *          (n*n entries each), |a_ij| < 2^30 and, for every row i,
 *          sum_j |a_ij| < 2^31
 *   n      1 <= n <= PERM_MAX_LEAF, else PERM_EINVAL
 *   count  1 <= count <= PERM_NOALLOC_MAX_COUNT, else PERM_EINVAL
 *   out    device, count*4 words: per(A_k) in 256-bit two's complement
 *   status device, count int32: PERM_OK, or PERM_EOVERFLOW (out set to 0)
 *          when an entry or a row's sum of |a_ij| is out of the range above,
 *          or when the bound min(prod_i sum_j |a_ij|, prod_j sum_i |a_ij|)
 *          exceeds 2^(254-n)
 *   stream cudaStream_t; the call only enqueues work and returns.
 * Working memory is one file-scope device array of PERM_NOALLOC_SCRATCH_BYTES
 * that every GPU which loads the library keeps until the process exits.
 * Every call uses that same array and clears it first, so calls whose work
 * overlaps on the GPU (on different streams, or from different host threads
 * at the same time) race and give wrong results; issue them one after
 * another on one stream.  The first call on each device looks up the
 * array's device address (cudaGetSymbolAddress) with that device current;
 * make that first call before any stream capture begins. */
#define PERM_NOALLOC_MAX_COUNT 4096
#define PERM_NOALLOC_SCRATCH_BYTES (256 + 32 * PERM_NOALLOC_MAX_COUNT)
perm_status perm_leaf_batch_noalloc(const int64_t* a, int32_t n, int32_t count, uint64_t* out,
                                    int32_t* status, void* stream);

/* ---- measurement -------------------------------------------------------------- */

/* Integer multiply-add throughput probe: `blocks` x 256 threads each run
 * `iters` iterations of 16 independent 32-bit IMAD chains.  ms receives the
 * kernel time; imad_per_s the executed IMAD rate. */
perm_status perm_ubench_imad(int32_t blocks, int32_t iters, void* stream, float* ms,
                             double* imad_per_s);

/* Human-readable text for a status, and the last CUDA error text seen by
 * this thread. */
const char* perm_status_string(perm_status s);
const char* perm_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* PERM_H_ */
