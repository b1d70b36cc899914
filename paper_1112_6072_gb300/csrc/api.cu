// Host side of the C ABI declared in include/perm.h: validation and
// canonical CSR (a1), the level loop of the expansion (a2, a3), estimate and
// ordering (a4-a6), the two persistent evaluation launches and the sum
// (a7, a8), result recovery, and the learned-model entry points.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <memory>
#include <mutex>
#include <numeric>
#include <thread>
#include <string>
#include <vector>

#include "internal.h"
#include "wide.cuh"

size_t mlp_scratch_floats(int32_t count);

// ---------------------------------------------------------------- errors
static thread_local std::string g_last_error;

void set_last_error(const char* what, cudaError_t e) {
  g_last_error = std::string(what) + ": " + cudaGetErrorString(e);
}

void set_last_error_text(const char* what) noexcept {
  try {
    g_last_error = what;
  } catch (...) {
  }
}

extern "C" const char* perm_last_error(void) { return g_last_error.c_str(); }

extern "C" const char* perm_status_string(perm_status s) {
  switch (s) {
    case PERM_OK: return "ok";
    case PERM_EINVAL: return "invalid argument";
    case PERM_EOVERFLOW: return "value or bound beyond the exact paths";
    case PERM_ETIMEOUT: return "device watchdog expired";
    case PERM_ECUDA: return "CUDA error";
    case PERM_ESHORTBUF: return "output buffer too short";
    case PERM_ENOMEM: return "out of memory";
    case PERM_ESTATE: return "call out of sequence";
  }
  return "unknown status";
}

#define CK(call)                                  \
  do {                                            \
    cudaError_t e_ = (call);                      \
    if (e_ != cudaSuccess) {                      \
      set_last_error(#call, e_);                  \
      return e_ == cudaErrorMemoryAllocation ? PERM_ENOMEM : PERM_ECUDA; \
    }                                             \
  } while (0)

extern "C" void perm_opts_default(perm_opts* o) {
  if (!o) return;
  memset(o, 0, sizeof(*o));
  o->split_depth = -1;
  o->leaf_size = 0;
  o->order = PERM_ORDER_LPT;
  o->kklll_trials = 0;
  o->seed = 0x5EEDull;
  o->workers_per_sm = 0;
  o->chunk_log2 = 0;
  o->stream = nullptr;
  o->timeout_ns = 0;
  o->model_uses_estimate = 1;
  o->fused_levels = 1;
  o->dense_split = 0;
  o->expand_walk = 1;
}

// ---------------------------------------------------------------- memory
// Without a caller allocator, device memory comes from a stream-ordered pool
// of the library's own (one per device) that keeps up to kPoolKeepBytes of
// freed memory mapped, so repeated plans do not map and unmap it again.
static const uint64_t kPoolKeepBytes = 4ull << 30;

static cudaMemPool_t library_pool() {
  static std::mutex mu;
  static std::map<int, cudaMemPool_t> pools;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return nullptr;
  std::lock_guard<std::mutex> lock(mu);
  auto it = pools.find(dev);
  if (it != pools.end()) return it->second;
  cudaMemPoolProps props;
  memset(&props, 0, sizeof(props));
  props.allocType = cudaMemAllocationTypePinned;
  props.location.type = cudaMemLocationTypeDevice;
  props.location.id = dev;
  cudaMemPool_t pool = nullptr;
  if (cudaMemPoolCreate(&pool, &props) != cudaSuccess) return nullptr;
  uint64_t keep = kPoolKeepBytes;
  cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
  pools[dev] = pool;
  return pool;
}

struct Mem {
  perm_opts opts;
  cudaStream_t s;
  cudaMemPool_t pool = nullptr;
  std::vector<void*> live;
  void* get(size_t bytes) {
    if (bytes == 0) bytes = 16;
    void* p = nullptr;
    if (opts.alloc) {
      p = opts.alloc(bytes, (void*)s, opts.alloc_ctx);
    } else if ((pool ? cudaMallocFromPoolAsync(&p, bytes, pool, s) : cudaMallocAsync(&p, bytes, s)) !=
               cudaSuccess) {
      p = nullptr;
    }
    if (p) live.push_back(p);
    return p;
  }
  void put(void* p) {
    if (!p) return;
    auto it = std::find(live.begin(), live.end(), p);
    if (it != live.end()) live.erase(it);
    if (opts.alloc && opts.free)
      opts.free(p, (void*)s, opts.alloc_ctx);
    else
      cudaFreeAsync(p, s);
  }
  void release_all() {
    for (void* p : live) {
      if (opts.alloc && opts.free)
        opts.free(p, (void*)s, opts.alloc_ctx);
      else
        cudaFreeAsync(p, s);
    }
    live.clear();
  }
};

template <typename T>
static T* dget(Mem& M, int64_t n) {
  return reinterpret_cast<T*>(M.get(sizeof(T) * (size_t)(n > 0 ? n : 1)));
}

static bool alloc_jobs(Mem& M, JobArrays& a, int64_t n) {
  a.m = dget<int32_t>(M, n);
  a.nnz = dget<int32_t>(M, n);
  a.off = dget<int64_t>(M, n);
  a.mat = dget<int32_t>(M, n);
  a.depth_left = dget<int32_t>(M, n);
  a.coef = dget<uint64_t>(M, 4 * n);
  return a.m && a.nnz && a.off && a.mat && a.depth_left && a.coef;
}

static void free_jobs(Mem& M, JobArrays& a) {
  M.put(a.m);
  M.put(a.nnz);
  M.put(a.off);
  M.put(a.mat);
  M.put(a.depth_left);
  M.put(a.coef);
  memset(&a, 0, sizeof(a));
}

// A device buffer that only grows (by at least half its size), so a level
// loop reuses it instead of allocating per level.
struct Grow {
  void* p = nullptr;
  size_t cap = 0;
};

static bool grow(Mem& M, Grow& g, size_t bytes) {
  if (bytes <= g.cap && g.p) return true;
  M.put(g.p);
  const size_t nb = std::max(bytes, g.cap + g.cap / 2);
  g.p = M.get(nb);
  g.cap = g.p ? nb : 0;
  return g.p != nullptr;
}

// Job header arrays with a capacity.
struct JobBuf {
  Grow m, nnz, off, mat, dl, coef;
  bool ensure(Mem& M, int64_t n) {
    const size_t k = (size_t)std::max<int64_t>(n, 1);
    return grow(M, m, 4 * k) && grow(M, nnz, 4 * k) && grow(M, off, 8 * k) && grow(M, mat, 4 * k) &&
           grow(M, dl, 4 * k) && grow(M, coef, 32 * k);
  }
  JobArrays view() const {
    JobArrays a;
    a.m = reinterpret_cast<int32_t*>(m.p);
    a.nnz = reinterpret_cast<int32_t*>(nnz.p);
    a.off = reinterpret_cast<int64_t*>(off.p);
    a.mat = reinterpret_cast<int32_t*>(mat.p);
    a.depth_left = reinterpret_cast<int32_t*>(dl.p);
    a.coef = reinterpret_cast<uint64_t*>(coef.p);
    return a;
  }
  void free(Mem& M) {
    for (Grow* g : {&m, &nnz, &off, &mat, &dl, &coef}) {
      M.put(g->p);
      g->p = nullptr;
      g->cap = 0;
    }
  }
  void release_ownership() {
    for (Grow* g : {&m, &nnz, &off, &mat, &dl, &coef}) {
      g->p = nullptr;
      g->cap = 0;
    }
  }
};

// Prepared evaluation of one queue: host-side split into leaf and
// depth-first queues, leaf kernel variants, and the device buffers the
// launches use.  Kept with the job set so the launch sequence can be
// captured once into a CUDA graph and replayed.
// E.sum layout: status summary, retry positions, evaluation key histogram
#define SUM_STATUS 0
#define SUM_RETRY 1
#define SUM_HIST (SUM_RETRY + EVAL_DFS_GROUPS + 1)
#define SUM_RFLAG (SUM_HIST + EVAL_KEYS)  // single-launch mode: a depth-first job handed on
#define SUM_WORDS (SUM_RFLAG + 1)

// depth-first group g of the grouped queue: tile 64 first, ring width 2 then 4
static inline int dfs_group_tile(int g) { return g >= 2 ? 32 : 64; }
static inline int dfs_group_w(int g) { return (g & 1) ? 4 : 2; }

struct EvalState {
  int64_t nq = 0;  // queue length (all jobs, or the subset given)
  int64_t nl = 0, nd = 0;
  int64_t db[EVAL_DFS_GROUPS + 1] = {0, 0, 0, 0, 0};  // depth-first group bounds in d_dq
  std::vector<std::pair<int64_t, int64_t>> groups;  // (offset, count) in the grouped leaf queue
  std::vector<int32_t> group_cls;
  uint32_t* d_q = nullptr;   // the queue as evaluated
  uint32_t* d_g = nullptr;   // grouped queue: leaf variants, then depth-first W = 2, W = 4
  uint32_t* d_lq = nullptr;  // = d_g
  uint32_t* d_dq = nullptr;  // = d_g + nl
  uint32_t* d_rq = nullptr;  // retry queue
  int32_t* rflags = nullptr;
  int32_t* rpos = nullptr;
  uint64_t* counts = nullptr;
  uint64_t* prefix = nullptr;
  uint32_t* owner = nullptr;  // task -> grouped leaf queue position
  void* stmp = nullptr;
  size_t stb = 0;
  unsigned long long* ctr = nullptr;  // [0] leaf tasks, [1 + g] depth-first group g
  unsigned long long* sum = nullptr;  // SUM_WORDS entries
  int64_t* undo = nullptr;
  int64_t undo_w = 0;
  int frames = 64;
  int chunk = 10;
  bool wide_first = false;
  // single-launch mode (perm_opts.single_launch)
  bool single = false;
  int single_w = 2;                 // ring words of the persistent kernel (0: residues)
  uint32_t* keys = nullptr;         // evaluation key per queue position
  unsigned long long* pctr = nullptr;  // [0] queue positions taken, [1] board
  uint32_t* task_ctr = nullptr;     // 2 * nq: tasks taken, tasks finished
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  cudaStream_t cap = nullptr;
};

// ---------------------------------------------------------------- handles
struct perm_jobs {
  perm_plan* plan = nullptr;
  int64_t n = 0;
  JobArrays a{};
  uint64_t* arena = nullptr;
  int64_t arena_words = 0;
  int max_order = 0;
  std::vector<int32_t> h_m;
  std::vector<int64_t> order_count;  // jobs per order (PERM_MAX_N + 1 entries)
  uint32_t* d_queue = nullptr;
  bool has_order = false;
  float* d_logap = nullptr;
  bool has_logap = false;
  JobOut out{};
  EvalState* ev = nullptr;
};

static void free_eval(Mem& M, perm_jobs* J) {
  EvalState* E = J->ev;
  if (!E) return;
  if (E->exec) cudaGraphExecDestroy(E->exec);
  if (E->graph) cudaGraphDestroy(E->graph);
  if (E->cap) cudaStreamDestroy(E->cap);
  for (void* p : {(void*)E->d_q, (void*)E->d_g, (void*)E->d_rq, (void*)E->rflags, (void*)E->rpos,
                  (void*)E->counts, (void*)E->prefix, (void*)E->owner, E->stmp, (void*)E->ctr, (void*)E->sum,
                  (void*)E->undo, (void*)E->keys, (void*)E->pctr, (void*)E->task_ctr})
    M.put(p);
  delete E;
  J->ev = nullptr;
}

// Host words left uninitialised on allocation: every word is written by
// the thread that fills its block (a zero fill of the whole arena would run
// on one thread).
struct HostWords {
  std::unique_ptr<uint64_t[]> p;
  size_t n = 0;
  void alloc(size_t k) {
    p.reset(new uint64_t[k > 0 ? k : 1]);
    n = k;
  }
  uint64_t* data() const { return p.get(); }
  size_t size() const { return n; }
};

struct perm_plan {
  perm_opts opts{};
  cudaStream_t s = nullptr;
  Mem M;
  int count = 0;
  int sms = 0;
  int L = 0;
  bool leaf_only = false;
  std::vector<int32_t> n, w, kbits, depth;
  std::vector<int8_t> trivial;  // 0 none, 1 per = 0, 2 per = 1
  HostWords h_arena;
  std::vector<int64_t> h_off;
  std::vector<int32_t> h_nnz;
  int32_t* d_mat_w = nullptr;
  unsigned long long* d_mat_acc = nullptr;
  perm_jobs* jobs = nullptr;
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;  // around the last evaluation
  cudaEvent_t xe0 = nullptr, xe1 = nullptr;  // around the last expansion
  float last_ms = 0.f;
  float last_expand_ms = 0.f;
  int32_t last_launches = 0;
  bool evaluated = false;
  bool subset = false;  // the last evaluation covered a sub-queue (perm_eval_subset)
  int32_t expand_driver = -1;  // driver of the last expansion: 0 levels, 1 fused levels, 2 traversal
  std::vector<float> mlp;
  ModP mod{0u, 0u, 0u};        // p = 0: the exact ring path; else the residue path modulo p
};

// ---------------------------------------------------------------- a1: plan
static double log2_bound(const perm_matrix& A, bool& binary) {
  // min(prod of row abs sums, prod of column abs sums), and Bregman's bound
  // prod (r_i!)^(1/r_i) for 0/1 matrices (valid for per of a 0/1 matrix)
  const int n = A.n;
  double rs[PERM_MAX_N], cs[PERM_MAX_N];
  int rc[PERM_MAX_N];
  for (int i = 0; i < n; ++i) {
    rs[i] = cs[i] = 0.0;
    rc[i] = 0;
  }
  binary = true;
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) {
      const int64_t v = A.a[(size_t)i * A.ld + j];
      const double av = std::fabs((double)v);
      rs[i] += av;
      cs[j] += av;
      if (v != 0) rc[i]++;
      if (v != 0 && v != 1) binary = false;
    }
  double lr = 0, lc = 0, lb = 0;
  for (int i = 0; i < n; ++i) {
    lr += std::log2(rs[i]);
    lc += std::log2(cs[i]);
    if (rc[i] > 0) lb += std::lgamma((double)rc[i] + 1.0) / (double)rc[i] / std::log(2.0);
  }
  double b = std::min(lr, lc);
  if (binary) b = std::min(b, lb);
  return b;
}

static int count_nnz(const perm_matrix& A) {
  int nnz = 0;
  for (int i = 0; i < A.n; ++i)
    for (int j = 0; j < A.n; ++j) nnz += A.a[(size_t)i * A.ld + j] != 0;
  return nnz;
}

// CSR block of A (nnz nonzeros) into b (blk_words(n, nnz) zeroed words)
static void put_csr(uint64_t* b, const perm_matrix& A, int nnz) {
  const int n = A.n;
  std::memset(b, 0, 8 * (size_t)blk_words(n, nnz));
  uint16_t* rp = reinterpret_cast<uint16_t*>(b);
  uint8_t* col = reinterpret_cast<uint8_t*>(b + blk_rp_words(n));
  int64_t* val = reinterpret_cast<int64_t*>(b + blk_rp_words(n) + blk_col_words(nnz));
  int k = 0;
  for (int i = 0; i < n; ++i) {
    rp[i] = (uint16_t)k;
    for (int j = 0; j < n; ++j) {
      const int64_t v = A.a[(size_t)i * A.ld + j];
      if (v != 0) {
        col[k] = (uint8_t)j;
        val[k] = v;
        ++k;
      }
    }
  }
  rp[n] = (uint16_t)k;
}

// fn(i) for i in [0, count): on up to 16 host threads for large batches
template <class F>
static void parallel_for(int32_t count, F fn) {
  unsigned th = std::thread::hardware_concurrency();
  th = th == 0 ? 1 : (th > 16 ? 16 : th);
  if (count < 4096 || th == 1) {
    for (int32_t i = 0; i < count; ++i) fn(i);
    return;
  }
  std::vector<std::thread> pool;
  const int32_t chunk = (count + (int32_t)th - 1) / (int32_t)th;
  for (unsigned t = 0; t < th; ++t) {
    const int32_t lo = (int32_t)t * chunk, hi = std::min(count, lo + chunk);
    if (lo >= hi) break;
    pool.emplace_back([lo, hi, &fn]() {
      for (int32_t i = lo; i < hi; ++i) fn(i);
    });
  }
  for (auto& t : pool) t.join();
}

static perm_status perm_plan_create_impl(const perm_matrix* mats, int32_t count, const perm_opts* opts,
                                         perm_plan_t** out) {
  if (!out || !mats || count < 1) return PERM_EINVAL;
  *out = nullptr;
  perm_opts o;
  if (opts) o = *opts; else perm_opts_default(&o);
  if (o.leaf_size < 0 || o.leaf_size > PERM_MAX_LEAF) return PERM_EINVAL;
  if (o.chunk_log2 < 0 || o.chunk_log2 > 30) return PERM_EINVAL;
  int maxn = 0;
  for (int32_t i = 0; i < count; ++i) {
    const perm_matrix& A = mats[i];
    if (A.n < 0 || A.n > PERM_MAX_N || A.ld < A.n || (A.n > 0 && !A.a)) return PERM_EINVAL;
    maxn = std::max(maxn, A.n);
  }
  // residue path: every entry reduced into [0, p) first (a copy); the rest
  // of the set-up then sees residues, and no magnitude bound applies
  std::vector<std::vector<int64_t>> red;
  std::vector<perm_matrix> red_mats;
  if (o.modulus) {
    if (!modp_is_odd_prime(o.modulus)) return PERM_EINVAL;
    red.resize(count);
    red_mats.resize(count);
    parallel_for(count, [&](int32_t i) {
      const perm_matrix& A = mats[i];
      red[i].resize((size_t)A.n * A.n + 1);
      for (int r = 0; r < A.n; ++r)
        for (int c = 0; c < A.n; ++c) red[i][(size_t)r * A.n + c] = mod_of(A.a[(size_t)r * A.ld + c], o.modulus);
      red_mats[i] = perm_matrix{A.n, red[i].data(), std::max<int32_t>(A.n, 1)};
    });
    mats = red_mats.data();
  }
  perm_plan* P = new perm_plan();
  P->mod = o.modulus ? modp_make(o.modulus) : ModP{0u, 0u, 0u};
  P->opts = o;
  P->s = (cudaStream_t)o.stream;
  P->M.opts = o;
  P->M.s = P->s;
  if (!o.alloc) P->M.pool = library_pool();
  P->count = count;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&P->sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) {
    set_last_error("cudaDeviceGetAttribute", e);
    delete P;
    return PERM_ECUDA;
  }
  // leaf order and split depth
  P->leaf_only = (o.split_depth <= 0 && maxn <= PERM_MAX_LEAF && (o.leaf_size == 0 || o.leaf_size >= maxn));
  P->L = o.leaf_size > 0 ? o.leaf_size : (P->leaf_only ? std::max(maxn, 2) : 12);
  P->n.resize(count);
  P->w.resize(count);
  P->kbits.resize(count);
  P->depth.resize(count);
  P->trivial.assign(count, 0);
  P->h_off.assign(count, -1);
  P->h_nnz.assign(count, 0);
  // per matrix, in parallel: entry range, trivial cases, ring width from the
  // bound, nonzeros
  std::vector<uint8_t> over(count, 0), bad(count, 0);
  parallel_for(count, [&](int32_t i) {
    const perm_matrix& A = mats[i];
    for (int r = 0; r < A.n; ++r)
      for (int c = 0; c < A.n; ++c) {
        const int64_t v = A.a[(size_t)r * A.ld + c];
        if (v >= (1ll << 31) || v <= -(1ll << 31)) bad[i] = 1;
      }
    if (bad[i]) return;
    P->n[i] = A.n;
    P->depth[i] = P->leaf_only ? 0 : o.split_depth;  // -1: chosen during the expansion
    if (A.n == 0) {
      P->trivial[i] = 2;
      P->w[i] = 2;
      P->kbits[i] = 64;
      return;
    }
    // zero line -> per = 0
    bool zero = false;
    for (int r = 0; r < A.n && !zero; ++r) {
      bool rz = true, cz = true;
      for (int c = 0; c < A.n; ++c) {
        rz = rz && A.a[(size_t)r * A.ld + c] == 0;
        cz = cz && A.a[(size_t)c * A.ld + r] == 0;
      }
      zero = rz || cz;
    }
    if (zero) {
      P->trivial[i] = 1;
      P->w[i] = 2;
      P->kbits[i] = 64;
      return;
    }
    if (o.modulus) {  // results are residues: one ring width, no bound
      P->w[i] = 2;
      P->kbits[i] = 0;
      P->h_nnz[i] = count_nnz(A);
      return;
    }
    bool binary;
    const double lb = log2_bound(A, binary);
    const int need = (int)std::ceil(lb + 1e-9) + 2;  // |per| < 2^(need-1)
    // leaves have order <= Lmax: results are exact modulo 2^(64W - Lmax + 1)
    const int lmax = P->leaf_only ? A.n : PERM_MAX_LEAF;
    if (need <= 129 - lmax) {
      P->w[i] = 2;
      P->kbits[i] = 129 - lmax;
    } else if (need <= 257 - lmax) {
      P->w[i] = 4;
      P->kbits[i] = 257 - lmax;
    } else {
      over[i] = 1;
      return;
    }
    P->h_nnz[i] = count_nnz(A);
  });
  for (uint8_t b : bad)
    if (b) {
      delete P;
      return PERM_EINVAL;
    }
  for (uint8_t b : over)
    if (b) {
      delete P;
      return PERM_EOVERFLOW;
    }
  // blocks back to back in matrix order, filled in parallel
  int64_t words = 0;
  for (int32_t i = 0; i < count; ++i) {
    if (P->trivial[i]) continue;
    P->h_off[i] = words;
    words += blk_words(P->n[i], P->h_nnz[i]);
  }
  P->h_arena.alloc((size_t)words);
  parallel_for(count, [&](int32_t i) {
    if (!P->trivial[i]) put_csr(P->h_arena.data() + P->h_off[i], mats[i], P->h_nnz[i]);
  });
  P->d_mat_w = dget<int32_t>(P->M, count);
  P->d_mat_acc = dget<unsigned long long>(P->M, 4ll * count);
  if (!P->d_mat_w || !P->d_mat_acc) {
    P->M.release_all();
    delete P;
    return PERM_ENOMEM;
  }
  e = cudaMemcpyAsync(P->d_mat_w, P->w.data(), sizeof(int32_t) * count, cudaMemcpyHostToDevice, P->s);
  if (e == cudaSuccess) e = cudaMemsetAsync(P->d_mat_acc, 0, 32ull * count, P->s);
  if (e == cudaSuccess) e = cudaEventCreate(&P->ev0);
  if (e == cudaSuccess) e = cudaEventCreate(&P->ev1);
  if (e == cudaSuccess) e = cudaEventCreate(&P->xe0);
  if (e == cudaSuccess) e = cudaEventCreate(&P->xe1);
  if (e != cudaSuccess) {
    set_last_error("plan upload", e);
    P->M.release_all();
    delete P;
    return PERM_ECUDA;
  }
  *out = P;
  return PERM_OK;
}
extern "C" perm_status perm_plan_create(const perm_matrix* mats, int32_t count, const perm_opts* opts,
                                        perm_plan_t** out) {
  return guarded([&] { return perm_plan_create_impl(mats, count, opts, out); });
}

static void free_jobset(perm_plan* P) {
  perm_jobs* J = P->jobs;
  if (!J) return;
  free_eval(P->M, J);
  free_jobs(P->M, J->a);
  P->M.put(J->arena);
  P->M.put(J->d_queue);
  P->M.put(J->d_logap);
  P->M.put(J->out.acc);
  P->M.put(J->out.t_start);
  P->M.put(J->out.t_end);
  P->M.put(J->out.sm);
  P->M.put(J->out.status);
  P->M.put(J->out.leaves);
  P->M.put(J->out.nodes);
  delete J;
  P->jobs = nullptr;
}

extern "C" void perm_plan_destroy(perm_plan_t* P) {
  if (!P) return;
  cudaStreamSynchronize(P->s);
  free_jobset(P);
  P->M.release_all();
  if (P->ev0) cudaEventDestroy(P->ev0);
  if (P->ev1) cudaEventDestroy(P->ev1);
  if (P->xe0) cudaEventDestroy(P->xe0);
  if (P->xe1) cudaEventDestroy(P->xe1);
  cudaStreamSynchronize(P->s);
  delete P;
}

// ---------------------------------------------------------------- a2, a3: expansion
static const int64_t kTargetJobs = 1ll << 17;
// automatic depth: a level splits the jobs within this many orders of the
// largest job still to split
static const int kSplitBand = 2;
// automatic depth: jobs above this order are split further while the job
// count is below kSoftCapJobs (the depth-first evaluator holds three times
// as many warps per SM for jobs of order <= 32)
static const int kSoftOrder = 32;
static const int64_t kSoftCapJobs = 1ll << 25;
// fused (single-launch) expansion buffers: initial and largest capacities
static const int64_t kFusedJobs0 = 1ll << 17;
static const int64_t kFusedWords0 = 1ll << 23;
static const int64_t kFusedMaxJobs = 1ll << 20;
static const int64_t kFusedMaxWords = 1ll << 26;

static perm_status finish_jobset(perm_plan* P, perm_jobs* J, perm_jobs_t** jobs_out, int64_t* njobs);

// ---- a3 by the traversal driver (walk.cu) --------------------------------------
// jobs per traversal (outputs and queue slots) with a fixed depth
static const int64_t kWalkJobs = 1ll << 19;
// output slots a warp of the traversal reserves at a time (walk.cu)
static const int64_t kWalkOutChunk = 16;

struct WalkRoots {
  std::vector<int32_t> m, nnz, mat, dl;
  std::vector<int64_t> off;
};

// Expand the roots by the traversal.  done = false (and PERM_OK) when it does
// not apply or its buffers filled: the caller then runs the level-by-level
// driver.  levels_left replays the automatic depth rule from the per-depth
// counts; with the automatic depth the traversal runs to the end of the tree
// and is accepted when the rule reaches that depth, else it runs again with
// the depth the rule stops at.
template <class LevelsLeft>
static perm_status expand_by_walk(perm_plan* P, perm_jobs* J, WalkRoots R, int maxd, int max_open0, bool adaptive,
                                  int64_t target, LevelsLeft levels_left, bool& done) {
  done = false;
  Mem& M = P->M;
  cudaStream_t s = P->s;
  const int64_t nroots = (int64_t)R.m.size();
  const int K = P->opts.dense_split ? 3 : 2;
  const int bpl = K == 3 ? 2 : 1;
  int maxn = 0, minn = 1 << 30;
  int64_t sw = 2;
  for (int64_t r = 0; r < nroots; ++r) {
    maxn = std::max(maxn, R.m[r]);
    minn = std::min(minn, R.m[r]);
    sw = std::max<int64_t>(sw, blk_words(R.m[r], R.nnz[r]));
  }
  // the automatic depth's waiting band only matters for roots of several orders (or Eq. 2's third child)
  if (nroots == 0 || (adaptive && (K == 3 || minn != maxn))) return PERM_OK;
  int rbits = 0;
  while ((1ll << rbits) < nroots) ++rbits;
  const int key_bits = rbits + bpl * maxd;
  if (key_bits > 127) return PERM_OK;
  const int hist_len = maxd + 1;
  if (walk_tile_for(maxn) == 0) return PERM_OK;
  // phases: a 64-wide tile for the nodes above order 32, which hands the
  // nodes of order <= 32 to a 32-wide tile (more warps per SM)
  const bool wide_phase = maxn > 32;
  const int stage = (int)std::min<int64_t>((sw + 1) & ~1ll, 512);
  int64_t warps32 = 0, warps64 = 0;
  CK(walk_resident_warps(32, stage, hist_len, P->sms, &warps32));
  if (wide_phase) CK(walk_resident_warps(64, stage, hist_len, P->sms, &warps64));
  if (warps32 <= 0 || (wide_phase && warps64 <= 0)) return PERM_OK;
  // undo frames: a path below its subtree root is at most the order span of its phase
  // (Eq. 2's third child keeps the order: then the whole depth)
  const int frames32 = std::max(1, K == 3 ? maxd : std::min(maxd, 32));
  const int frames64 = std::max(1, K == 3 ? maxd : std::min(maxd, 64));
  const int64_t undo_words = std::max(warps32 * frames32 * walk_frame_words(32),
                                      wide_phase ? warps64 * frames64 * walk_frame_words(64) : 0);
  const int64_t hw = (int64_t)P->h_arena.size();
  // jobs, plus the slots a warp may leave unused in its last reserved chunk
  // (at most 64 resident warps per SM)
  const int64_t jobs_cap = adaptive ? 2 * target : kWalkJobs;
  const int64_t cap = jobs_cap + (int64_t)P->sms * 64 * kWalkOutChunk;
  const int64_t chunk = std::max<int64_t>(256, 2 * sw);
  // blocks: every job's and every handed-over node's, plus each warp's last chunk
  const int64_t cap_words =
      ((hw + 1) & ~1ll) + jobs_cap * std::max<int64_t>(96, sw / 2) + (int64_t)P->sms * 64 * chunk;
  // device buffers
  auto alloc_queue = [&](WalkQueue& Q, int64_t n) {
    Q.m = dget<int32_t>(M, n);
    Q.nnz = dget<int32_t>(M, n);
    Q.mat = dget<int32_t>(M, n);
    Q.dl = dget<int32_t>(M, n);
    Q.depth = dget<int32_t>(M, n);
    Q.off = dget<int64_t>(M, n);
    Q.coef = dget<uint64_t>(M, 4 * n);
    Q.key = dget<uint64_t>(M, 2 * n);
    Q.ready = dget<int32_t>(M, n);
    Q.cap = n;
    return Q.m && Q.nnz && Q.mat && Q.dl && Q.depth && Q.off && Q.coef && Q.key && Q.ready;
  };
  auto free_queue = [&](WalkQueue& Q) {
    for (void* p : {(void*)Q.m, (void*)Q.nnz, (void*)Q.mat, (void*)Q.dl, (void*)Q.depth, (void*)Q.off,
                    (void*)Q.coef, (void*)Q.key, (void*)Q.ready})
      M.put(p);
  };
  WalkQueue Q1{}, Q2{};
  const bool q_ok = alloc_queue(Q1, cap) && alloc_queue(Q2, cap);
  JobArrays out{};
  const bool out_ok = alloc_jobs(M, out, cap);
  uint64_t* out_key = dget<uint64_t>(M, 2 * cap);
  uint64_t* arena = dget<uint64_t>(M, cap_words);
  // [0, 1] work queue head, tail; [2] outstanding; [3] arena words; [4] output slots;
  // [5] jobs; [6] status; [7, 8] hand-over queue head, tail
  unsigned long long* ctr = dget<unsigned long long>(M, 10);
  unsigned long long* hist = dget<unsigned long long>(M, 2 * hist_len);
  int32_t* hmo = dget<int32_t>(M, hist_len);
  int64_t* undo = dget<int64_t>(M, undo_words);
  auto release = [&](bool keep_arena) {
    free_queue(Q1);
    free_queue(Q2);
    for (void* p : {(void*)out_key, (void*)ctr, (void*)hist, (void*)hmo, (void*)undo}) M.put(p);
    free_jobs(M, out);
    if (!keep_arena) M.put(arena);
  };
  if (!q_ok || !out_ok || !out_key || !arena || !ctr || !hist || !hmo || !undo) {
    release(false);
    return PERM_OK;  // too large for the traversal's buffers: the level-by-level driver grows its own
  }
  Q1.head = ctr + 0;
  Q1.tail = ctr + 1;
  Q2.head = ctr + 7;
  Q2.tail = ctr + 8;
  WalkArgs A{};
  A.outstanding = ctr + 2;
  A.arena_used = ctr + 3;
  A.out_used = ctr + 4;
  A.emitted = ctr + 5;
  A.err = reinterpret_cast<int32_t*>(ctr + 6);
  A.arena = arena;
  A.cap_words = cap_words;
  A.arena_chunk = chunk;
  A.out = out;
  A.out_key = out_key;
  A.cap_out = cap;
  A.hist_nodes = hist;
  A.hist_term = hist + hist_len;
  A.hist_maxopen = hmo;
  A.hist_len = hist_len;
  A.leaf_size = P->L;
  A.kslots = K;
  A.bits_per_level = bpl;
  A.key_levels = maxd;
  A.stage_words = stage;
  A.undo = undo;
  // an idle warp waits for the others' remaining work: at least a second,
  // whatever the evaluation watchdog
  A.timeout_ns = std::max<int64_t>(P->opts.timeout_ns > 0 ? P->opts.timeout_ns : 10000000000ll, 1000000000ll);
  A.mod = P->mod.p;
  // roots: blocks back to back at the start of the arena, queue slots [0, nroots)
  std::vector<uint64_t> coef(4 * nroots, 0ull), key(2 * nroots, 0ull);
  std::vector<int32_t> depth0(nroots, 0), ones(nroots, 1);
  for (int64_t r = 0; r < nroots; ++r) {
    coef[4 * r] = 1;
    const u128 k = (u128)r << (bpl * maxd);
    key[2 * r] = (uint64_t)k;
    key[2 * r + 1] = (uint64_t)(k >> 64);
  }
  CK(cudaMemcpyAsync(arena, P->h_arena.data(), 8 * hw, cudaMemcpyHostToDevice, s));
  CK(cudaMemcpyAsync(Q1.m, R.m.data(), 4 * nroots, cudaMemcpyHostToDevice, s));
  CK(cudaMemcpyAsync(Q1.nnz, R.nnz.data(), 4 * nroots, cudaMemcpyHostToDevice, s));
  CK(cudaMemcpyAsync(Q1.mat, R.mat.data(), 4 * nroots, cudaMemcpyHostToDevice, s));
  CK(cudaMemcpyAsync(Q1.depth, depth0.data(), 4 * nroots, cudaMemcpyHostToDevice, s));
  CK(cudaMemcpyAsync(Q1.off, R.off.data(), 8 * nroots, cudaMemcpyHostToDevice, s));
  CK(cudaMemcpyAsync(Q1.coef, coef.data(), 32 * nroots, cudaMemcpyHostToDevice, s));
  CK(cudaMemcpyAsync(Q1.key, key.data(), 16 * nroots, cudaMemcpyHostToDevice, s));
  bool fixed_rerun = false;
  for (int attempt = 0; attempt < 2; ++attempt) {
    CK(cudaMemcpyAsync(Q1.dl, R.dl.data(), 4 * nroots, cudaMemcpyHostToDevice, s));
    CK(cudaMemsetAsync(Q1.ready, 0, 4 * (size_t)cap, s));
    CK(cudaMemsetAsync(Q2.ready, 0, 4 * (size_t)cap, s));
    CK(cudaMemcpyAsync(Q1.ready, ones.data(), 4 * nroots, cudaMemcpyHostToDevice, s));
    CK(cudaMemsetAsync(out_key, 0xff, 16 * (size_t)cap, s));
    CK(cudaMemsetAsync(hist, 0, 16 * (size_t)hist_len, s));
    CK(cudaMemsetAsync(hmo, 0, 4 * (size_t)hist_len, s));
    unsigned long long c0[10] = {0, (unsigned long long)nroots, (unsigned long long)nroots,
                                 (unsigned long long)((hw + 1) & ~1ll), 0, 0, 0, 0, 0, 0};
    CK(cudaMemcpyAsync(ctr, c0, sizeof(c0), cudaMemcpyHostToDevice, s));
    int grid = 1;
    if (wide_phase) {
      A.q = Q1;
      A.hand = Q2;
      A.handover_order = 32;
      A.undo_words_per_warp = (int64_t)frames64 * walk_frame_words(64);
      A.max_rel_depth = frames64;
      A.warps_cap = warps64;
      CK(launch_expand_walk(A, 64, P->sms, &grid, s));
      // the narrower phase's work: the nodes handed over
      CK(cudaMemcpyAsync(ctr + 2, ctr + 8, 8, cudaMemcpyDeviceToDevice, s));
    }
    if (grid > 0) {
      A.q = wide_phase ? Q2 : Q1;
      A.hand = WalkQueue{};
      A.handover_order = 0;
      A.undo_words_per_warp = (int64_t)frames32 * walk_frame_words(32);
      A.max_rel_depth = frames32;
      A.warps_cap = warps32;
      CK(launch_expand_walk(A, 32, P->sms, &grid, s));
    }
    unsigned long long c1[10];
    std::vector<unsigned long long> hh(2 * hist_len);
    std::vector<int32_t> hm(hist_len);
    CK(cudaMemcpyAsync(c1, ctr, sizeof(c1), cudaMemcpyDeviceToHost, s));
    if (adaptive && !fixed_rerun) {
      CK(cudaMemcpyAsync(hh.data(), hist, 16 * hist_len, cudaMemcpyDeviceToHost, s));
      CK(cudaMemcpyAsync(hm.data(), hmo, 4 * hist_len, cudaMemcpyDeviceToHost, s));
    }
    CK(cudaStreamSynchronize(s));
    const int32_t err = (int32_t)(c1[6] & 0xffffffffu);
    if (grid == 0 || err == WALK_FULL) {
      release(false);
      return PERM_OK;
    }
    if (err != 0) {
      release(false);
      return (perm_status)err;
    }
    if (adaptive && !fixed_rerun) {
      // replay the automatic depth rule on the per-depth counts
      int64_t count = nroots, tcum = 0;
      int mopen = max_open0, D = 0;
      for (int level = 0;; ++level) {
        if (!levels_left(level, count, mopen) || level >= maxd) {
          D = level;
          break;
        }
        tcum += (int64_t)hh[hist_len + level];
        count = tcum + (int64_t)hh[level + 1];
        mopen = hm[level + 1];
      }
      if (hh[D] != hh[hist_len + D]) {
        // the rule stops above the end of the tree: the cut at depth D, as a fixed depth
        for (int64_t r = 0; r < nroots; ++r) R.dl[r] = D;
        fixed_rerun = true;
        continue;
      }
    }
    // the jobs in path-key order
    const int64_t used = (int64_t)c1[4] < cap ? (int64_t)c1[4] : cap;
    const int64_t nj = (int64_t)c1[5];
    uint64_t* kb = dget<uint64_t>(M, 2 * std::max<int64_t>(used, 1));
    uint32_t* ib = dget<uint32_t>(M, 2 * std::max<int64_t>(used, 1));
    const size_t tb = sort_tmp_bytes_u64(std::max<int64_t>(used, 1));
    void* tmp = M.get(tb);
    JobArrays fin{};
    const bool fin_ok = alloc_jobs(M, fin, std::max<int64_t>(nj, 1));
    if (!kb || !ib || !tmp || !fin_ok) {
      M.put(kb);
      M.put(ib);
      M.put(tmp);
      free_jobs(M, fin);
      release(false);
      return PERM_ENOMEM;
    }
    CK(launch_walk_order(out_key, used, key_bits, kb, kb + used, ib, ib + used, tmp, tb, s));
    CK(launch_walk_gather(ib + used, nj, out, fin, s));
    CK(cudaStreamSynchronize(s));
    M.put(kb);
    M.put(ib);
    M.put(tmp);
    release(true);
    J->n = nj;
    J->a = fin;
    J->arena = arena;
    J->arena_words = (int64_t)std::min<unsigned long long>(c1[3], (unsigned long long)cap_words);
    P->expand_driver = 2;
    done = true;
    return PERM_OK;
  }
  release(false);
  return PERM_OK;
}

static perm_status perm_expand_impl(perm_plan_t* P, perm_jobs_t** jobs_out, int64_t* njobs) {
  if (!P) return PERM_EINVAL;
  free_jobset(P);
  P->evaluated = false;
  cudaStream_t s = P->s;
  CK(cudaEventRecord(P->xe0, s));
  Mem& M = P->M;
  // roots
  std::vector<int32_t> rm, rnnz, rmat, rdl;
  std::vector<int64_t> roff;
  int maxn = 0, maxd = 0;
  int max_open = 0;  // largest order of a job still to split
  bool adaptive = false;
  for (int i = 0; i < P->count; ++i) {
    if (P->trivial[i]) continue;
    rm.push_back(P->n[i]);
    rnnz.push_back(P->h_nnz[i]);
    roff.push_back(P->h_off[i]);
    rmat.push_back(i);
    int d = P->depth[i];
    if (d < 0) {
      adaptive = true;
      d = P->n[i];
    }
    rdl.push_back(d);
    maxn = std::max(maxn, P->n[i]);
    maxd = std::max(maxd, d);
    if (d > 0 && P->n[i] > std::max(P->L, 2)) max_open = std::max(max_open, P->n[i]);
  }
  const int64_t nroots = (int64_t)rm.size();
  perm_jobs* J = new perm_jobs();
  J->plan = P;
  P->jobs = J;
  // about 2^17 jobs per matrix, at most 2^21 for a batch (enough queue for
  // every worker many times over)
  const int64_t target = kTargetJobs * std::min<int64_t>(16, std::max<int64_t>(1, nroots));
  // automatic depth: split while a job still to split is above
  // PERM_MAX_JOB_N, or above kSoftOrder while the jobs number fewer than
  // kSoftCapJobs, or while there are fewer jobs than the target; each
  // level splits only the jobs within kSplitBand orders of the largest one
  // still to split (the largest jobs first, so the matrices of a batch end
  // with jobs of similar order), the others wait
  auto levels_left = [&](int level, int64_t n, int mopen) {
    if (level >= maxd || n <= 0) return false;
    if (!adaptive) return true;
    return mopen > PERM_MAX_JOB_N || (mopen > kSoftOrder && n < kSoftCapJobs) || (n < target && mopen > 0);
  };
  if (P->opts.expand_walk && nroots > 0) {
    WalkRoots WR{rm, rnnz, rmat, rdl, roff};
    bool done = false;
    const perm_status st = expand_by_walk(P, J, WR, maxd, max_open, adaptive, target, levels_left, done);
    if (st != PERM_OK) return st;
    if (done) return finish_jobset(P, J, jobs_out, njobs);
  }
  // ping-pong job arrays and arenas, grown geometrically and reused across levels
  JobBuf jb[2];
  Grow ar[2], g_words, g_base, g_valid, g_pos, g_tmp;
  JobBuf slots;
  int cb = 0;  // index of the current level's buffers
  int64_t ncur = nroots;
  if (!jb[0].ensure(M, std::max<int64_t>(nroots, 1)) ||
      !grow(M, ar[0], 8 * (size_t)std::max<int64_t>((int64_t)P->h_arena.size(), 2)))
    return PERM_ENOMEM;
  JobArrays cur = jb[0].view();
  uint64_t* cur_arena = reinterpret_cast<uint64_t*>(ar[0].p);
  if (nroots > 0) {
    std::vector<uint64_t> coef(4 * nroots, 0ull);
    for (int64_t r = 0; r < nroots; ++r) coef[4 * r] = 1;
    CK(cudaMemcpyAsync(cur_arena, P->h_arena.data(), 8 * P->h_arena.size(), cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(cur.m, rm.data(), 4 * nroots, cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(cur.nnz, rnnz.data(), 4 * nroots, cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(cur.off, roff.data(), 8 * nroots, cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(cur.mat, rmat.data(), 4 * nroots, cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(cur.depth_left, rdl.data(), 4 * nroots, cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(cur.coef, coef.data(), 32 * nroots, cudaMemcpyHostToDevice, s));
  }
  // stat[0]: first error status (int32 in the low half), [1]: largest kept
  // order, [2]: words of the kept blocks, [3]: kept jobs, [4]: largest
  // order of a kept job still to split
  long long* d_stat = dget<long long>(M, 5);
  if (!d_stat) return PERM_ENOMEM;
  CK(cudaMemsetAsync(d_stat, 0, 40, s));
  int max_order = maxn;
  int64_t cur_arena_words = (int64_t)P->h_arena.size();  // roots sit back to back
  int64_t used_words = cur_arena_words;                    // words of the current jobs' blocks
  auto split_floor = [&](int mopen) { return adaptive ? mopen - kSplitBand : 0; };
  // child slots per parent: Eq. 2's third child needs a third slot
  const int K = P->opts.dense_split ? 3 : 2;
  int level0 = 0;
  bool used_fused = false;
  if (P->opts.fused_levels && levels_left(0, ncur, max_open)) {
    used_fused = true;
    // consecutive levels in one cooperative launch; buffers start small and
    // grow by 4x (the current level copied over) when the frontier outgrows
    // them, up to kFusedMaxJobs / kFusedMaxWords
    int64_t cap_jobs = std::max<int64_t>(kFusedJobs0, K * ncur);
    int64_t cap_words = std::max<int64_t>(kFusedWords0, K * used_words);
    ExpandFrontState* d_state = dget<ExpandFrontState>(M, 1);
    long long* d_partial = dget<long long>(M, PERM_FRONT_MAX_BLOCKS);
    unsigned long long* d_bar = dget<unsigned long long>(M, 1);
    unsigned long long* d_lw = dget<unsigned long long>(M, maxd);
    int32_t* d_lm = dget<int32_t>(M, maxd);
    int32_t* d_lo = dget<int32_t>(M, maxd);
    if (!d_state || !d_partial || !d_bar || !d_lw || !d_lm || !d_lo) return PERM_ENOMEM;
    CK(cudaMemsetAsync(d_lo, 0, 4 * (size_t)maxd, s));
    CK(cudaMemsetAsync(d_lw, 0, 8 * (size_t)maxd, s));
    CK(cudaMemsetAsync(d_lm, 0, 4 * (size_t)maxd, s));
    ExpandFrontState S;
    S.ncur = ncur;
    S.used_words = used_words;
    S.level = 0;
    S.max_order = max_order;
    S.max_open = max_open;
    S.cb = 0;
    for (;;) {
      const int ob = S.cb ^ 1;
      if (!jb[ob].ensure(M, cap_jobs) || !grow(M, ar[ob], 8 * (size_t)cap_words) || !slots.ensure(M, cap_jobs) ||
          !grow(M, g_valid, 4 * (size_t)cap_jobs))
        return PERM_ENOMEM;
      if (jb[S.cb].m.cap < 4 * (size_t)cap_jobs || ar[S.cb].cap < 8 * (size_t)cap_words) {
        // move the current level into the other (large) buffers
        const JobArrays src = jb[S.cb].view(), dst = jb[ob].view();
        CK(cudaMemcpyAsync(dst.m, src.m, 4 * S.ncur, cudaMemcpyDeviceToDevice, s));
        CK(cudaMemcpyAsync(dst.nnz, src.nnz, 4 * S.ncur, cudaMemcpyDeviceToDevice, s));
        CK(cudaMemcpyAsync(dst.off, src.off, 8 * S.ncur, cudaMemcpyDeviceToDevice, s));
        CK(cudaMemcpyAsync(dst.mat, src.mat, 4 * S.ncur, cudaMemcpyDeviceToDevice, s));
        CK(cudaMemcpyAsync(dst.depth_left, src.depth_left, 4 * S.ncur, cudaMemcpyDeviceToDevice, s));
        CK(cudaMemcpyAsync(dst.coef, src.coef, 32 * S.ncur, cudaMemcpyDeviceToDevice, s));
        CK(cudaMemcpyAsync(ar[ob].p, ar[S.cb].p, 8 * (size_t)S.used_words, cudaMemcpyDeviceToDevice, s));
        S.cb = ob;
        if (!jb[S.cb ^ 1].ensure(M, cap_jobs) || !grow(M, ar[S.cb ^ 1], 8 * (size_t)cap_words))
          return PERM_ENOMEM;
      }
      ExpandFrontArgs F;
      for (int k = 0; k < 2; ++k) {
        F.buf[k] = jb[k].view();
        F.arena[k] = reinterpret_cast<uint64_t*>(ar[k].p);
      }
      F.cap_jobs = cap_jobs;
      F.cap_words = cap_words;
      F.mod = P->mod.p;
      F.slots = slots.view();
      F.valid = reinterpret_cast<int32_t*>(g_valid.p);
      F.kslots = K;
      F.leaf_size = P->L;
      F.max_levels = maxd;
      F.adaptive = adaptive ? 1 : 0;
      F.big_order = PERM_MAX_JOB_N;
      F.band = kSplitBand;
      F.soft_order = kSoftOrder;
      F.soft_cap_jobs = kSoftCapJobs;
      F.target_jobs = target;
      F.state = d_state;
      F.partial = d_partial;
      F.bar = d_bar;
      F.lvl_words = d_lw;
      F.lvl_maxo = d_lm;
      F.lvl_maxopen = d_lo;
      F.err = reinterpret_cast<int32_t*>(d_stat);
      CK(cudaMemcpyAsync(d_state, &S, sizeof(S), cudaMemcpyHostToDevice, s));
      CK(cudaMemsetAsync(d_bar, 0, 8, s));
      int grid = 0;
      CK(launch_expand_front(F, S.max_order, &grid, s));
      if (grid == 0) break;  // no cooperative launch on this device
      long long st0 = 0;
      CK(cudaMemcpyAsync(&S, d_state, sizeof(S), cudaMemcpyDeviceToHost, s));
      CK(cudaMemcpyAsync(&st0, d_stat, 8, cudaMemcpyDeviceToHost, s));
      CK(cudaStreamSynchronize(s));
      const int32_t herr = (int32_t)(st0 & 0xffffffff);
      if (herr != 0) return (perm_status)herr;
      if (!levels_left(S.level, S.ncur, S.max_open)) break;
      const bool room = K * S.ncur > cap_jobs || K * S.used_words > cap_words;
      if (!room) continue;  // the orders now fit a narrower variant: launch it
      // stopped for room: grow, or hand over to the per-level loop
      if (cap_jobs >= kFusedMaxJobs || cap_words >= kFusedMaxWords) break;
      if (K * S.ncur > cap_jobs) cap_jobs = std::min<int64_t>(kFusedMaxJobs, 4 * cap_jobs);
      if (K * S.used_words > cap_words) cap_words = std::min<int64_t>(kFusedMaxWords, 4 * cap_words);
      if (K * S.ncur > cap_jobs || K * S.used_words > cap_words) break;
    }
    M.put(d_state);
    M.put(d_partial);
    M.put(d_bar);
    M.put(d_lw);
    M.put(d_lm);
    M.put(d_lo);
    cb = S.cb;
    cur = jb[cb].view();
    cur_arena = reinterpret_cast<uint64_t*>(ar[cb].p);
    ncur = S.ncur;
    max_order = S.max_order;
    max_open = S.max_open;
    used_words = S.used_words;
    cur_arena_words = S.used_words;
    level0 = S.level;
  }
  for (int level = level0; levels_left(level, ncur, max_open); ++level) {
    // every parent reserves K child slots of its own block size
    const int64_t out_words = K * used_words;
    const int nb = cb ^ 1;
    const size_t tb = std::max(scan_tmp_bytes_i64(ncur), scan_tmp_bytes_i32(K * ncur));
    if (!grow(M, g_words, 8 * (size_t)ncur) || !grow(M, g_base, 8 * (size_t)ncur) ||
        !grow(M, g_valid, 4 * (size_t)(K * ncur)) || !grow(M, g_pos, 4 * (size_t)(K * ncur)) || !grow(M, g_tmp, tb) ||
        !grow(M, ar[nb], 8 * (size_t)std::max<int64_t>(out_words, 2)) || !slots.ensure(M, K * ncur))
      return PERM_ENOMEM;
    int64_t* words = reinterpret_cast<int64_t*>(g_words.p);
    int64_t* base = reinterpret_cast<int64_t*>(g_base.p);
    int32_t* valid = reinterpret_cast<int32_t*>(g_valid.p);
    int32_t* pos = reinterpret_cast<int32_t*>(g_pos.p);
    uint64_t* next_arena = reinterpret_cast<uint64_t*>(ar[nb].p);
    CK(launch_child_capacity(cur, ncur, K, words, s));
    CK(scan_exclusive_i64(words, base, ncur, g_tmp.p, g_tmp.cap, s));
    ExpandLevelArgs A;
    A.parent = cur;
    A.arena_in = cur_arena;
    A.np = ncur;
    A.child = slots.view();
    A.arena_out = next_arena;
    A.child_off_base = base;
    A.valid = valid;
    A.kslots = K;
    A.leaf_size = P->L;
    A.split_floor = split_floor(max_open);
    A.mod = P->mod.p;
    A.err = reinterpret_cast<int32_t*>(d_stat);
    CK(launch_expand_level(A, max_order, s));
    CK(scan_exclusive_i32(valid, pos, K * ncur, g_tmp.p, g_tmp.cap, s));
    // the kept children: at most K * ncur; size the next arrays for that bound
    if (!jb[nb].ensure(M, K * ncur)) return PERM_ENOMEM;
    CK(cudaMemsetAsync(d_stat + 1, 0, 32, s));
    CK(launch_compact_jobs(slots.view(), valid, pos, K * ncur, jb[nb].view(), std::max(P->L, 2), d_stat + 1, s));
    long long st[5] = {0, 0, 0, 0, 0};
    CK(cudaMemcpyAsync(st, d_stat, 40, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    const int32_t herr = (int32_t)(st[0] & 0xffffffff);
    if (herr != 0) return (perm_status)herr;
    cb = nb;
    cur = jb[cb].view();
    cur_arena = next_arena;
    cur_arena_words = out_words;
    ncur = st[3];
    max_order = (int)st[1];  // carried jobs keep their order
    used_words = st[2];
    max_open = (int)st[4];
  }
  M.put(d_stat);
  P->expand_driver = used_fused ? 1 : 0;
  // the current buffers become the job set; the rest is released
  J->n = ncur;
  J->a = jb[cb].view();
  J->arena = cur_arena;
  J->arena_words = cur_arena_words;
  jb[cb].release_ownership();
  ar[cb].p = nullptr;
  jb[cb ^ 1].free(M);
  M.put(ar[cb ^ 1].p);
  slots.free(M);
  M.put(g_words.p);
  M.put(g_base.p);
  M.put(g_valid.p);
  M.put(g_pos.p);
  M.put(g_tmp.p);
  return finish_jobset(P, J, jobs_out, njobs);
}

// The job set's host copy of the job orders, and its output arrays.
static perm_status finish_jobset(perm_plan* P, perm_jobs* J, perm_jobs_t** jobs_out, int64_t* njobs) {
  Mem& M = P->M;
  cudaStream_t s = P->s;
  const int64_t ncur = J->n;
  const JobArrays cur = J->a;
  CK(cudaEventRecord(P->xe1, s));
  J->h_m.resize(ncur);
  if (ncur > 0) CK(cudaMemcpyAsync(J->h_m.data(), cur.m, 4 * ncur, cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  CK(cudaEventElapsedTime(&P->last_expand_ms, P->xe0, P->xe1));
  J->max_order = 0;
  J->order_count.assign(PERM_MAX_N + 1, 0);
  for (int32_t v : J->h_m) {
    J->max_order = std::max(J->max_order, (int)v);
    J->order_count[std::min(std::max(v, 0), PERM_MAX_N)] += 1;
  }
  // outputs
  const int64_t nj = std::max<int64_t>(ncur, 1);
  J->out.acc = dget<unsigned long long>(M, 4 * nj);
  J->out.t_start = dget<unsigned long long>(M, nj);
  J->out.t_end = dget<unsigned long long>(M, nj);
  J->out.sm = dget<int32_t>(M, nj);
  J->out.status = dget<int32_t>(M, nj);
  J->out.leaves = dget<unsigned long long>(M, nj);
  J->out.nodes = dget<unsigned long long>(M, nj);
  J->d_queue = dget<uint32_t>(M, nj);
  J->d_logap = dget<float>(M, nj);
  if (!J->out.acc || !J->out.t_start || !J->out.t_end || !J->out.sm || !J->out.status || !J->out.leaves ||
      !J->out.nodes || !J->d_queue || !J->d_logap)
    return PERM_ENOMEM;
  if (jobs_out) *jobs_out = J;
  if (njobs) *njobs = ncur;
  return PERM_OK;
}
extern "C" perm_status perm_expand(perm_plan_t* P, perm_jobs_t** jobs_out, int64_t* njobs) {
  return guarded([&] { return perm_expand_impl(P, jobs_out, njobs); });
}

static perm_status perm_last_expand_ms_impl(perm_plan_t* P, float* ms) {
  if (!P || !ms) return PERM_EINVAL;
  if (P->expand_driver < 0) return PERM_ESTATE;
  *ms = P->last_expand_ms;
  return PERM_OK;
}
extern "C" perm_status perm_last_expand_ms(perm_plan_t* P, float* ms) {
  return guarded([&] { return perm_last_expand_ms_impl(P, ms); });
}

static perm_status perm_expand_driver_impl(perm_plan_t* P, int32_t* driver) {
  if (!P || !driver) return PERM_EINVAL;
  if (P->expand_driver < 0) return PERM_ESTATE;
  *driver = P->expand_driver;
  return PERM_OK;
}
extern "C" perm_status perm_expand_driver(perm_plan_t* P, int32_t* driver) {
  return guarded([&] { return perm_expand_driver_impl(P, driver); });
}

// ---------------------------------------------------------------- a4: estimate
static perm_status perm_estimate_impl(perm_jobs_t* J, float* log_ap) {
  if (!J) return PERM_EINVAL;
  perm_plan* P = J->plan;
  if (J->max_order > PERM_MAX_N) return PERM_EINVAL;
  void* scratch = P->M.get(kklll_scratch_bytes(J->n, J->max_order, P->opts.kklll_trials));
  if (!scratch) return PERM_ENOMEM;
  CK(launch_kklll(J->a, J->n, J->arena, P->opts.kklll_trials, P->opts.seed, J->d_logap, J->max_order, scratch,
                  P->s));
  P->M.put(scratch);
  J->has_logap = true;
  if (log_ap && J->n > 0) {
    CK(cudaMemcpyAsync(log_ap, J->d_logap, 4 * J->n, cudaMemcpyDeviceToHost, P->s));
    CK(cudaStreamSynchronize(P->s));
  }
  return PERM_OK;
}
extern "C" perm_status perm_estimate(perm_jobs_t* J, float* log_ap) {
  return guarded([&] { return perm_estimate_impl(J, log_ap); });
}

static perm_status perm_job_features_impl(perm_jobs_t* J, float* feats) {
  if (!J || !feats) return PERM_EINVAL;
  perm_plan* P = J->plan;
  const bool use_ap = P->opts.model_uses_estimate != 0;
  if (use_ap && !J->has_logap) {
    perm_status st = perm_estimate(J, nullptr);
    if (st != PERM_OK) return st;
  }
  float* d = dget<float>(P->M, J->n * PERM_MLP_FEATURES);
  if (!d) return PERM_ENOMEM;
  CK(launch_features(J->a, J->n, J->arena, use_ap ? J->d_logap : nullptr, d, P->s));
  CK(cudaMemcpyAsync(feats, d, sizeof(float) * J->n * PERM_MLP_FEATURES, cudaMemcpyDeviceToHost, P->s));
  CK(cudaStreamSynchronize(P->s));
  P->M.put(d);
  return PERM_OK;
}
extern "C" perm_status perm_job_features(perm_jobs_t* J, float* feats) {
  return guarded([&] { return perm_job_features_impl(J, feats); });
}

// ---------------------------------------------------------------- a5, a6: order
static perm_status sort_queue_by(perm_plan* P, perm_jobs* J, const float* d_keys) {
  Mem& M = P->M;
  const int64_t n = J->n;
  std::vector<uint32_t> iota(n);
  std::iota(iota.begin(), iota.end(), 0u);
  uint32_t* vin = dget<uint32_t>(M, n);
  float* kout = dget<float>(M, n);
  size_t tb = sort_tmp_bytes_f32(n);
  void* tmp = M.get(tb);
  if (!vin || !kout || !tmp) return PERM_ENOMEM;
  CK(cudaMemcpyAsync(vin, iota.data(), 4 * n, cudaMemcpyHostToDevice, P->s));
  CK(sort_desc_f32(d_keys, kout, vin, J->d_queue, n, tmp, tb, P->s));
  CK(cudaStreamSynchronize(P->s));
  M.put(vin);
  M.put(kout);
  M.put(tmp);
  return PERM_OK;
}

static perm_status perm_order_impl(perm_jobs_t* J, int32_t kind, uint32_t* order_out) {
  if (!J) return PERM_EINVAL;
  perm_plan* P = J->plan;
  const int64_t n = J->n;
  if (n == 0) {
    J->has_order = true;
    return PERM_OK;
  }
  if (kind == PERM_ORDER_NATURAL) {
    CK(launch_iota_u32(J->d_queue, n, P->s));
  } else if (kind == PERM_ORDER_LPT || (kind == PERM_ORDER_LEARNED && P->mlp.empty())) {
    if (!J->has_logap) {
      perm_status st = perm_estimate(J, nullptr);
      if (st != PERM_OK) return st;
    }
    perm_status st = sort_queue_by(P, J, J->d_logap);
    if (st != PERM_OK) return st;
  } else if (kind == PERM_ORDER_LEARNED) {
    const bool use_ap = P->opts.model_uses_estimate != 0;
    if (use_ap && !J->has_logap) {
      perm_status st = perm_estimate(J, nullptr);
      if (st != PERM_OK) return st;
    }
    float* feats = dget<float>(P->M, n * PERM_MLP_FEATURES);
    float* params = dget<float>(P->M, PERM_MLP_PARAMS);
    float* pred = dget<float>(P->M, n);
    if (!feats || !params || !pred) return PERM_ENOMEM;
    CK(cudaMemcpyAsync(params, P->mlp.data(), 4 * PERM_MLP_PARAMS, cudaMemcpyHostToDevice, P->s));
    CK(launch_features(J->a, n, J->arena, use_ap ? J->d_logap : nullptr, feats, P->s));
    CK(mlp_predict(params, feats, (int32_t)n, pred, P->s));
    perm_status st = sort_queue_by(P, J, pred);
    P->M.put(feats);
    P->M.put(params);
    P->M.put(pred);
    if (st != PERM_OK) return st;
  } else {
    return PERM_EINVAL;
  }
  J->has_order = true;
  if (order_out) {
    CK(cudaMemcpyAsync(order_out, J->d_queue, 4 * n, cudaMemcpyDeviceToHost, P->s));
    CK(cudaStreamSynchronize(P->s));
  }
  return PERM_OK;
}
extern "C" perm_status perm_order(perm_jobs_t* J, int32_t kind, uint32_t* order_out) {
  return guarded([&] { return perm_order_impl(J, kind, order_out); });
}

// ---------------------------------------------------------------- a7, a8: evaluate
// prepare: split the queue, classify leaf variants, upload, size buffers.
// resident depth-first warps per SM for a tile width
static int dfs_wps(const perm_plan* P, int tile) {
  if (P->opts.workers_per_sm > 0) return P->opts.workers_per_sm;
  return tile <= 32 ? 24 : 10;
}

// order: the queue (nq distinct job indices), or NULL for the order set by
// perm_order (every job).  Jobs outside the queue are not evaluated: their
// records stay zero and they add nothing to the sums.
static perm_status eval_prepare(perm_jobs* J, const uint32_t* order, int64_t nq_in) {
  perm_plan* P = J->plan;
  cudaStream_t s = P->s;
  Mem& M = P->M;
  const int64_t nj = J->n;
  const int leaf_max = std::max(P->L, 2);
  if (J->max_order > leaf_max && J->max_order > PERM_MAX_JOB_N) return PERM_EINVAL;
  if (order && (nq_in < 0 || nq_in > nj)) return PERM_EINVAL;
  const int64_t n = order ? nq_in : nj;  // queue length
  free_eval(M, J);
  J->ev = new EvalState();
  EvalState& E = *J->ev;
  E.nq = n;
  E.d_q = dget<uint32_t>(M, n);
  E.sum = dget<unsigned long long>(M, SUM_WORDS);
  E.ctr = dget<unsigned long long>(M, 1 + EVAL_DFS_GROUPS);
  if (!E.d_q || !E.sum || !E.ctr) return PERM_ENOMEM;
  if (order) {
    std::vector<uint8_t> seen(nj, 0);
    for (int64_t k = 0; k < n; ++k) {
      if (order[k] >= (uint64_t)nj || seen[order[k]]) return PERM_EINVAL;
      seen[order[k]] = 1;
    }
    if (n) CK(cudaMemcpyAsync(E.d_q, order, 4 * n, cudaMemcpyHostToDevice, s));
  } else {
    if (!J->has_order) {
      perm_status st = perm_order(J, P->opts.order, nullptr);
      if (st != PERM_OK) return st;
    }
    if (n) CK(cudaMemcpyAsync(E.d_q, J->d_queue, 4 * n, cudaMemcpyDeviceToDevice, s));
  }
  // group the queue on the device: leaf jobs by kernel variant, then the
  // depth-first jobs by ring width, queue order kept inside every group
  unsigned long long* hist = E.sum + SUM_HIST;
  CK(cudaMemsetAsync(hist, 0, 8 * EVAL_KEYS, s));
  E.d_g = dget<uint32_t>(M, n);
  uint32_t* keys = dget<uint32_t>(M, 2 * n);
  uint32_t* vals = dget<uint32_t>(M, n);
  const size_t sort_b = sort_tmp_bytes_u32(std::max<int64_t>(n, 1), 7);
  void* sort_tmp = M.get(sort_b);
  if (!E.d_g || !keys || !vals || !sort_tmp) return PERM_ENOMEM;
  std::vector<unsigned long long> h(EVAL_KEYS, 0ull);
  if (n) {
    CK(launch_eval_keys(E.d_q, n, J->a, J->arena, P->d_mat_w, leaf_max, P->mod.p != 0, keys, vals, hist, s));
    CK(sort_asc_u32(keys, keys + n, vals, E.d_g, n, 7, sort_tmp, sort_b, s));
    CK(cudaMemcpyAsync(h.data(), hist, 8 * EVAL_KEYS, cudaMemcpyDeviceToHost, s));
  }
  E.single = P->opts.single_launch != 0;
  if (E.single)
    E.keys = keys;  // keys[0, n) stay in queue order (the sort wrote its output after them)
  else
    M.put(keys);
  M.put(vals);
  M.put(sort_tmp);
  CK(cudaStreamSynchronize(s));
  int64_t nl = 0;
  for (int k = 0; k < EVAL_KEY_DFS; ++k) {
    if (h[k] == 0) continue;
    E.groups.push_back({nl, (int64_t)h[k]});
    E.group_cls.push_back(k);
    nl += (int64_t)h[k];
  }
  E.nl = nl;
  E.db[0] = 0;
  for (int g = 0; g < EVAL_DFS_GROUPS; ++g) E.db[g + 1] = E.db[g] + (int64_t)h[EVAL_KEY_DFS + g];
  E.nd = E.db[EVAL_DFS_GROUPS];
  E.d_lq = E.d_g;
  E.d_dq = E.d_g + nl;
  const int64_t nd = E.nd;
  E.counts = dget<uint64_t>(M, nl + 1);
  E.prefix = dget<uint64_t>(M, nl + 1);
  E.stb = std::max(scan_tmp_bytes_u64(nl + 1), scan_tmp_bytes_i32(nd + 1));
  E.stmp = M.get(E.stb);
  E.d_rq = dget<uint32_t>(M, nd);
  E.rflags = dget<int32_t>(M, nd + 1);
  E.rpos = dget<int32_t>(M, nd + 1);
  // the narrow variant (int32 tile, leaves <= 16 rows) unless the leaf order needs the wide one
  E.wide_first = P->L > 16;
  E.chunk = P->opts.chunk_log2 > 0 ? P->opts.chunk_log2 : 10;
  uint64_t leaf_tasks = 0;
  if (order && n < nj) {  // a sub-queue: its own jobs
    for (int64_t k = 0; k < n; ++k)
      if (J->h_m[order[k]] <= leaf_max) leaf_tasks += leaf_tasks_host(J->h_m[order[k]], E.chunk);
  } else {  // every job (any order): from the count of jobs per order
    for (int m = 0; m <= std::min(leaf_max, PERM_MAX_N); ++m)
      if (J->order_count[m]) leaf_tasks += (uint64_t)J->order_count[m] * leaf_tasks_host(m, E.chunk);
  }
  E.owner = dget<uint32_t>(M, (int64_t)std::max<uint64_t>(leaf_tasks, 1));
  int dfs_warps = 0, max_tile = 32;
  for (int g = 0; g < EVAL_DFS_GROUPS; ++g) {
    if (E.db[g + 1] == E.db[g]) continue;
    const int tile = dfs_group_tile(g);
    max_tile = std::max(max_tile, tile);
    for (bool w : {false, true}) {
      const int wpb = dfs_warps_per_block(tile, w);
      dfs_warps = std::max(dfs_warps, P->sms * ((dfs_wps(P, tile) + wpb - 1) / wpb) * wpb);
    }
  }
  // Eq. 2's third child keeps the order, so a path can hold more levels than rows
  E.frames = P->opts.dense_split ? 4 * max_tile : max_tile;
  E.undo_w = dfs_undo_words(max_tile, E.frames);
  int64_t undo_words = E.undo_w * dfs_warps;
  if (E.single) {
    // ring of the persistent kernel: the widest matrix's (residues: 0)
    E.single_w = 2;
    for (int i = 0; i < P->count; ++i) E.single_w = std::max(E.single_w, (int)P->w[i]);
    if (P->mod.p) E.single_w = 0;
    int64_t pw = 0;
    CK(persist_warps(E.single_w, !E.wide_first, P->sms, &pw));
    // the persistent kernel's depth-first part: 32-wide tiles
    undo_words = std::max(undo_words, dfs_undo_words(32, E.frames) * pw);
    E.pctr = dget<unsigned long long>(M, 2);
    E.task_ctr = dget<uint32_t>(M, 2 * std::max<int64_t>(n, 1));
    if (!E.pctr || !E.task_ctr) return PERM_ENOMEM;
  }
  E.undo = (nd > 0 || E.single) ? dget<int64_t>(M, undo_words) : nullptr;
  if (!E.counts || !E.prefix || !E.owner || !E.stmp || !E.d_rq || !E.rflags || !E.rpos ||
      ((nd > 0 || E.single) && !E.undo))
    return PERM_ENOMEM;
  return PERM_OK;
}

// arguments of depth-first group g over queue[0, nq)
static DfsArgs dfs_args(perm_jobs* J, int g, const uint32_t* queue, int64_t nq) {
  perm_plan* P = J->plan;
  EvalState& E = *J->ev;
  DfsArgs D{};
  D.queue = queue;
  D.nq = nq;
  D.jobs = J->a;
  D.arena = J->arena;
  D.mat_w = P->d_mat_w;
  D.leaf_size = P->L;
  D.job_counter = E.ctr + 1 + g;
  D.out = J->out;
  D.mat_acc = P->d_mat_acc;
  D.undo = E.undo;
  D.undo_words_per_warp = E.undo_w;
  D.timeout_ns = P->opts.timeout_ns > 0 ? P->opts.timeout_ns : 10000000000ll;
  D.three = P->opts.dense_split ? 1 : 0;
  D.max_depth = E.frames;
  D.mod = P->mod;
  return D;
}

// enqueue: memsets and launches only (no host synchronisation), on stream s.
static cudaError_t eval_enqueue(perm_jobs* J, cudaStream_t s) {
  perm_plan* P = J->plan;
  EvalState& E = *J->ev;
  const int64_t nj = std::max<int64_t>(J->n, 1);
  cudaError_t e;
  int launches = 0;
#define EQ(call)                          \
  do {                                    \
    if ((e = (call)) != cudaSuccess) return e; \
  } while (0)
  EQ(cudaMemsetAsync(J->out.acc, 0, 32 * nj, s));
  EQ(cudaMemsetAsync(J->out.t_start, 0xff, 8 * nj, s));
  EQ(cudaMemsetAsync(J->out.t_end, 0, 8 * nj, s));
  EQ(cudaMemsetAsync(J->out.status, 0, 4 * nj, s));
  EQ(cudaMemsetAsync(J->out.sm, 0xff, 4 * nj, s));
  EQ(cudaMemsetAsync(J->out.leaves, 0, 8 * nj, s));
  EQ(cudaMemsetAsync(J->out.nodes, 0, 8 * nj, s));
  EQ(cudaMemsetAsync(P->d_mat_acc, 0, 32ull * P->count, s));
  EQ(cudaMemsetAsync(E.ctr, 0, 8 * (1 + EVAL_DFS_GROUPS), s));
  EQ(cudaMemsetAsync(E.sum + SUM_STATUS, 0xff, 8, s));
  if (E.single) {
    // depth-first jobs of order > 32 first (tile 64), then everything else in one
    // launch; a job the narrow tile hands on only raises a flag here (the
    // wide rerun happens after, when the flag is set)
    EQ(cudaMemsetAsync(E.sum + SUM_RFLAG, 0, 8, s));
    for (int g = 0; g < EVAL_DFS_GROUPS; ++g) {
      const int64_t nq = E.db[g + 1] - E.db[g];
      if (nq == 0 || dfs_group_tile(g) != 64) continue;
      DfsArgs d = dfs_args(J, g, E.d_dq + E.db[g], nq);
      d.retry_flag = E.sum + SUM_RFLAG;
      EQ(launch_dfs(d, 64, E.wide_first, dfs_group_w(g), P->sms, dfs_wps(P, 64), s));
      ++launches;
    }
    EQ(cudaMemsetAsync(E.pctr, 0, 8, s));
    EQ(cudaMemsetAsync(E.pctr + 1, 0xff, 8, s));
    EQ(cudaMemsetAsync(E.task_ctr, 0, 8 * (size_t)std::max<int64_t>(E.nq, 1), s));
    PersistArgs A{};
    A.queue = E.d_q;
    A.keys = E.keys;
    A.nq = E.nq;
    A.chunk_log2 = E.chunk;
    A.qctr = E.pctr;
    A.board = reinterpret_cast<long long*>(E.pctr + 1);
    A.task_next = E.task_ctr;
    A.task_done = E.task_ctr + std::max<int64_t>(E.nq, 1);
    A.dfs = dfs_args(J, 2, nullptr, 0);
    A.dfs.undo_words_per_warp = dfs_undo_words(32, E.frames);
    A.dfs.retry_flag = E.sum + SUM_RFLAG;
    if (E.nq > 0) {
      EQ(launch_persist(A, E.single_w, !E.wide_first, P->sms, s));
      ++launches;
    }
    if (J->n > 0) {
      EQ(launch_status_summary(J->out.status, J->n, E.sum + SUM_STATUS, s));
      ++launches;
    }
    P->last_launches = launches;
    return cudaSuccess;
  }
  // depth-first groups: tile 64 (the largest jobs) first; each its own job counter
  for (int g = 0; g < EVAL_DFS_GROUPS; ++g) {
    const int64_t nq = E.db[g + 1] - E.db[g];
    if (nq == 0) continue;
    const int tile = dfs_group_tile(g);
    EQ(launch_dfs(dfs_args(J, g, E.d_dq + E.db[g], nq), tile, E.wide_first, dfs_group_w(g), P->sms,
                  dfs_wps(P, tile), s));
    ++launches;
  }
  if (E.nl > 0) {
    // one task scan for the grouped leaf queue, then one persistent grid per
    // kernel variant over its slice
    EQ(launch_leaf_tasks(E.d_lq, E.nl, J->a, E.chunk, E.counts, E.prefix, E.owner, E.stmp, E.stb, s));
    launches += 4;
    for (size_t g = 0; g < E.groups.size(); ++g) {
      const int64_t o = E.groups[g].first;
      EQ(launch_leaf_batch(E.d_lq + o, E.groups[g].second, E.group_cls[g], E.prefix + o, E.owner, o, J->a,
                           J->arena, E.chunk,
                           E.ctr, J->out, P->mod, P->sms, s));
      ++launches;
    }
    EQ(launch_leaf_finalize(E.d_lq, E.nl, J->a, J->out, P->d_mat_acc, P->mod.p, s));
    ++launches;
  }
  if (E.nd > 0 && !E.wide_first) {
    // jobs the narrow depth-first variant handed on, for the wide one
    RetryBounds rb;
    for (int g = 0; g <= EVAL_DFS_GROUPS; ++g) rb.b[g] = E.db[g];
    EQ(launch_retry_collect(E.d_dq, E.nd, rb, J->out.status, E.rflags, E.rpos, E.stmp, E.stb, E.d_rq,
                            E.sum + SUM_RETRY, s));
    launches += 4;
  }
  if (J->n > 0) {
    EQ(launch_status_summary(J->out.status, J->n, E.sum + SUM_STATUS, s));
    ++launches;
  }
#undef EQ
  P->last_launches = launches;
  return cudaSuccess;
}

// finish: wait, re-run jobs the narrow depth-first variant handed on, and
// read the status summary and (optionally) the per-job records.
static perm_status eval_finish(perm_jobs* J, perm_job_result* results) {
  perm_plan* P = J->plan;
  EvalState& E = *J->ev;
  cudaStream_t s = P->s;
  const int64_t n = J->n;
  CK(cudaEventSynchronize(P->ev1));
  CK(cudaEventElapsedTime(&P->last_ms, P->ev0, P->ev1));
  unsigned long long sum[SUM_HIST];
  for (int k = 0; k < SUM_HIST; ++k) sum[k] = k == SUM_STATUS ? ~0ull : 0ull;
  if (n) CK(cudaMemcpyAsync(sum, E.sum, sizeof(sum), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  if (E.single) {
    // single-launch mode collects the jobs handed on only when one was
    for (int k = 0; k <= EVAL_DFS_GROUPS; ++k) sum[SUM_RETRY + k] = 0;
    unsigned long long flag = 0;
    if (n && E.nd > 0 && !E.wide_first) {
      CK(cudaMemcpyAsync(&flag, E.sum + SUM_RFLAG, 8, cudaMemcpyDeviceToHost, s));
      CK(cudaStreamSynchronize(s));
    }
    if (flag) {
      RetryBounds rb;
      for (int g = 0; g <= EVAL_DFS_GROUPS; ++g) rb.b[g] = E.db[g];
      CK(launch_retry_collect(E.d_dq, E.nd, rb, J->out.status, E.rflags, E.rpos, E.stmp, E.stb, E.d_rq,
                              E.sum + SUM_RETRY, s));
      CK(cudaMemcpyAsync(sum + SUM_RETRY, E.sum + SUM_RETRY, 8 * (EVAL_DFS_GROUPS + 1), cudaMemcpyDeviceToHost, s));
      CK(cudaStreamSynchronize(s));
    }
  }
  const unsigned long long* at = sum + SUM_RETRY;
  if (n && E.nd > 0 && !E.wide_first && at[EVAL_DFS_GROUPS] > 0) {
    // jobs the narrow variant handed on run again on the wide one, by group
    CK(cudaMemsetAsync(E.ctr, 0, 8 * (1 + EVAL_DFS_GROUPS), s));
    float ms2 = 0.f;
    CK(cudaEventRecord(P->ev0, s));
    for (int g = 0; g < EVAL_DFS_GROUPS; ++g) {
      const int64_t nr = (int64_t)(at[g + 1] - at[g]);
      if (nr == 0) continue;
      const int tile = dfs_group_tile(g);
      CK(launch_dfs(dfs_args(J, g, E.d_rq + at[g], nr), tile, true, dfs_group_w(g), P->sms, dfs_wps(P, tile), s));
      P->last_launches += 1;
    }
    CK(cudaEventRecord(P->ev1, s));
    CK(cudaMemsetAsync(E.sum + SUM_STATUS, 0xff, 8, s));
    CK(launch_status_summary(J->out.status, n, E.sum + SUM_STATUS, s));
    CK(cudaMemcpyAsync(sum + SUM_STATUS, E.sum + SUM_STATUS, 8, cudaMemcpyDeviceToHost, s));
    CK(cudaEventSynchronize(P->ev1));
    CK(cudaEventElapsedTime(&ms2, P->ev0, P->ev1));
    CK(cudaStreamSynchronize(s));
    P->last_ms += ms2;
    P->last_launches += 1;
  }
  if (results && n) {
    std::vector<unsigned long long> acc(4 * n), t0(n), t1(n), lv(n), nd_(n);
    std::vector<int32_t> sm(n), mat(n), nnz(n), st(n);
    std::vector<uint32_t> q(n);
    CK(cudaMemcpyAsync(acc.data(), J->out.acc, 32 * n, cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(t0.data(), J->out.t_start, 8 * n, cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(t1.data(), J->out.t_end, 8 * n, cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(lv.data(), J->out.leaves, 8 * n, cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(nd_.data(), J->out.nodes, 8 * n, cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(sm.data(), J->out.sm, 4 * n, cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(st.data(), J->out.status, 4 * n, cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(mat.data(), J->a.mat, 4 * n, cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(nnz.data(), J->a.nnz, 4 * n, cudaMemcpyDeviceToHost, s));
    if (E.nq) CK(cudaMemcpyAsync(q.data(), E.d_q, 4 * E.nq, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    std::vector<int32_t> qpos(n, -1);
    for (int64_t k = 0; k < E.nq; ++k) qpos[q[k]] = (int32_t)k;
    for (int64_t j = 0; j < n; ++j) {
      perm_job_result& r = results[j];
      r.matrix = mat[j];
      r.order = J->h_m[j];
      r.nnz = nnz[j];
      r.status = st[j];
      for (int w = 0; w < 4; ++w) r.value[w] = acc[4 * j + w];
      r.t_start_ns = (int64_t)t0[j];
      r.t_end_ns = (int64_t)t1[j];
      r.sm = sm[j];
      r.queue_pos = qpos[j];
      r.leaves = (int64_t)lv[j];
      r.nodes = (int64_t)nd_[j];
    }
  }
  // the lowest job index with a failed status decides the call's status
  if (sum[SUM_STATUS] != ~0ull) return (perm_status)(sum[SUM_STATUS] & 255);
  P->evaluated = true;
  return PERM_OK;
}

static perm_status eval_run(perm_jobs_t* J, const uint32_t* order, int64_t count, perm_job_result* results) {
  if (!J) return PERM_EINVAL;
  perm_plan* P = J->plan;
  perm_status st = eval_prepare(J, order, count);
  if (st != PERM_OK) return st;
  CK(cudaEventRecord(P->ev0, P->s));
  CK(eval_enqueue(J, P->s));
  CK(cudaEventRecord(P->ev1, P->s));
  return eval_finish(J, results);
}
extern "C" perm_status perm_eval_batch(perm_jobs_t* J, const uint32_t* order, perm_job_result* results) {
  return guarded([&] {
    if (J) J->plan->subset = false;
    return eval_run(J, order, J ? J->n : 0, results);
  });
}

extern "C" perm_status perm_eval_subset(perm_jobs_t* J, const uint32_t* queue, int64_t count,
                                        perm_job_result* results) {
  if (!J || (!queue && count > 0)) return PERM_EINVAL;
  static const uint32_t none = 0;
  return guarded([&] {
    J->plan->subset = true;
    return eval_run(J, queue ? queue : &none, count, results);
  });
}

static perm_status perm_eval_replay_impl(perm_jobs_t* J, perm_job_result* results) {
  if (!J) return PERM_EINVAL;
  perm_plan* P = J->plan;
  EvalState* E = J->ev;
  if (!E) return PERM_ESTATE;
  if (!E->exec) {
    // capture the launch sequence once, on a stream of the library's own
    // (the caller's stream may be the legacy default stream, which cannot capture)
    CK(cudaStreamSynchronize(P->s));
    if (!E->cap) CK(cudaStreamCreateWithFlags(&E->cap, cudaStreamNonBlocking));
    CK(cudaStreamBeginCapture(E->cap, cudaStreamCaptureModeThreadLocal));
    const cudaError_t ce = eval_enqueue(J, E->cap);
    cudaGraph_t g = nullptr;
    const cudaError_t ee = cudaStreamEndCapture(E->cap, &g);
    CK(ce);
    CK(ee);
    E->graph = g;
    CK(cudaGraphInstantiate(&E->exec, E->graph, 0));
  }
  CK(cudaEventRecord(P->ev0, P->s));
  CK(cudaGraphLaunch(E->exec, P->s));
  CK(cudaEventRecord(P->ev1, P->s));
  return eval_finish(J, results);
}
extern "C" perm_status perm_eval_replay(perm_jobs_t* J, perm_job_result* results) {
  return guarded([&] { return perm_eval_replay_impl(J, results); });
}

static perm_status perm_last_eval_launches_impl(perm_plan_t* P, int32_t* launches) {
  if (!P || !launches) return PERM_EINVAL;
  *launches = P->last_launches;
  return PERM_OK;
}
extern "C" perm_status perm_last_eval_launches(perm_plan_t* P, int32_t* launches) {
  return guarded([&] { return perm_last_eval_launches_impl(P, launches); });
}

static perm_status perm_last_eval_ms_impl(perm_plan_t* P, float* ms) {
  if (!P || !ms) return PERM_EINVAL;
  *ms = P->last_ms;
  return PERM_OK;
}
extern "C" perm_status perm_last_eval_ms(perm_plan_t* P, float* ms) {
  return guarded([&] { return perm_last_eval_ms_impl(P, ms); });
}

// ---------------------------------------------------------------- a8: results
static void low_bits_signed(const uint64_t* w, int K, uint64_t* out) {
  // keep bits [0, K), sign-extend from bit K-1
  for (int k = 0; k < 4; ++k) out[k] = w[k];
  if (K >= 256) return;
  const int word = (K - 1) / 64, bit = (K - 1) % 64;
  const bool neg = (out[word] >> bit) & 1;
  const uint64_t keep = bit == 63 ? ~0ull : ((1ull << (bit + 1)) - 1);
  out[word] = neg ? (out[word] | ~keep) : (out[word] & keep);
  for (int k = word + 1; k < 4; ++k) out[k] = neg ? ~0ull : 0ull;
}

static perm_status result_words(perm_plan* P, std::vector<uint64_t>& words) {
  words.assign(4ull * P->count, 0ull);
  if (!P->evaluated) return PERM_ESTATE;
  std::vector<uint64_t> raw(4ull * P->count);
  CK(cudaMemcpyAsync(raw.data(), P->d_mat_acc, 32ull * P->count, cudaMemcpyDeviceToHost, P->s));
  CK(cudaStreamSynchronize(P->s));
  for (int i = 0; i < P->count; ++i) {
    uint64_t* o = &words[4ull * i];
    if (P->trivial[i] == 1) continue;
    if (P->trivial[i] == 2) {
      if (P->subset) continue;  // a sub-queue sum: the matrix has no job
      o[0] = 1;
      continue;
    }
    if (P->mod.p)
      o[0] = raw[4ull * i] % P->mod.p;  // a sum of residues: the residue of per(A_i)
    else
      low_bits_signed(&raw[4ull * i], P->kbits[i], o);
  }
  return PERM_OK;
}

static perm_status perm_result_words_impl(perm_plan_t* P, uint64_t* out, int32_t count) {
  if (!P || !out || count < P->count) return PERM_EINVAL;
  std::vector<uint64_t> w;
  perm_status st = result_words(P, w);
  if (st != PERM_OK) return st;
  memcpy(out, w.data(), 32ull * P->count);
  return PERM_OK;
}
extern "C" perm_status perm_result_words(perm_plan_t* P, uint64_t* out, int32_t count) {
  return guarded([&] { return perm_result_words_impl(P, out, count); });
}

static perm_status perm_result_bits_impl(perm_plan_t* P, int32_t index, int32_t* bits) {
  if (!P || !bits || index < 0 || index >= P->count) return PERM_EINVAL;
  *bits = P->mod.p ? 0 : P->kbits[index];  // residues carry no ring width
  return PERM_OK;
}
extern "C" perm_status perm_result_bits(perm_plan_t* P, int32_t index, int32_t* bits) {
  return guarded([&] { return perm_result_bits_impl(P, index, bits); });
}

static perm_status perm_result_impl(perm_plan_t* P, int32_t index, uint32_t* limbs, int32_t cap, int32_t* nlimbs,
                                    int32_t* sign) {
  if (!P || index < 0 || index >= P->count || !nlimbs || !sign) return PERM_EINVAL;
  std::vector<uint64_t> w;
  perm_status st = result_words(P, w);
  if (st != PERM_OK) return st;
  uint64_t v[4];
  for (int k = 0; k < 4; ++k) v[k] = w[4ull * index + k];
  const bool neg = (v[3] >> 63) & 1;
  if (neg) {  // magnitude of a two's complement value
    u256 t;
    for (int k = 0; k < 4; ++k) t.w[k] = v[k];
    t = u256_neg(t);
    for (int k = 0; k < 4; ++k) v[k] = t.w[k];
  }
  uint32_t l[8];
  for (int k = 0; k < 4; ++k) {
    l[2 * k] = (uint32_t)v[k];
    l[2 * k + 1] = (uint32_t)(v[k] >> 32);
  }
  int n = 8;
  while (n > 0 && l[n - 1] == 0) --n;
  *nlimbs = n;
  *sign = n == 0 ? 0 : (neg ? -1 : 1);
  if (cap < n || (n > 0 && !limbs)) return PERM_ESHORTBUF;
  for (int k = 0; k < n; ++k) limbs[k] = l[k];
  return PERM_OK;
}
extern "C" perm_status perm_result(perm_plan_t* P, int32_t index, uint32_t* limbs, int32_t cap, int32_t* nlimbs,
                                   int32_t* sign) {
  return guarded([&] { return perm_result_impl(P, index, limbs, cap, nlimbs, sign); });
}

static perm_status perm_jobs_export_impl(perm_jobs_t* J, int64_t* total_entries, int32_t* sizes, int64_t* mats,
                                         uint64_t* coef, int32_t* matrix) {
  if (!J || !total_entries) return PERM_EINVAL;
  perm_plan* P = J->plan;
  const int64_t n = J->n;
  int64_t tot = 0;
  for (int64_t j = 0; j < n; ++j) tot += (int64_t)J->h_m[j] * J->h_m[j];
  *total_entries = tot;
  if (!sizes) return PERM_OK;
  std::vector<uint64_t> arena(mats ? (size_t)std::max<int64_t>(J->arena_words, 1) : 1);
  std::vector<int64_t> off(n);
  std::vector<int32_t> nnz(n), mat(n);
  std::vector<uint64_t> cf(4 * n);
  if (n) {
    if (mats) CK(cudaMemcpyAsync(arena.data(), J->arena, 8 * J->arena_words, cudaMemcpyDeviceToHost, P->s));
    CK(cudaMemcpyAsync(off.data(), J->a.off, 8 * n, cudaMemcpyDeviceToHost, P->s));
    CK(cudaMemcpyAsync(nnz.data(), J->a.nnz, 4 * n, cudaMemcpyDeviceToHost, P->s));
    CK(cudaMemcpyAsync(mat.data(), J->a.mat, 4 * n, cudaMemcpyDeviceToHost, P->s));
    CK(cudaMemcpyAsync(cf.data(), J->a.coef, 32 * n, cudaMemcpyDeviceToHost, P->s));
    CK(cudaStreamSynchronize(P->s));
  }
  int64_t o = 0;
  for (int64_t j = 0; j < n; ++j) {
    const int m = J->h_m[j];
    sizes[j] = m;
    if (mats) {
      int64_t* d = mats + o;
      for (int64_t k = 0; k < (int64_t)m * m; ++k) d[k] = 0;
      CsrView v = csr_view(arena.data(), off[j], m, nnz[j]);
      for (int r = 0; r < m; ++r)
        for (int p = v.rowptr[r]; p < v.rowptr[r + 1]; ++p) d[(int64_t)r * m + v.col[p]] = v.val[p];
    }
    o += (int64_t)m * m;
    if (coef)
      for (int w = 0; w < 4; ++w) coef[4 * j + w] = cf[4 * j + w];
    if (matrix) matrix[j] = mat[j];
  }
  return PERM_OK;
}
extern "C" perm_status perm_jobs_export(perm_jobs_t* J, int64_t* total_entries, int32_t* sizes, int64_t* mats,
                                        uint64_t* coef, int32_t* matrix) {
  return guarded([&] { return perm_jobs_export_impl(J, total_entries, sizes, mats, coef, matrix); });
}

static perm_status perm_jobs_select_impl(perm_jobs_t* J, const int64_t* idx, int64_t count, int32_t* sizes,
                                         int64_t* mats, int64_t mats_cap, uint64_t* coef, int32_t* matrix,
                                         int64_t* entries) {
  if (!J || count < 0 || (count > 0 && (!idx || !sizes)) || !entries) return PERM_EINVAL;
  perm_plan* P = J->plan;
  int64_t tot = 0;
  for (int64_t k = 0; k < count; ++k) {
    if (idx[k] < 0 || idx[k] >= J->n) return PERM_EINVAL;
    sizes[k] = J->h_m[idx[k]];
    tot += (int64_t)sizes[k] * sizes[k];
  }
  *entries = tot;
  if (mats && mats_cap < tot) return PERM_ESHORTBUF;
  int64_t o = 0;
  for (int64_t k = 0; k < count; ++k) {
    const int64_t j = idx[k];
    const int m = sizes[k];
    int64_t off = 0;
    int32_t nnz = 0, mat = 0;
    uint64_t cf[4] = {0, 0, 0, 0};
    CK(cudaMemcpyAsync(&off, J->a.off + j, 8, cudaMemcpyDeviceToHost, P->s));
    CK(cudaMemcpyAsync(&nnz, J->a.nnz + j, 4, cudaMemcpyDeviceToHost, P->s));
    CK(cudaMemcpyAsync(&mat, J->a.mat + j, 4, cudaMemcpyDeviceToHost, P->s));
    CK(cudaMemcpyAsync(cf, J->a.coef + 4 * j, 32, cudaMemcpyDeviceToHost, P->s));
    CK(cudaStreamSynchronize(P->s));
    if (mats) {
      const int64_t bw = blk_words(m, nnz);
      std::vector<uint64_t> blk((size_t)std::max<int64_t>(bw, 1));
      CK(cudaMemcpyAsync(blk.data(), J->arena + off, 8 * bw, cudaMemcpyDeviceToHost, P->s));
      CK(cudaStreamSynchronize(P->s));
      int64_t* d = mats + o;
      for (int64_t e = 0; e < (int64_t)m * m; ++e) d[e] = 0;
      CsrView v = csr_view(blk.data(), 0, m, nnz);
      for (int r = 0; r < m; ++r)
        for (int q = v.rowptr[r]; q < v.rowptr[r + 1]; ++q) d[(int64_t)r * m + v.col[q]] = v.val[q];
    }
    o += (int64_t)m * m;
    if (coef)
      for (int w = 0; w < 4; ++w) coef[4 * k + w] = cf[w];
    if (matrix) matrix[k] = mat;
  }
  return PERM_OK;
}
extern "C" perm_status perm_jobs_select(perm_jobs_t* J, const int64_t* idx, int64_t count, int32_t* sizes,
                                        int64_t* mats, int64_t mats_cap, uint64_t* coef, int32_t* matrix,
                                        int64_t* entries) {
  return guarded([&] { return perm_jobs_select_impl(J, idx, count, sizes, mats, mats_cap, coef, matrix, entries); });
}

static perm_status perm_exact_impl(const perm_matrix* a, const perm_opts* opts, uint32_t* limbs, int32_t cap,
                                   int32_t* nlimbs, int32_t* sign) {
  perm_plan_t* P = nullptr;
  perm_status st = perm_plan_create(a, 1, opts, &P);
  if (st != PERM_OK) return st;
  perm_jobs_t* J = nullptr;
  int64_t nj = 0;
  st = perm_expand(P, &J, &nj);
  if (st == PERM_OK && nj > 0) st = perm_order(J, P->opts.order, nullptr);
  if (st == PERM_OK) st = perm_eval_batch(J, nullptr, nullptr);
  if (st == PERM_OK) st = perm_result(P, 0, limbs, cap, nlimbs, sign);
  perm_plan_destroy(P);
  return st;
}
extern "C" perm_status perm_exact(const perm_matrix* a, const perm_opts* opts, uint32_t* limbs, int32_t cap,
                                  int32_t* nlimbs, int32_t* sign) {
  return guarded([&] { return perm_exact_impl(a, opts, limbs, cap, nlimbs, sign); });
}

// ---------------------------------------------------------------- learned model
struct Scratch {
  cudaStream_t s;
  std::vector<void*> p;
  template <typename T>
  T* get(size_t n) {
    void* q = nullptr;
    if (cudaMallocAsync(&q, sizeof(T) * (n ? n : 1), s) != cudaSuccess) return nullptr;
    p.push_back(q);
    return reinterpret_cast<T*>(q);
  }
  ~Scratch() {
    for (void* q : p) cudaFreeAsync(q, s);
    cudaStreamSynchronize(s);
  }
};

static perm_status perm_mlp_grad_impl(const float* params, const float* feats, const float* target, int32_t count,
                                      void* stream, float* loss, float* grad) {
  if (!params || !feats || !target || count < 1 || !loss || !grad) return PERM_EINVAL;
  Scratch S{(cudaStream_t)stream, {}};
  float* dp = S.get<float>(PERM_MLP_PARAMS);
  float* dx = S.get<float>((size_t)count * PERM_MLP_FEATURES);
  float* dy = S.get<float>(count);
  float* sc = S.get<float>(mlp_scratch_floats(count));
  float* dg = S.get<float>(PERM_MLP_PARAMS);
  float* dl = S.get<float>(1);
  if (!dp || !dx || !dy || !sc || !dg || !dl) return PERM_ENOMEM;
  CK(cudaMemcpyAsync(dp, params, 4 * PERM_MLP_PARAMS, cudaMemcpyHostToDevice, S.s));
  CK(cudaMemcpyAsync(dx, feats, 4ull * count * PERM_MLP_FEATURES, cudaMemcpyHostToDevice, S.s));
  CK(cudaMemcpyAsync(dy, target, 4ull * count, cudaMemcpyHostToDevice, S.s));
  CK(mlp_forward_backward(dp, dx, dy, count, sc, dg, dl, S.s));
  CK(cudaMemcpyAsync(grad, dg, 4 * PERM_MLP_PARAMS, cudaMemcpyDeviceToHost, S.s));
  CK(cudaMemcpyAsync(loss, dl, 4, cudaMemcpyDeviceToHost, S.s));
  CK(cudaStreamSynchronize(S.s));
  return PERM_OK;
}
extern "C" perm_status perm_mlp_grad(const float* params, const float* feats, const float* target, int32_t count,
                                     void* stream, float* loss, float* grad) {
  return guarded([&] { return perm_mlp_grad_impl(params, feats, target, count, stream, loss, grad); });
}

static perm_status perm_mlp_train_impl(float* params, const float* feats, const float* target, int32_t count,
                                       int32_t steps, float lr, void* stream, float* final_loss) {
  if (!params || !feats || !target || count < 1 || steps < 0) return PERM_EINVAL;
  Scratch S{(cudaStream_t)stream, {}};
  float* dp = S.get<float>(PERM_MLP_PARAMS);
  float* dx = S.get<float>((size_t)count * PERM_MLP_FEATURES);
  float* dy = S.get<float>(count);
  float* sc = S.get<float>(mlp_scratch_floats(count));
  float* dg = S.get<float>(PERM_MLP_PARAMS);
  float* m1 = S.get<float>(PERM_MLP_PARAMS);
  float* m2 = S.get<float>(PERM_MLP_PARAMS);
  float* dl = S.get<float>(1);
  if (!dp || !dx || !dy || !sc || !dg || !m1 || !m2 || !dl) return PERM_ENOMEM;
  CK(cudaMemcpyAsync(dp, params, 4 * PERM_MLP_PARAMS, cudaMemcpyHostToDevice, S.s));
  CK(cudaMemcpyAsync(dx, feats, 4ull * count * PERM_MLP_FEATURES, cudaMemcpyHostToDevice, S.s));
  CK(cudaMemcpyAsync(dy, target, 4ull * count, cudaMemcpyHostToDevice, S.s));
  CK(cudaMemsetAsync(m1, 0, 4 * PERM_MLP_PARAMS, S.s));
  CK(cudaMemsetAsync(m2, 0, 4 * PERM_MLP_PARAMS, S.s));
  for (int32_t t = 1; t <= steps; ++t) {
    CK(mlp_forward_backward(dp, dx, dy, count, sc, dg, dl, S.s));
    CK(mlp_adam_step(dp, dg, m1, m2, t, lr, S.s));
  }
  if (final_loss) {
    CK(mlp_forward_backward(dp, dx, dy, count, sc, dg, dl, S.s));
    CK(cudaMemcpyAsync(final_loss, dl, 4, cudaMemcpyDeviceToHost, S.s));
  }
  CK(cudaMemcpyAsync(params, dp, 4 * PERM_MLP_PARAMS, cudaMemcpyDeviceToHost, S.s));
  CK(cudaStreamSynchronize(S.s));
  return PERM_OK;
}
extern "C" perm_status perm_mlp_train(float* params, const float* feats, const float* target, int32_t count,
                                      int32_t steps, float lr, void* stream, float* final_loss) {
  return guarded([&] { return perm_mlp_train_impl(params, feats, target, count, steps, lr, stream, final_loss); });
}

static perm_status perm_mlp_predict_impl(const float* params, const float* feats, int32_t count, void* stream,
                                         float* pred) {
  if (!params || !feats || count < 1 || !pred) return PERM_EINVAL;
  Scratch S{(cudaStream_t)stream, {}};
  float* dp = S.get<float>(PERM_MLP_PARAMS);
  float* dx = S.get<float>((size_t)count * PERM_MLP_FEATURES);
  float* dy = S.get<float>(count);
  if (!dp || !dx || !dy) return PERM_ENOMEM;
  CK(cudaMemcpyAsync(dp, params, 4 * PERM_MLP_PARAMS, cudaMemcpyHostToDevice, S.s));
  CK(cudaMemcpyAsync(dx, feats, 4ull * count * PERM_MLP_FEATURES, cudaMemcpyHostToDevice, S.s));
  CK(mlp_predict(dp, dx, count, dy, S.s));
  CK(cudaMemcpyAsync(pred, dy, 4ull * count, cudaMemcpyDeviceToHost, S.s));
  CK(cudaStreamSynchronize(S.s));
  return PERM_OK;
}
extern "C" perm_status perm_mlp_predict(const float* params, const float* feats, int32_t count, void* stream,
                                        float* pred) {
  return guarded([&] { return perm_mlp_predict_impl(params, feats, count, stream, pred); });
}

static perm_status perm_mlp_attach_impl(perm_plan_t* P, const float* params) {
  if (!P || !params) return PERM_EINVAL;
  P->mlp.assign(params, params + PERM_MLP_PARAMS);
  if (P->jobs) P->jobs->has_order = false;
  return PERM_OK;
}
extern "C" perm_status perm_mlp_attach(perm_plan_t* P, const float* params) {
  return guarded([&] { return perm_mlp_attach_impl(P, params); });
}

// ---------------------------------------------------------------- measurement
static perm_status perm_ubench_imad_impl(int32_t blocks, int32_t iters, void* stream, float* ms, double* rate) {
  if (blocks < 1 || iters < 1 || !ms || !rate) return PERM_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  Scratch S{s, {}};
  uint32_t* sink = S.get<uint32_t>(blocks);
  if (!sink) return PERM_ENOMEM;
  cudaEvent_t a, b;
  CK(cudaEventCreate(&a));
  CK(cudaEventCreate(&b));
  CK(launch_ubench_imad(blocks, iters, sink, s));  // warm-up
  CK(cudaEventRecord(a, s));
  CK(launch_ubench_imad(blocks, iters, sink, s));
  CK(cudaEventRecord(b, s));
  CK(cudaEventSynchronize(b));
  CK(cudaEventElapsedTime(ms, a, b));
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  *rate = (double)blocks * 256.0 * 16.0 * (double)iters / (*ms * 1e-3);
  return PERM_OK;
}
extern "C" perm_status perm_ubench_imad(int32_t blocks, int32_t iters, void* stream, float* ms, double* rate) {
  return guarded([&] { return perm_ubench_imad_impl(blocks, iters, stream, ms, rate); });
}
