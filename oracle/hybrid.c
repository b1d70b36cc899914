/*
 * ORACLE -- test infrastructure only.  Plain, slow, exact CPU reference for the
 * sparse-permanent path.  Only tests/, __graft_entry__.smoke() and bench.py's
 * CPU-baseline leg may load this library; the product path never does.
 *
 * What it computes (paper sections cited per function):
 *   - per(A), the permanent of Eq. 1, by Algorithm H_per (Section 2.1): the
 *     expansion of Eq. 2 while the smallest line count s satisfies s < 5 and
 *     n > 2 (and n > L, an optional leaf cut-off), else Ryser's formula.
 *   - the job list of Algorithm PH, Step 2 (Section 2.2): Eq. 2 applied level
 *     by level, children appended in order ("natural order").
 *   - Ryser's inclusion-exclusion formula written out over all 2^n column
 *     subsets (Section 1), with no Gray code and no Nijenhuis-Wilf offset.
 *
 * Readings of the paper taken here (the paper leaves them open):
 *   - pivot: s = min over all row and column nonzero counts; the lowest-index
 *     row with count s is taken, else the lowest-index column with count s;
 *   - the pivot row's nonzeros j1 < j2 < j3 < j4 play the roles of a, b, c, d
 *     of Eq. 2; merge(p, q) deletes the pivot row, replaces column p by
 *     M[i][p]*col_q + M[i][q]*col_p and deletes column q, other columns keep
 *     their order;
 *   - k = s nonzeros: k=1 -> (v1 * minor(i, j1)); k=2 -> merge(j1, j2);
 *     k=3 -> merge(j1, j2), (v3 * minor(i, j3)); k=4 -> merge(j1, j2),
 *     merge(j3, j4).  A scalar factor is carried as a per-job coefficient;
 *   - a column pivot is the same rule applied to the transpose;
 *   - a child holding a zero row or zero column is not emitted (its permanent
 *     is 0);
 *   - in the level-by-level expansion a node that is a leaf (n <= max(L, 2),
 *     or s >= 5) is carried unchanged to the next level, in place;
 *   - option "three" (s >= 5 split, not in Algorithm H_per, which sends such
 *     a node to R-NW): Eq. 2 with all three children -- A1 = merge(j1, j2),
 *     A2 = merge(j3, j4) (c*y4 + d*y3 in column j3, column j4 deleted), A3 =
 *     the node with the pivot line's entries at j1..j4 set to 0 (same order);
 *     then only n <= max(L, 2) makes a leaf.
 *
 * Exactness: matrix entries are int64 and every multiply/add on them is
 * overflow-checked (an overflow makes the call fail with ORACLE_EOVERFLOW);
 * coefficients, leaf values and sums are signed big integers.
 */
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORACLE_OK 0
#define ORACLE_EINVAL 1
#define ORACLE_EOVERFLOW 2
#define ORACLE_ESHORTBUF 5
#define ORACLE_ENOMEM 6

#define MAXN 128
#define BI_LIMBS 80 /* 2560-bit magnitude */

/* ---------------- signed big integer, sign-magnitude, uint32 limbs ------- */
typedef struct {
  int neg;         /* 1 if negative (never set for zero) */
  int len;         /* number of used limbs; 0 means zero */
  uint32_t d[BI_LIMBS];
} bigint;

static void bi_zero(bigint* x) { x->neg = 0; x->len = 0; }

static void bi_trim(bigint* x) {
  while (x->len > 0 && x->d[x->len - 1] == 0) x->len--;
  if (x->len == 0) x->neg = 0;
}

static void bi_from_i64(bigint* x, int64_t v) {
  uint64_t m = v < 0 ? (uint64_t)0 - (uint64_t)v : (uint64_t)v;
  x->neg = v < 0;
  x->d[0] = (uint32_t)m;
  x->d[1] = (uint32_t)(m >> 32);
  x->len = 2;
  bi_trim(x);
}

/* |a| + |b| into r (magnitudes only). Returns 0 or ORACLE_EOVERFLOW. */
static int mag_add(bigint* r, const bigint* a, const bigint* b) {
  int n = a->len > b->len ? a->len : b->len;
  uint64_t carry = 0;
  for (int i = 0; i < n; i++) {
    uint64_t s = carry;
    if (i < a->len) s += a->d[i];
    if (i < b->len) s += b->d[i];
    r->d[i] = (uint32_t)s;
    carry = s >> 32;
  }
  r->len = n;
  if (carry) {
    if (n >= BI_LIMBS) return ORACLE_EOVERFLOW;
    r->d[n] = (uint32_t)carry;
    r->len = n + 1;
  }
  return 0;
}

/* compare magnitudes */
static int mag_cmp(const bigint* a, const bigint* b) {
  if (a->len != b->len) return a->len < b->len ? -1 : 1;
  for (int i = a->len - 1; i >= 0; i--)
    if (a->d[i] != b->d[i]) return a->d[i] < b->d[i] ? -1 : 1;
  return 0;
}

/* |a| - |b| into r, requires |a| >= |b| */
static void mag_sub(bigint* r, const bigint* a, const bigint* b) {
  int64_t borrow = 0;
  for (int i = 0; i < a->len; i++) {
    int64_t s = (int64_t)a->d[i] - borrow - (i < b->len ? (int64_t)b->d[i] : 0);
    borrow = s < 0;
    if (s < 0) s += ((int64_t)1 << 32);
    r->d[i] = (uint32_t)s;
  }
  r->len = a->len;
}

/* r = a + b (r may alias a or b) */
static int bi_add(bigint* r, const bigint* a, const bigint* b) {
  bigint t;
  if (a->neg == b->neg) {
    int e = mag_add(&t, a, b);
    if (e) return e;
    t.neg = a->neg;
  } else if (mag_cmp(a, b) >= 0) {
    mag_sub(&t, a, b);
    t.neg = a->neg;
  } else {
    mag_sub(&t, b, a);
    t.neg = b->neg;
  }
  bi_trim(&t);
  *r = t;
  return 0;
}

/* r = a * b, schoolbook */
static int bi_mul(bigint* r, const bigint* a, const bigint* b) {
  bigint t;
  if (a->len == 0 || b->len == 0) { bi_zero(r); return 0; }
  if (a->len + b->len > BI_LIMBS) {
    /* may still fit after trimming; compute into a wider scratch */
    uint32_t w[2 * BI_LIMBS];
    memset(w, 0, sizeof(w));
    for (int i = 0; i < a->len; i++) {
      uint64_t carry = 0;
      for (int j = 0; j < b->len; j++) {
        uint64_t cur = (uint64_t)a->d[i] * b->d[j] + w[i + j] + carry;
        w[i + j] = (uint32_t)cur;
        carry = cur >> 32;
      }
      w[i + b->len] = (uint32_t)carry;
    }
    int n = a->len + b->len;
    while (n > 0 && w[n - 1] == 0) n--;
    if (n > BI_LIMBS) return ORACLE_EOVERFLOW;
    memcpy(t.d, w, (size_t)n * 4);
    t.len = n;
  } else {
    memset(t.d, 0, sizeof(uint32_t) * (size_t)(a->len + b->len));
    for (int i = 0; i < a->len; i++) {
      uint64_t carry = 0;
      for (int j = 0; j < b->len; j++) {
        uint64_t cur = (uint64_t)a->d[i] * b->d[j] + t.d[i + j] + carry;
        t.d[i + j] = (uint32_t)cur;
        carry = cur >> 32;
      }
      t.d[i + b->len] = (uint32_t)carry;
    }
    t.len = a->len + b->len;
  }
  t.neg = a->neg ^ b->neg;
  bi_trim(&t);
  *r = t;
  return 0;
}

static int bi_mul_i64(bigint* r, const bigint* a, int64_t v) {
  bigint b;
  bi_from_i64(&b, v);
  return bi_mul(r, a, &b);
}

/* export magnitude as little-endian uint32 limbs */
static int bi_export(const bigint* x, uint32_t* limbs, int cap, int* nlimbs, int* sign) {
  *nlimbs = x->len;
  *sign = x->len == 0 ? 0 : (x->neg ? -1 : 1);
  if (x->len > cap) return ORACLE_ESHORTBUF;
  for (int i = 0; i < x->len; i++) limbs[i] = x->d[i];
  return ORACLE_OK;
}

/* ---------------- dense exact matrices ---------------------------------- */
typedef struct {
  int n;
  int64_t* a; /* n*n row-major, owned */
} mat;

static int mat_alloc(mat* m, int n) {
  m->n = n;
  m->a = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n * n : 1));
  return m->a ? 0 : ORACLE_ENOMEM;
}
static void mat_free(mat* m) { free(m->a); m->a = NULL; }
#define AT(m, i, j) ((m)->a[(size_t)(i) * (m)->n + (j)])

/* Ryser's formula (Section 1): per(A) = (-1)^n sum_{S subset [n]} (-1)^{|S|}
 * prod_i sum_{j in S} a_ij, every subset enumerated in binary order and every
 * row sum recomputed from the matrix.  Exact big-integer products and sum. */
static int ryser_textbook(const mat* m, bigint* out) {
  int n = m->n;
  bi_zero(out);
  if (n == 0) { bi_from_i64(out, 1); return 0; }
  if (n > 30) return ORACLE_EINVAL;
  uint64_t nsub = (uint64_t)1 << n;
  bigint term, acc;
  bi_zero(&acc);
  for (uint64_t S = 1; S < nsub; S++) {
    bi_from_i64(&term, 1);
    int zero = 0;
    for (int i = 0; i < n && !zero; i++) {
      int64_t rs = 0;
      for (int j = 0; j < n; j++)
        if (S >> j & 1) {
          if (__builtin_add_overflow(rs, AT(m, i, j), &rs)) return ORACLE_EOVERFLOW;
        }
      if (rs == 0) { zero = 1; break; }
      int e = bi_mul_i64(&term, &term, rs);
      if (e) return e;
    }
    if (zero) continue;
    int size = __builtin_popcountll(S);
    if ((n - size) & 1) term.neg = !term.neg && term.len > 0;
    int e = bi_add(&acc, &acc, &term);
    if (e) return e;
  }
  *out = acc;
  return 0;
}

/* line counts; returns 1 if some row or column is all zero */
static int line_counts(const mat* m, int* rc, int* cc) {
  int n = m->n;
  for (int j = 0; j < n; j++) cc[j] = 0;
  for (int i = 0; i < n; i++) {
    rc[i] = 0;
    for (int j = 0; j < n; j++)
      if (AT(m, i, j) != 0) { rc[i]++; cc[j]++; }
  }
  for (int i = 0; i < n; i++)
    if (rc[i] == 0 || cc[i] == 0) return 1;
  return 0;
}

typedef struct {
  int s;        /* smallest line count */
  int is_col;   /* 1 if the pivot line is a column */
  int idx;      /* pivot line index */
} pivot_t;

/* Algorithm H_per, Step 1: s = min line count; tie-break reading above. */
static pivot_t choose_pivot(const int* rc, const int* cc, int n) {
  pivot_t p = {1 << 30, 0, -1};
  for (int i = 0; i < n; i++)
    if (rc[i] < p.s) { p.s = rc[i]; p.idx = i; p.is_col = 0; }
  for (int j = 0; j < n; j++)
    if (cc[j] < p.s) { p.s = cc[j]; p.idx = j; p.is_col = 1; }
  return p;
}

static void transpose_into(const mat* src, mat* dst) {
  int n = src->n;
  for (int i = 0; i < n; i++)
    for (int j = 0; j < n; j++) AT(dst, j, i) = AT(src, i, j);
}

/* child = src without row i and column q, column p replaced by
 * src[i][p]*col_q + src[i][q]*col_p (Eq. 2's a*y2 + b*y1). */
static int make_merge(const mat* src, int i, int p, int q, mat* child) {
  int n = src->n;
  int64_t a = AT(src, i, p), b = AT(src, i, q);
  int ri = 0;
  for (int r = 0; r < n; r++) {
    if (r == i) continue;
    int ci = 0;
    for (int c = 0; c < n; c++) {
      if (c == q) continue;
      int64_t v = AT(src, r, c);
      if (c == p) {
        int64_t t1, t2;
        if (__builtin_mul_overflow(a, AT(src, r, q), &t1)) return ORACLE_EOVERFLOW;
        if (__builtin_mul_overflow(b, AT(src, r, p), &t2)) return ORACLE_EOVERFLOW;
        if (__builtin_add_overflow(t1, t2, &v)) return ORACLE_EOVERFLOW;
      }
      child->a[(size_t)ri * (n - 1) + ci] = v;
      ci++;
    }
    ri++;
  }
  child->n = n - 1;
  return 0;
}

/* child = src without row i and column p */
static void make_minor(const mat* src, int i, int p, mat* child) {
  int n = src->n;
  int ri = 0;
  for (int r = 0; r < n; r++) {
    if (r == i) continue;
    int ci = 0;
    for (int c = 0; c < n; c++) {
      if (c == p) continue;
      child->a[(size_t)ri * (n - 1) + ci] = AT(src, r, c);
      ci++;
    }
    ri++;
  }
  child->n = n - 1;
}

/* One step of Eq. 2 on a node that is not a leaf.  Fills up to 3 children
 * (already transposed back for a column pivot) and their scalar factors:
 * two for k < 5 (the readings above), three for k >= 5 (option "three").
 * Children with a zero line are dropped.  Returns the number kept, or a
 * negative error code. */
static int e2_children(const mat* node, const pivot_t* pv, mat* ch, int64_t* fac) {
  int n = node->n;
  mat t, work;
  const mat* src = node;
  int e;
  if (pv->is_col) {
    if ((e = mat_alloc(&t, n))) return -e;
    transpose_into(node, &t);
    src = &t;
  }
  int i = pv->idx;
  int js[MAXN], k = 0;
  for (int j = 0; j < n; j++)
    if (AT(src, i, j) != 0) js[k++] = j;
  /* k == pv->s here */
  int nout = 0;
  if ((e = mat_alloc(&work, n))) { if (pv->is_col) mat_free(&t); return -e; }
  for (int c = 0; c < 3; c++) {
    int kind = 0; /* 1 merge, 2 minor, 3 pivot row's first four entries cleared */
    int p = 0, q = 0;
    int64_t f = 1;
    if (c == 0) {
      if (k == 1) { kind = 2; p = js[0]; f = AT(src, i, p); }
      else { kind = 1; p = js[0]; q = js[1]; }
    } else if (c == 1) {
      if (k == 3) { kind = 2; p = js[2]; f = AT(src, i, p); }
      else if (k >= 4) { kind = 1; p = js[2]; q = js[3]; }
      else break;
    } else {
      if (k >= 5) kind = 3;
      else break;
    }
    int cn = n - 1;
    work.n = n;
    if (kind == 1) {
      if ((e = make_merge(src, i, p, q, &work))) { nout = -e; break; }
    } else if (kind == 2) {
      make_minor(src, i, p, &work);
    } else {
      cn = n;
      memcpy(work.a, src->a, sizeof(int64_t) * (size_t)n * n);
      for (int u = 0; u < 4; u++) work.a[(size_t)i * n + js[u]] = 0;
    }
    mat* out = &ch[nout];
    if ((e = mat_alloc(out, cn))) { nout = -e; break; }
    if (pv->is_col) {
      work.n = cn;
      transpose_into(&work, out);
    } else {
      memcpy(out->a, work.a, sizeof(int64_t) * (size_t)cn * cn);
    }
    int rc[MAXN], cc[MAXN];
    if (cn > 0 && line_counts(out, rc, cc)) { mat_free(out); continue; }
    fac[nout] = f;
    nout++;
  }
  mat_free(&work);
  if (pv->is_col) mat_free(&t);
  return nout;
}

static int is_leaf(const mat* m, int L, int three, const pivot_t* pv) {
  int cut = L > 2 ? L : 2;
  return m->n <= cut || (pv->s >= 5 && !three);
}

/* Algorithm H_per (Section 2.1), recursive, with coefficient. */
static int hper_rec(const mat* m, int L, int three, bigint* out) {
  int n = m->n;
  bi_zero(out);
  if (n == 0) { bi_from_i64(out, 1); return 0; }
  int rc[MAXN], cc[MAXN];
  if (line_counts(m, rc, cc)) return 0;
  pivot_t pv = choose_pivot(rc, cc, n);
  if (is_leaf(m, L, three, &pv)) return ryser_textbook(m, out);
  mat ch[3];
  int64_t fac[3];
  int k = e2_children(m, &pv, ch, fac);
  if (k < 0) return -k;
  int err = 0;
  for (int c = 0; c < k; c++) {
    bigint sub;
    if (!err) err = hper_rec(&ch[c], L, three, &sub);
    if (!err && fac[c] != 1) err = bi_mul_i64(&sub, &sub, fac[c]);
    if (!err) err = bi_add(out, out, &sub);
    mat_free(&ch[c]);
  }
  return err;
}

/* ---------------- job lists (Algorithm PH, Step 2) ----------------------- */
typedef struct {
  mat m;
  bigint coef;
} job_t;

typedef struct {
  job_t* v;
  int64_t n, cap;
} joblist;

static int jl_push(joblist* l, job_t* j) {
  if (l->n == l->cap) {
    int64_t nc = l->cap ? 2 * l->cap : 64;
    job_t* nv = (job_t*)realloc(l->v, sizeof(job_t) * (size_t)nc);
    if (!nv) return ORACLE_ENOMEM;
    l->v = nv;
    l->cap = nc;
  }
  l->v[l->n++] = *j;
  return 0;
}

static void jl_free(joblist* l) {
  for (int64_t i = 0; i < l->n; i++) mat_free(&l->v[i].m);
  free(l->v);
  l->v = NULL;
  l->n = l->cap = 0;
}

/* Expand d levels.  The root is dropped if it has a zero line. */
static int expand_levels(const int64_t* a, int n, int d, int L, int three, joblist* out) {
  joblist cur = {0}, nxt = {0};
  job_t root;
  int e;
  if ((e = mat_alloc(&root.m, n))) return e;
  memcpy(root.m.a, a, sizeof(int64_t) * (size_t)n * n);
  bi_from_i64(&root.coef, 1);
  int rc[MAXN], cc[MAXN];
  if (n > 0 && line_counts(&root.m, rc, cc)) { mat_free(&root.m); *out = cur; return 0; }
  if ((e = jl_push(&cur, &root))) return e;
  for (int lvl = 0; lvl < d; lvl++) {
    for (int64_t w = 0; w < cur.n; w++) {
      job_t* jb = &cur.v[w];
      int m = jb->m.n;
      pivot_t pv = {0, 0, 0};
      if (m > 0) {
        line_counts(&jb->m, rc, cc);
        pv = choose_pivot(rc, cc, m);
      }
      if (m == 0 || is_leaf(&jb->m, L, three, &pv)) {
        job_t keep = *jb;
        jb->m.a = NULL;
        if ((e = jl_push(&nxt, &keep))) goto fail;
        continue;
      }
      mat ch[3];
      int64_t fac[3];
      int k = e2_children(&jb->m, &pv, ch, fac);
      if (k < 0) { e = -k; goto fail; }
      for (int c = 0; c < k; c++) {
        job_t cj;
        cj.m = ch[c];
        cj.coef = jb->coef;
        if (fac[c] != 1 && (e = bi_mul_i64(&cj.coef, &cj.coef, fac[c]))) goto fail;
        if ((e = jl_push(&nxt, &cj))) goto fail;
      }
    }
    jl_free(&cur);
    cur = nxt;
    nxt.v = NULL;
    nxt.n = nxt.cap = 0;
  }
  *out = cur;
  return 0;
fail:
  jl_free(&cur);
  jl_free(&nxt);
  return e;
}

/* ---------------- threads over jobs ------------------------------------ */
typedef struct {
  joblist* jobs;
  int L;
  int three;
  int64_t next;
  pthread_mutex_t mu;
  bigint* per_job;   /* per(job) without coefficient */
  int err;
} pool_t;

static void* worker(void* arg) {
  pool_t* P = (pool_t*)arg;
  for (;;) {
    pthread_mutex_lock(&P->mu);
    int64_t w = P->next++;
    int stop = P->err;
    pthread_mutex_unlock(&P->mu);
    if (stop || w >= P->jobs->n) break;
    int e = hper_rec(&P->jobs->v[w].m, P->L, P->three, &P->per_job[w]);
    if (e) {
      pthread_mutex_lock(&P->mu);
      if (!P->err) P->err = e;
      pthread_mutex_unlock(&P->mu);
    }
  }
  return NULL;
}

static int eval_jobs(joblist* jobs, int L, int three, int nthreads, bigint* per_job) {
  pool_t P;
  P.jobs = jobs;
  P.L = L;
  P.three = three;
  P.next = 0;
  P.per_job = per_job;
  P.err = 0;
  pthread_mutex_init(&P.mu, NULL);
  if (nthreads < 1) nthreads = 1;
  if (nthreads > 256) nthreads = 256;
  pthread_t th[256];
  int started = 0;
  for (int t = 0; t < nthreads; t++)
    if (pthread_create(&th[t], NULL, worker, &P) == 0) started++;
  if (started == 0) worker(&P);
  for (int t = 0; t < started; t++) pthread_join(th[t], NULL);
  pthread_mutex_destroy(&P.mu);
  return P.err;
}

static int check_input(int n, const int64_t* a) {
  if (n < 0 || n > MAXN || (n > 0 && !a)) return ORACLE_EINVAL;
  return 0;
}

/* ---------------- exported entry points --------------------------------- */

/* per(A) by textbook Ryser (Section 1). n <= 30. */
int oracle_ryser(int n, const int64_t* a, uint32_t* limbs, int cap, int* nlimbs, int* sign) {
  int e = check_input(n, a);
  if (e) return e;
  if (n > 30) return ORACLE_EINVAL;
  mat m;
  if ((e = mat_alloc(&m, n))) return e;
  memcpy(m.a, a, sizeof(int64_t) * (size_t)n * n);
  bigint r;
  e = ryser_textbook(&m, &r);
  mat_free(&m);
  if (e) return e;
  return bi_export(&r, limbs, cap, nlimbs, sign);
}

/* per(A) by Algorithm PH: expand d levels (Step 2), evaluate every job by
 * H_per with leaf cut-off L (Step 3, nthreads workers), sum (Step 4).
 * three: split s >= 5 nodes by Eq. 2's three children. */
int oracle_permanent(int n, const int64_t* a, int d, int L, int three, int nthreads,
                     uint32_t* limbs, int cap, int* nlimbs, int* sign) {
  int e = check_input(n, a);
  if (e) return e;
  if (n == 0) {
    bigint one;
    bi_from_i64(&one, 1);
    return bi_export(&one, limbs, cap, nlimbs, sign);
  }
  joblist jobs = {0};
  if ((e = expand_levels(a, n, d < 0 ? 0 : d, L, three, &jobs))) return e;
  bigint* pj = (bigint*)calloc((size_t)(jobs.n > 0 ? jobs.n : 1), sizeof(bigint));
  if (!pj) { jl_free(&jobs); return ORACLE_ENOMEM; }
  e = eval_jobs(&jobs, L, three, nthreads, pj);
  bigint tot;
  bi_zero(&tot);
  for (int64_t w = 0; !e && w < jobs.n; w++) {
    bigint t;
    e = bi_mul(&t, &pj[w], &jobs.v[w].coef);
    if (!e) e = bi_add(&tot, &tot, &t);
  }
  free(pj);
  jl_free(&jobs);
  if (e) return e;
  return bi_export(&tot, limbs, cap, nlimbs, sign);
}

/* Job list after d levels of Algorithm PH, Step 2.  Two-call protocol:
 * with sizes == NULL only *njobs and *total_entries are set.  Otherwise
 * sizes[w] = job order, mats gets the row-major dense jobs back to back,
 * coef_limbs[w*coef_cap ...] the |coef| limbs, coef_sign[w] its sign. */
int oracle_jobs(int n, const int64_t* a, int d, int L, int three, int64_t* njobs, int64_t* total_entries,
                int32_t* sizes, int64_t* mats, uint32_t* coef_limbs, int coef_cap,
                int32_t* coef_sign) {
  int e = check_input(n, a);
  if (e) return e;
  joblist jobs = {0};
  if ((e = expand_levels(a, n, d < 0 ? 0 : d, L, three, &jobs))) return e;
  int64_t tot = 0;
  for (int64_t w = 0; w < jobs.n; w++) tot += (int64_t)jobs.v[w].m.n * jobs.v[w].m.n;
  *njobs = jobs.n;
  *total_entries = tot;
  if (sizes) {
    int64_t off = 0;
    for (int64_t w = 0; w < jobs.n && !e; w++) {
      int m = jobs.v[w].m.n;
      sizes[w] = m;
      memcpy(mats + off, jobs.v[w].m.a, sizeof(int64_t) * (size_t)m * m);
      off += (int64_t)m * m;
      int nl, sg;
      e = bi_export(&jobs.v[w].coef, coef_limbs + w * coef_cap, coef_cap, &nl, &sg);
      coef_sign[w] = sg;
    }
  }
  jl_free(&jobs);
  return e;
}

/* per(job) for each of count dense jobs (row-major, back to back), by H_per
 * with leaf cut-off L, nthreads workers.  Results as limbs per job
 * (cap limbs each), with nlimbs[w] and sign[w]. */
int oracle_job_permanents(int64_t count, const int32_t* sizes, const int64_t* mats, int L, int three,
                          int nthreads, uint32_t* limbs, int cap, int32_t* nlimbs,
                          int32_t* sign) {
  joblist jobs = {0};
  int e = 0;
  int64_t off = 0;
  for (int64_t w = 0; w < count; w++) {
    job_t j;
    int m = sizes[w];
    if (m < 0 || m > MAXN) { jl_free(&jobs); return ORACLE_EINVAL; }
    if ((e = mat_alloc(&j.m, m))) { jl_free(&jobs); return e; }
    memcpy(j.m.a, mats + off, sizeof(int64_t) * (size_t)m * m);
    off += (int64_t)m * m;
    bi_from_i64(&j.coef, 1);
    if ((e = jl_push(&jobs, &j))) { jl_free(&jobs); return e; }
  }
  bigint* pj = (bigint*)calloc((size_t)(count > 0 ? count : 1), sizeof(bigint));
  if (!pj) { jl_free(&jobs); return ORACLE_ENOMEM; }
  e = eval_jobs(&jobs, L, three, nthreads, pj);
  for (int64_t w = 0; !e && w < count; w++) {
    int nl, sg;
    e = bi_export(&pj[w], limbs + w * cap, cap, &nl, &sg);
    nlimbs[w] = nl;
    sign[w] = sg;
  }
  free(pj);
  jl_free(&jobs);
  return e;
}
