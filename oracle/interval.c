/*
 * interval.c -- the per-cell run rule computed over interval maps, on any
 * number of host threads.
 *
 * TEST INFRASTRUCTURE ONLY (like oracle.c): used by the tests, to check the
 * CUDA path on traces too large for the per-cell oracle, and by the timed CPU
 * baseline of the benchmark. Nothing in the product path links or calls it.
 * It shares no code, header or table with the CUDA sources, and none with
 * oracle.c either: it restates the same rule independently, and the tests pin
 * it to oracle.c (equal edge sets on every trace both can run) and to the
 * pairwise brute force.
 *
 * What it computes: exactly orc_analyze's edge set (Section 2.2: dependences
 * inferred from the data tasks use; Section 5):
 *   (O1) a task's rectangles on one cell combine into one privilege:
 *        read+read = read, reduce+reduce = reduce, any other mix = write;
 *   (O2) per cell, in program order, a write is a run of its own, consecutive
 *        reads form one run, consecutive reduces form one run; a task joining
 *        a read/reduce run gets an edge from every member of the run before
 *        it, a task starting a new run gets an edge from every member of the
 *        current run;
 *   (O4) explicit predecessors add their edges as given.
 *
 * How: cells are independent, so every row of the domain (every column range
 * of a 1-D domain) can be swept alone. Along a row, neighbouring cells with
 * the same history hold the same run state, so the row is kept as a sorted
 * list of segments [x0, next x0), each holding one state: the kind of the
 * current run, its members and the members of the run before it. A task's
 * rectangles on a row are cut into pieces of one combined privilege (O1) and
 * every segment a piece covers takes the O2 step; neighbours left with equal
 * states merge. Run member lists are immutable, newest member first, and
 * shared between segments by reference counting, so splitting a segment copies
 * two pointers. A write run keeps no previous run (nothing ever reads it),
 * which lets the segments one write covers merge into one.
 *
 * Threads own chunks of rows (of columns in 1-D) and walk every launch in
 * program order over their chunk; a per-thread stamp keeps a thread from
 * emitting one (src, dst) twice, and the union of the threads' pairs is
 * deduplicated into the canonical CSR (rows by source, columns ascending).
 */
#include <pthread.h>
#include <stdatomic.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define K_READ 0
#define K_WRITE 1
#define K_REDUCE 2
#define K_NONE 3

/* ------------------------------------------------------------------ */
/* run member lists: immutable, newest first, reference counted        */
/* ------------------------------------------------------------------ */
typedef struct mnode {
  int32_t task;
  int32_t refs;
  struct mnode* next;
} mnode;

typedef struct {
  mnode* free_list;
  mnode** blocks;
  int64_t nblocks, capblocks;
  int failed;
} mpool;

static mnode* mp_get(mpool* p) {
  if (!p->free_list) {
    const int64_t per = 1 << 16;
    mnode* blk = (mnode*)malloc((size_t)per * sizeof(mnode));
    if (!blk) {
      p->failed = 1;
      return NULL;
    }
    if (p->nblocks == p->capblocks) {
      int64_t nc = p->capblocks ? p->capblocks * 2 : 64;
      mnode** nb = (mnode**)realloc(p->blocks, (size_t)nc * sizeof(mnode*));
      if (!nb) {
        free(blk);
        p->failed = 1;
        return NULL;
      }
      p->blocks = nb;
      p->capblocks = nc;
    }
    p->blocks[p->nblocks++] = blk;
    for (int64_t k = 0; k < per; ++k) {
      blk[k].next = p->free_list;
      p->free_list = &blk[k];
    }
  }
  mnode* m = p->free_list;
  p->free_list = m->next;
  return m;
}

static void mp_free_all(mpool* p) {
  for (int64_t k = 0; k < p->nblocks; ++k) free(p->blocks[k]);
  free(p->blocks);
  memset(p, 0, sizeof(*p));
}

static void m_ref(mnode* m) {
  if (m) m->refs++;
}

static void m_unref(mpool* p, mnode* m) {
  while (m && --m->refs == 0) {
    mnode* nx = m->next;
    m->next = p->free_list;
    p->free_list = m;
    m = nx;
  }
}

/* a new list: task in front of `rest` (takes a reference on rest) */
static mnode* m_cons(mpool* p, int32_t task, mnode* rest) {
  mnode* m = mp_get(p);
  if (!m) return NULL;
  m->task = task;
  m->refs = 1;
  m->next = rest;
  m_ref(rest);
  return m;
}

/* ------------------------------------------------------------------ */
/* one row as sorted segments                                          */
/* ------------------------------------------------------------------ */
typedef struct {
  int64_t x0;   /* first cell of the segment; it ends where the next begins */
  int32_t kind; /* kind of the current run, K_NONE before any access */
  mnode* cur;   /* members of the current run */
  mnode* prev;  /* members of the run before it (NULL for a write run) */
} seg_t;

typedef struct {
  seg_t* s;
  int32_t n, cap;
} row_t;

static int row_reserve(row_t* r, int32_t need) {
  if (need <= r->cap) return 0;
  int32_t nc = r->cap ? r->cap : 8;
  while (nc < need) nc *= 2;
  seg_t* ns = (seg_t*)realloc(r->s, (size_t)nc * sizeof(seg_t));
  if (!ns) return -1;
  r->s = ns;
  r->cap = nc;
  return 0;
}

/* index of the segment holding cell x (x >= r->s[0].x0) */
static int32_t row_find(const row_t* r, int64_t x) {
  int32_t lo = 0, hi = r->n - 1;
  while (lo < hi) {
    int32_t mid = (lo + hi + 1) >> 1;
    if (r->s[mid].x0 <= x) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

/* makes x the first cell of a segment; returns its index, -1 on failure */
static int32_t row_split(row_t* r, int64_t x) {
  int32_t i = row_find(r, x);
  if (r->s[i].x0 == x) return i;
  if (row_reserve(r, r->n + 1)) return -1;
  memmove(&r->s[i + 2], &r->s[i + 1], (size_t)(r->n - i - 1) * sizeof(seg_t));
  r->s[i + 1] = r->s[i];
  r->s[i + 1].x0 = x;
  m_ref(r->s[i + 1].cur);
  m_ref(r->s[i + 1].prev);
  r->n++;
  return i + 1;
}

/* ------------------------------------------------------------------ */
/* per-thread work                                                     */
/* ------------------------------------------------------------------ */
typedef struct {
  uint64_t* v;
  int64_t n, cap;
} pairs_t;

static int pairs_push(pairs_t* a, uint64_t x) {
  if (a->n == a->cap) {
    int64_t nc = a->cap ? a->cap * 2 : 1 << 16;
    uint64_t* nv = (uint64_t*)realloc(a->v, (size_t)nc * sizeof(uint64_t));
    if (!nv) return -1;
    a->v = nv;
    a->cap = nc;
  }
  a->v[a->n++] = x;
  return 0;
}

typedef struct {
  /* the launches */
  int32_t ndim, n;
  int64_t dlo[2], ext[2];
  const int32_t* req_off;
  const int64_t* lo;
  const int64_t* hi;
  const uint8_t* priv;
  /* chunks: rows [c*rows_per, ...) in 2-D, columns in 1-D */
  int64_t nchunks, per_chunk;
  atomic_llong next_chunk;
  atomic_int failed;
} job_t;

typedef struct {
  job_t* job;
  pairs_t out;
  int32_t* stamp; /* stamp[src] == dst: (src, dst) already emitted by this thread */
  mpool pool;
  /* scratch for one task's pieces */
  int64_t* ybnd;
  int64_t* xbnd;
  int32_t* cover;
  int64_t* piece_l;
  int64_t* piece_r;
  int32_t* piece_p;
  int32_t scratch_cap;
  pthread_t tid;
} worker_t;

static int emit_list(worker_t* w, const mnode* m, int32_t j) {
  for (; m; m = m->next) {
    if (w->stamp[m->task] != j) {
      w->stamp[m->task] = j;
      if (pairs_push(&w->out, ((uint64_t)(uint32_t)m->task << 32) | (uint32_t)j)) return -1;
    }
  }
  return 0;
}

static int same_state(const seg_t* a, const seg_t* b) {
  return a->kind == b->kind && a->cur == b->cur && a->prev == b->prev;
}

/* task j accesses cells [l, r] of row `row` with privilege p (after O1) */
static int row_apply(worker_t* w, row_t* row, int64_t l, int64_t r, int32_t p, int32_t j, int64_t row_end) {
  mpool* pool = &w->pool;
  int32_t i0 = row_split(row, l);
  if (i0 < 0) return -1;
  if (r + 1 <= row_end && row_split(row, r + 1) < 0) return -1;
  int32_t i1 = i0;
  while (i1 < row->n && row->s[i1].x0 <= r) ++i1; /* segments [i0, i1) are covered */
  mnode* solo = NULL;                           /* the one-member run {j}, shared */
  mnode* memo_in = NULL;                        /* last joined run and its extension */
  mnode* memo_out = NULL;
  for (int32_t i = i0; i < i1; ++i) {
    seg_t* s = &row->s[i];
    if (s->cur && s->kind == p && p != K_WRITE) {
      /* j joins the current run: edges from the run before it */
      if (emit_list(w, s->prev, j)) return -1;
      mnode* ext;
      if (memo_in == s->cur && memo_out) {
        ext = memo_out;
        m_ref(ext);
      } else {
        ext = m_cons(pool, j, s->cur);
        if (!ext) return -1;
        memo_in = s->cur;
        memo_out = ext;
      }
      m_unref(pool, s->cur);
      s->cur = ext;
    } else {
      /* j starts a new run: edges from every member of the current run */
      if (emit_list(w, s->cur, j)) return -1;
      if (!solo) {
        solo = m_cons(pool, j, NULL);
        if (!solo) return -1;
      } else {
        m_ref(solo);
      }
      m_unref(pool, s->prev);
      if (p == K_WRITE) {
        m_unref(pool, s->cur);
        s->prev = NULL;
      } else {
        s->prev = s->cur;
      }
      s->cur = solo;
      s->kind = p;
    }
  }
  /* merge equal neighbours from the segment before the range to the one after */
  int32_t a = i0 > 0 ? i0 - 1 : 0;
  int32_t b = i1 < row->n ? i1 : row->n - 1;
  int32_t k = a;
  for (int32_t i = a + 1; i <= b; ++i) {
    if (same_state(&row->s[k], &row->s[i])) {
      m_unref(pool, row->s[i].cur);
      m_unref(pool, row->s[i].prev);
    } else {
      row->s[++k] = row->s[i];
    }
  }
  int32_t removed = b - k;
  if (removed > 0) {
    memmove(&row->s[k + 1], &row->s[b + 1], (size_t)(row->n - b - 1) * sizeof(seg_t));
    row->n -= removed;
  }
  return 0;
}

static int grow_scratch(worker_t* w, int32_t nr) {
  if (nr <= w->scratch_cap) return 0;
  int32_t c = nr * 2 + 2;
  free(w->ybnd);
  free(w->xbnd);
  free(w->cover);
  free(w->piece_l);
  free(w->piece_r);
  free(w->piece_p);
  w->ybnd = (int64_t*)malloc((size_t)c * sizeof(int64_t));
  w->xbnd = (int64_t*)malloc((size_t)c * sizeof(int64_t));
  w->cover = (int32_t*)malloc((size_t)c * sizeof(int32_t));
  w->piece_l = (int64_t*)malloc((size_t)c * sizeof(int64_t));
  w->piece_r = (int64_t*)malloc((size_t)c * sizeof(int64_t));
  w->piece_p = (int32_t*)malloc((size_t)c * sizeof(int32_t));
  w->scratch_cap = nr;
  return (w->ybnd && w->xbnd && w->cover && w->piece_l && w->piece_r && w->piece_p) ? 0 : -1;
}

static int cmp_i64(const void* a, const void* b) {
  int64_t x = *(const int64_t*)a, y = *(const int64_t*)b;
  return x < y ? -1 : (x > y ? 1 : 0);
}

static int64_t sort_unique(int64_t* a, int64_t n) {
  qsort(a, (size_t)n, sizeof(int64_t), cmp_i64);
  int64_t m = 0;
  for (int64_t k = 0; k < n; ++k)
    if (k == 0 || a[k] != a[m - 1]) a[m++] = a[k];
  return m;
}

/* O1 on one task's rectangles: a rectangle's privilege combined into a cell's */
static int32_t combine(int32_t have, int32_t add) {
  if (have == K_NONE) return add;
  if (have == add && add != K_WRITE) return add;
  return K_WRITE;
}

/* sweeps rows [ya, yb] x columns [xa, xb] (domain-relative) over all launches */
static int sweep_chunk(worker_t* w, int64_t ya, int64_t yb, int64_t xa, int64_t xb) {
  job_t* J = w->job;
  const int D = J->ndim;
  int64_t nrows = yb - ya + 1;
  row_t* rows = (row_t*)calloc((size_t)nrows, sizeof(row_t));
  if (!rows) return -1;
  int rc = 0;
  for (int64_t y = 0; y < nrows && !rc; ++y) {
    if (row_reserve(&rows[y], 8)) rc = -1;
    else {
      rows[y].n = 1;
      rows[y].s[0].x0 = xa;
      rows[y].s[0].kind = K_NONE;
      rows[y].s[0].cur = rows[y].s[0].prev = NULL;
    }
  }
  for (int32_t j = 0; j < J->n && !rc; ++j) {
    const int32_t r0 = J->req_off[j], r1 = J->req_off[j + 1];
    if (r1 == r0) continue;
    if (grow_scratch(w, r1 - r0)) {
      rc = -1;
      break;
    }
    /* the task's rectangles clipped to the chunk: row bands of one cover set */
    int32_t nb = 0;
    for (int32_t q = r0; q < r1; ++q) {
      int64_t x0 = J->lo[(int64_t)q * D] - J->dlo[0], x1 = J->hi[(int64_t)q * D] - J->dlo[0];
      int64_t y0 = D == 2 ? J->lo[(int64_t)q * 2 + 1] - J->dlo[1] : 0;
      int64_t y1 = D == 2 ? J->hi[(int64_t)q * 2 + 1] - J->dlo[1] : 0;
      if (x1 < xa || x0 > xb || y1 < ya || y0 > yb) continue;
      w->ybnd[nb++] = y0 < ya ? ya : y0;
      w->ybnd[nb++] = (y1 > yb ? yb : y1) + 1;
    }
    if (nb == 0) continue;
    nb = (int32_t)sort_unique(w->ybnd, nb);
    for (int32_t bk = 0; bk + 1 < nb && !rc; ++bk) {
      const int64_t by0 = w->ybnd[bk], by1 = w->ybnd[bk + 1] - 1;
      /* rectangles covering this band, and their x boundaries */
      int32_t nc = 0, nx = 0;
      for (int32_t q = r0; q < r1; ++q) {
        int64_t x0 = J->lo[(int64_t)q * D] - J->dlo[0], x1 = J->hi[(int64_t)q * D] - J->dlo[0];
        int64_t y0 = D == 2 ? J->lo[(int64_t)q * 2 + 1] - J->dlo[1] : 0;
        int64_t y1 = D == 2 ? J->hi[(int64_t)q * 2 + 1] - J->dlo[1] : 0;
        if (x1 < xa || x0 > xb || y0 > by0 || y1 < by0) continue;
        w->cover[nc++] = q;
        w->xbnd[nx++] = x0 < xa ? xa : x0;
        w->xbnd[nx++] = (x1 > xb ? xb : x1) + 1;
      }
      if (nc == 0) continue;
      nx = (int32_t)sort_unique(w->xbnd, nx);
      /* pieces of one combined privilege (O1) */
      int32_t np = 0;
      for (int32_t e = 0; e + 1 < nx; ++e) {
        const int64_t l = w->xbnd[e], r = w->xbnd[e + 1] - 1;
        int32_t p = K_NONE;
        for (int32_t c = 0; c < nc; ++c) {
          const int32_t q = w->cover[c];
          int64_t x0 = J->lo[(int64_t)q * D] - J->dlo[0], x1 = J->hi[(int64_t)q * D] - J->dlo[0];
          if (x0 <= l && r <= x1) p = combine(p, (int32_t)J->priv[q]);
        }
        if (p == K_NONE) continue;
        w->piece_l[np] = l;
        w->piece_r[np] = r;
        w->piece_p[np] = p;
        ++np;
      }
      for (int64_t y = by0; y <= by1 && !rc; ++y)
        for (int32_t k = 0; k < np && !rc; ++k)
          rc = row_apply(w, &rows[y - ya], w->piece_l[k], w->piece_r[k], w->piece_p[k], j, xb);
    }
  }
  for (int64_t y = 0; y < nrows; ++y) {
    for (int32_t i = 0; i < rows[y].n; ++i) {
      m_unref(&w->pool, rows[y].s[i].cur);
      m_unref(&w->pool, rows[y].s[i].prev);
    }
    free(rows[y].s);
  }
  free(rows);
  if (w->pool.failed) rc = -1;
  return rc;
}

static void* worker_main(void* arg) {
  worker_t* w = (worker_t*)arg;
  job_t* J = w->job;
  for (;;) {
    if (atomic_load(&J->failed)) break;
    long long c = atomic_fetch_add(&J->next_chunk, 1);
    if (c >= J->nchunks) break;
    int64_t a = (int64_t)c * J->per_chunk;
    int rc;
    if (J->ndim == 2) {
      int64_t b = a + J->per_chunk - 1;
      if (b > J->ext[1] - 1) b = J->ext[1] - 1;
      rc = sweep_chunk(w, a, b, 0, J->ext[0] - 1);
    } else {
      int64_t b = a + J->per_chunk - 1;
      if (b > J->ext[0] - 1) b = J->ext[0] - 1;
      rc = sweep_chunk(w, 0, 0, a, b);
    }
    if (rc) atomic_store(&J->failed, 1);
  }
  return NULL;
}

/* ------------------------------------------------------------------ */
/* result: canonical CSR                                               */
/* ------------------------------------------------------------------ */
typedef struct {
  int32_t n;
  int64_t n_edges;
  int64_t* row_ptr;
  int32_t* col;
} b3_result;

static int cmp_i32(const void* a, const void* b) {
  int32_t x = *(const int32_t*)a, y = *(const int32_t*)b;
  return x < y ? -1 : (x > y ? 1 : 0);
}

typedef struct {
  int32_t v0, v1;
  int64_t* cnt_off;  /* bucket offsets (with duplicates) */
  int32_t* bucket;
  int64_t* uniq;     /* per row: distinct count */
  pthread_t tid;
} rowsort_t;

static void* rowsort_main(void* arg) {
  rowsort_t* t = (rowsort_t*)arg;
  for (int32_t v = t->v0; v < t->v1; ++v) {
    int32_t* b = t->bucket + t->cnt_off[v];
    int64_t m = t->cnt_off[v + 1] - t->cnt_off[v];
    if (m > 1) qsort(b, (size_t)m, sizeof(int32_t), cmp_i32);
    int64_t u = 0;
    for (int64_t k = 0; k < m; ++k)
      if (k == 0 || b[k] != b[u - 1]) b[u++] = b[k];
    t->uniq[v] = u;
  }
  return NULL;
}

/* Returns a handle (NULL on allocation failure). threads <= 0: one thread. */
void* orc_b3_analyze(int32_t ndim, const int64_t* dom_lo, const int64_t* dom_hi, int32_t n,
                     const int32_t* req_off, const int64_t* lo, const int64_t* hi, const uint8_t* priv,
                     const int32_t* pred_off, const int32_t* pred, int32_t threads) {
  if (threads < 1) threads = 1;
  job_t J;
  memset(&J, 0, sizeof(J));
  J.ndim = ndim;
  J.n = n;
  J.dlo[0] = dom_lo[0];
  J.ext[0] = dom_hi[0] - dom_lo[0] + 1;
  J.dlo[1] = ndim == 2 ? dom_lo[1] : 0;
  J.ext[1] = ndim == 2 ? dom_hi[1] - dom_lo[1] + 1 : 1;
  J.req_off = req_off;
  J.lo = lo;
  J.hi = hi;
  J.priv = priv;
  const int64_t span = ndim == 2 ? J.ext[1] : J.ext[0];
  int64_t want = (int64_t)threads * 4;
  J.per_chunk = (span + want - 1) / want;
  if (J.per_chunk < 1) J.per_chunk = 1;
  J.nchunks = (span + J.per_chunk - 1) / J.per_chunk;
  if (n == 0 || req_off[n] == 0) J.nchunks = 0;
  atomic_init(&J.next_chunk, 0);
  atomic_init(&J.failed, 0);

  worker_t* W = (worker_t*)calloc((size_t)threads, sizeof(worker_t));
  b3_result* res = (b3_result*)calloc(1, sizeof(b3_result));
  int64_t* deg = (int64_t*)calloc((size_t)n + 1, sizeof(int64_t));
  int32_t* bucket = NULL;
  rowsort_t* RS = NULL;
  int ok = W && res && deg;
  for (int t = 0; ok && t < threads; ++t) {
    W[t].job = &J;
    W[t].stamp = (int32_t*)malloc((size_t)(n ? n : 1) * sizeof(int32_t));
    if (!W[t].stamp) ok = 0;
    else
      for (int32_t v = 0; v < n; ++v) W[t].stamp[v] = -1;
  }
  int started = 0;
  if (ok) {
    for (int t = 1; t < threads; ++t) {
      if (pthread_create(&W[t].tid, NULL, worker_main, &W[t])) {
        atomic_store(&J.failed, 1);
        break;
      }
      started = t;
    }
    worker_main(&W[0]);
    for (int t = 1; t <= started; ++t) pthread_join(W[t].tid, NULL);
    if (atomic_load(&J.failed)) ok = 0;
  }
  /* O4: explicit predecessors */
  pairs_t expl = {0, 0, 0};
  if (ok && pred_off) {
    for (int32_t j = 0; ok && j < n; ++j)
      for (int32_t k = pred_off[j]; k < pred_off[j + 1]; ++k)
        if (pairs_push(&expl, ((uint64_t)(uint32_t)pred[k] << 32) | (uint32_t)j)) {
          ok = 0;
          break;
        }
  }
  /* bucket every pair by source, then sort and deduplicate each row */
  int64_t total = 0;
  if (ok) {
    for (int t = 0; t < threads; ++t)
      for (int64_t k = 0; k < W[t].out.n; ++k) deg[(W[t].out.v[k] >> 32) + 1]++;
    for (int64_t k = 0; k < expl.n; ++k) deg[(expl.v[k] >> 32) + 1]++;
    for (int32_t v = 0; v < n; ++v) deg[v + 1] += deg[v];
    total = deg[n];
    bucket = (int32_t*)malloc((size_t)(total ? total : 1) * sizeof(int32_t));
    res->row_ptr = (int64_t*)malloc(((size_t)n + 1) * sizeof(int64_t));
    if (!bucket || !res->row_ptr) ok = 0;
  }
  if (ok) {
    int64_t* fill = res->row_ptr; /* scratch cursor, rewritten below */
    memcpy(fill, deg, ((size_t)n + 1) * sizeof(int64_t));
    for (int t = 0; t < threads; ++t)
      for (int64_t k = 0; k < W[t].out.n; ++k) {
        uint64_t x = W[t].out.v[k];
        bucket[fill[x >> 32]++] = (int32_t)(x & 0xffffffffu);
      }
    for (int64_t k = 0; k < expl.n; ++k) {
      uint64_t x = expl.v[k];
      bucket[fill[x >> 32]++] = (int32_t)(x & 0xffffffffu);
    }
    for (int t = 0; t < threads; ++t) {
      free(W[t].out.v);
      W[t].out.v = NULL;
    }
    int64_t* uniq = (int64_t*)malloc((size_t)(n ? n : 1) * sizeof(int64_t));
    RS = (rowsort_t*)calloc((size_t)threads, sizeof(rowsort_t));
    if (!uniq || !RS) {
      free(uniq);
      ok = 0;
    } else {
      int32_t per = (n + threads - 1) / threads;
      int nst = 0;
      for (int t = 0; t < threads; ++t) {
        RS[t].v0 = t * per < n ? t * per : n;
        RS[t].v1 = (t + 1) * per < n ? (t + 1) * per : n;
        RS[t].cnt_off = deg;
        RS[t].bucket = bucket;
        RS[t].uniq = uniq;
      }
      for (int t = 1; t < threads; ++t) {
        if (pthread_create(&RS[t].tid, NULL, rowsort_main, &RS[t])) break;
        nst = t;
      }
      for (int t = nst + 1; t < threads; ++t) rowsort_main(&RS[t]);
      rowsort_main(&RS[0]);
      for (int t = 1; t <= nst; ++t) pthread_join(RS[t].tid, NULL);
      res->row_ptr[0] = 0;
      for (int32_t v = 0; v < n; ++v) res->row_ptr[v + 1] = res->row_ptr[v] + uniq[v];
      res->n_edges = res->row_ptr[n];
      res->col = (int32_t*)malloc((size_t)(res->n_edges ? res->n_edges : 1) * sizeof(int32_t));
      if (!res->col) ok = 0;
      else
        for (int32_t v = 0; v < n; ++v)
          memcpy(res->col + res->row_ptr[v], bucket + deg[v], (size_t)uniq[v] * sizeof(int32_t));
      res->n = n;
      free(uniq);
    }
  }
  if (W)
    for (int t = 0; t < threads; ++t) {
      free(W[t].out.v);
      free(W[t].stamp);
      free(W[t].ybnd);
      free(W[t].xbnd);
      free(W[t].cover);
      free(W[t].piece_l);
      free(W[t].piece_r);
      free(W[t].piece_p);
      mp_free_all(&W[t].pool);
    }
  free(W);
  free(expl.v);
  free(deg);
  free(bucket);
  free(RS);
  if (!ok) {
    if (res) {
      free(res->row_ptr);
      free(res->col);
      free(res);
    }
    return NULL;
  }
  return res;
}

int64_t orc_b3_edges(void* h) { return ((b3_result*)h)->n_edges; }

void orc_b3_copy(void* h, int64_t* row_ptr, int32_t* col) {
  b3_result* r = (b3_result*)h;
  memcpy(row_ptr, r->row_ptr, ((size_t)r->n + 1) * sizeof(int64_t));
  memcpy(col, r->col, (size_t)r->n_edges * sizeof(int32_t));
}

void orc_b3_free(void* h) {
  b3_result* r = (b3_result*)h;
  if (!r) return;
  free(r->row_ptr);
  free(r->col);
  free(r);
}
