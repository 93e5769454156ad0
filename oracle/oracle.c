/*
 * oracle.c -- plain, slow, obviously-correct CPU oracle.
 *
 * TEST INFRASTRUCTURE ONLY. Nothing in the product path may link or call this
 * file: it exists so that tests, the smoke check and the timed CPU baseline of
 * the benchmark can compare the CUDA path against an independent
 * implementation. It shares no code, header, table or helper with the CUDA
 * sources.
 *
 * What it computes (all integer work, so results are exact):
 *
 *  orc_analyze    implicit dependence analysis over a program-ordered stream
 *                 of task launches with region requirements (Section 2.2's
 *                 "tasks describe what data they will access, and then the
 *                 system performs an analysis to discover the necessary
 *                 dependencies", Section 5). The paper does not define the
 *                 edge rule; this file follows the per-cell run reading:
 *                 (O1) a task's several rectangles on one cell combine into one
 *                      privilege: read+read = read, reduce+reduce = reduce,
 *                      anything else = write;
 *                 (O2) per cell, accesses in program order form runs (a write
 *                      is a run of its own, consecutive reads form one run,
 *                      consecutive reduces form one run); every member of a run
 *                      gets an edge from every member of the run before it;
 *                 (O4) explicit predecessor lists (Fig. 3's launch(..., pre))
 *                      add their edges as given.
 *                 Edges are deduplicated; the canonical form is CSR by source,
 *                 columns ascending.
 *  orc_topo_order Kahn's algorithm with the smallest ready id first: one
 *                 order that Algorithm 1's interpreter may produce (INIT seeds
 *                 every node without incoming edges, COMPLETED_EDGE releases a
 *                 node when its last incoming edge is removed).
 *  orc_run        executes the task bodies in a given order (NULL = program
 *                 order, i.e. sequential semantics): EMPTY, SPIN (integer
 *                 LCG), FMA (Section 6's floating-point task loop), COUNTER
 *                 and the order-sensitive CHECK.
 *
 * Parity: O1/O2 themselves are a reading of the paper, pinned by brute force
 * (pairwise run-boundary count, interference soundness and completeness) and
 * closed forms in the tests; the executor is pinned by the paper's Fig. 6(c)
 * four-task DAG and by "execution in any topological order equals program
 * order" properties.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define P_READ 0
#define P_WRITE 1
#define P_REDUCE 2
#define P_NONE 255

/* ------------------------------------------------------------------ */
/* growable arrays                                                     */
/* ------------------------------------------------------------------ */
typedef struct {
  uint64_t* v;
  int64_t n, cap;
} vec64;

static int vec64_push(vec64* a, uint64_t x) {
  if (a->n == a->cap) {
    int64_t nc = a->cap ? a->cap * 2 : 1024;
    uint64_t* nv = (uint64_t*)realloc(a->v, (size_t)nc * sizeof(uint64_t));
    if (!nv) return -1;
    a->v = nv;
    a->cap = nc;
  }
  a->v[a->n++] = x;
  return 0;
}

typedef struct {
  uint8_t kind;
  int32_t n, cap;
  int32_t* m; /* member task ids, in program order */
} run_t;

static int run_push(run_t* r, int32_t task) {
  if (r->n == r->cap) {
    int32_t nc = r->cap ? r->cap * 2 : 4;
    int32_t* nm = (int32_t*)realloc(r->m, (size_t)nc * sizeof(int32_t));
    if (!nm) return -1;
    r->m = nm;
    r->cap = nc;
  }
  r->m[r->n++] = task;
  return 0;
}

/* O1: privilege of one task on one cell after combining its rectangles. */
static uint8_t orc_combine(uint8_t have, uint8_t add) {
  if (have == P_NONE) return add;
  if (have == add && add != P_WRITE) return add; /* read+read, reduce+reduce */
  return P_WRITE;                                 /* every other mix */
}

/* ------------------------------------------------------------------ */
/* domain geometry                                                     */
/* ------------------------------------------------------------------ */
typedef struct {
  int ndim;
  int64_t lo[2], ext[2];
  int64_t ncells;
} dom_t;

static void dom_init(dom_t* d, int ndim, const int64_t* lo, const int64_t* hi) {
  d->ndim = ndim;
  d->lo[0] = lo[0];
  d->ext[0] = hi[0] - lo[0] + 1;
  d->lo[1] = ndim == 2 ? lo[1] : 0;
  d->ext[1] = ndim == 2 ? hi[1] - lo[1] + 1 : 1;
  d->ncells = d->ext[0] * d->ext[1];
}

/* Collects the cells task j touches with their combined privilege (O1).
 * stamp[c] == j marks a cell already seen for this task. */
static int gather_task_cells(const dom_t* d, int32_t j, const int32_t* req_off, const int64_t* lo,
                             const int64_t* hi, const uint8_t* priv, int32_t* stamp,
                             uint8_t* comb, int64_t** cells, int64_t* ncells, int64_t* capcells) {
  *ncells = 0;
  for (int32_t r = req_off[j]; r < req_off[j + 1]; ++r) {
    int64_t x0 = lo[(int64_t)r * d->ndim] - d->lo[0];
    int64_t x1 = hi[(int64_t)r * d->ndim] - d->lo[0];
    int64_t y0 = 0, y1 = 0;
    if (d->ndim == 2) {
      y0 = lo[(int64_t)r * 2 + 1] - d->lo[1];
      y1 = hi[(int64_t)r * 2 + 1] - d->lo[1];
    }
    for (int64_t y = y0; y <= y1; ++y) {
      for (int64_t x = x0; x <= x1; ++x) {
        int64_t c = y * d->ext[0] + x;
        if (stamp[c] != j) {
          stamp[c] = j;
          comb[c] = priv[r];
          if (*ncells == *capcells) {
            int64_t nc = *capcells ? *capcells * 2 : 4096;
            int64_t* nv = (int64_t*)realloc(*cells, (size_t)nc * sizeof(int64_t));
            if (!nv) return -1;
            *cells = nv;
            *capcells = nc;
          }
          (*cells)[(*ncells)++] = c;
        } else {
          comb[c] = orc_combine(comb[c], priv[r]);
        }
      }
    }
  }
  return 0;
}

static int cmp_u64(const void* a, const void* b) {
  uint64_t x = *(const uint64_t*)a, y = *(const uint64_t*)b;
  return x < y ? -1 : (x > y ? 1 : 0);
}

/* ------------------------------------------------------------------ */
/* dependence analysis                                                 */
/* ------------------------------------------------------------------ */
typedef struct {
  int64_t n_edges;
  int32_t* src;
  int32_t* dst;
} orc_result;

/* Returns NULL on allocation failure. pred_off/pred may be NULL. */
void* orc_analyze(int32_t ndim, const int64_t* dom_lo, const int64_t* dom_hi, int32_t n,
                  const int32_t* req_off, const int64_t* lo, const int64_t* hi,
                  const uint8_t* priv, const int32_t* pred_off, const int32_t* pred) {
  dom_t d;
  dom_init(&d, ndim, dom_lo, dom_hi);
  int has_rects = n > 0 && req_off[n] > 0;
  int64_t nc = has_rects ? d.ncells : 0;
  run_t* last = (run_t*)calloc((size_t)(nc ? nc : 1), sizeof(run_t));
  run_t* prev = (run_t*)calloc((size_t)(nc ? nc : 1), sizeof(run_t));
  int32_t* stamp = (int32_t*)malloc((size_t)(nc ? nc : 1) * sizeof(int32_t));
  uint8_t* comb = (uint8_t*)malloc((size_t)(nc ? nc : 1));
  vec64 pairs = {0, 0, 0};
  int64_t* cells = NULL;
  int64_t ncell = 0, capcell = 0;
  orc_result* res = (orc_result*)calloc(1, sizeof(orc_result));
  if (!last || !prev || !stamp || !comb || !res) goto fail;
  for (int64_t c = 0; c < nc; ++c) stamp[c] = -1;

  for (int32_t j = 0; j < n; ++j) {
    /* O4: explicit predecessors */
    if (pred_off) {
      for (int32_t k = pred_off[j]; k < pred_off[j + 1]; ++k)
        if (vec64_push(&pairs, ((uint64_t)(uint32_t)pred[k] << 32) | (uint32_t)j)) goto fail;
    }
    if (!has_rects) continue;
    /* O1 */
    if (gather_task_cells(&d, j, req_off, lo, hi, priv, stamp, comb, &cells, &ncell, &capcell))
      goto fail;
    /* O2: per-cell runs */
    for (int64_t q = 0; q < ncell; ++q) {
      int64_t c = cells[q];
      uint8_t p = comb[c];
      run_t* L = &last[c];
      run_t* P = &prev[c];
      if (L->n > 0 && L->kind == p && p != P_WRITE) {
        /* j joins the current run: edges from the run before it */
        for (int32_t k = 0; k < P->n; ++k)
          if (vec64_push(&pairs, ((uint64_t)(uint32_t)P->m[k] << 32) | (uint32_t)j)) goto fail;
        if (run_push(L, j)) goto fail;
      } else {
        /* j starts a new run: edges from every member of the current run */
        for (int32_t k = 0; k < L->n; ++k)
          if (vec64_push(&pairs, ((uint64_t)(uint32_t)L->m[k] << 32) | (uint32_t)j)) goto fail;
        run_t tmp = *P; /* the old previous run's storage is recycled */
        *P = *L;
        *L = tmp;
        L->n = 0;
        L->kind = p;
        if (run_push(L, j)) goto fail;
      }
    }
  }
  /* dedupe: sort (src, dst) keys and keep distinct ones */
  if (pairs.n) qsort(pairs.v, (size_t)pairs.n, sizeof(uint64_t), cmp_u64);
  int64_t e = 0;
  for (int64_t k = 0; k < pairs.n; ++k)
    if (k == 0 || pairs.v[k] != pairs.v[k - 1]) pairs.v[e++] = pairs.v[k];
  res->n_edges = e;
  res->src = (int32_t*)malloc((size_t)(e ? e : 1) * sizeof(int32_t));
  res->dst = (int32_t*)malloc((size_t)(e ? e : 1) * sizeof(int32_t));
  if (!res->src || !res->dst) goto fail;
  for (int64_t k = 0; k < e; ++k) {
    res->src[k] = (int32_t)(pairs.v[k] >> 32);
    res->dst[k] = (int32_t)(pairs.v[k] & 0xffffffffu);
  }
  for (int64_t c = 0; c < nc; ++c) {
    free(last[c].m);
    free(prev[c].m);
  }
  free(last);
  free(prev);
  free(stamp);
  free(comb);
  free(cells);
  free(pairs.v);
  return res;
fail:
  if (last && prev)
    for (int64_t c = 0; c < nc; ++c) {
      free(last[c].m);
      free(prev[c].m);
    }
  free(last);
  free(prev);
  free(stamp);
  free(comb);
  free(cells);
  free(pairs.v);
  if (res) {
    free(res->src);
    free(res->dst);
    free(res);
  }
  return NULL;
}

int64_t orc_result_edges(void* h) { return ((orc_result*)h)->n_edges; }

void orc_result_copy(void* h, int32_t* src, int32_t* dst) {
  orc_result* r = (orc_result*)h;
  memcpy(src, r->src, (size_t)r->n_edges * sizeof(int32_t));
  memcpy(dst, r->dst, (size_t)r->n_edges * sizeof(int32_t));
}

void orc_result_free(void* h) {
  orc_result* r = (orc_result*)h;
  if (!r) return;
  free(r->src);
  free(r->dst);
  free(r);
}

/* ------------------------------------------------------------------ */
/* Kahn's algorithm, smallest ready id first (binary min-heap)         */
/* ------------------------------------------------------------------ */
static void heap_push(int32_t* h, int64_t* n, int32_t x) {
  int64_t i = (*n)++;
  h[i] = x;
  while (i > 0) {
    int64_t p = (i - 1) / 2;
    if (h[p] <= h[i]) break;
    int32_t t = h[p];
    h[p] = h[i];
    h[i] = t;
    i = p;
  }
}

static int32_t heap_pop(int32_t* h, int64_t* n) {
  int32_t top = h[0];
  h[0] = h[--(*n)];
  int64_t i = 0;
  for (;;) {
    int64_t l = 2 * i + 1, r = l + 1, s = i;
    if (l < *n && h[l] < h[s]) s = l;
    if (r < *n && h[r] < h[s]) s = r;
    if (s == i) break;
    int32_t t = h[s];
    h[s] = h[i];
    h[i] = t;
    i = s;
  }
  return top;
}

/* Returns the number of tasks ordered (< n means the graph had a cycle). */
int64_t orc_topo_order(int32_t n, const int64_t* row_ptr, const int32_t* col, int32_t* order) {
  int32_t* cnt = (int32_t*)calloc((size_t)(n ? n : 1), sizeof(int32_t));
  int32_t* heap = (int32_t*)malloc((size_t)(n ? n : 1) * sizeof(int32_t));
  if (!cnt || !heap) {
    free(cnt);
    free(heap);
    return -1;
  }
  for (int64_t e = 0; e < row_ptr[n]; ++e) cnt[col[e]]++;
  int64_t hn = 0, k = 0;
  for (int32_t v = 0; v < n; ++v)
    if (cnt[v] == 0) heap_push(heap, &hn, v); /* INIT: every node without in-edges */
  while (hn > 0) {
    int32_t v = heap_pop(heap, &hn);
    order[k++] = v;
    for (int64_t e = row_ptr[v]; e < row_ptr[v + 1]; ++e)
      if (--cnt[col[e]] == 0) heap_push(heap, &hn, col[e]); /* last in-edge removed */
  }
  free(cnt);
  free(heap);
  return k;
}

/* ------------------------------------------------------------------ */
/* task bodies                                                         */
/* ------------------------------------------------------------------ */
#define BODY_EMPTY 0
#define BODY_SPIN 1
#define BODY_COUNTER 2
#define BODY_CHECK 3
#define BODY_FMA 4

/* murmur3's 32-bit finaliser */
static uint32_t orc_fmix32(uint32_t h) {
  h ^= h >> 16;
  h *= 0x85ebca6bu;
  h ^= h >> 13;
  h *= 0xc2b2ae35u;
  h ^= h >> 16;
  return h;
}

uint32_t orc_mix32(uint32_t a, uint32_t b) { return orc_fmix32(a ^ (b * 0x9E3779B1u)); }

uint32_t orc_spin(uint32_t x, int32_t iters) {
  for (int32_t k = 0; k < iters; ++k) x = x * 1664525u + 1013904223u;
  return x;
}

/* The floating-point loop of a compute-bound Task Bench kernel (Section 6):
 * x = (float)task, then `iters` fused multiply-adds x = x * 0.999f + 0.25f in
 * binary32, each rounded once to nearest even (C99 fmaf). Returns x's bits. */
uint32_t orc_fma(uint32_t task, int32_t iters) {
  float x = (float)task;
  for (int32_t k = 0; k < iters; ++k) x = fmaf(x, 0.999f, 0.25f);
  uint32_t bits;
  memcpy(&bits, &x, 4);
  return bits;
}

/* Runs the bodies of tasks order[0..count) (order == NULL: 0..n-1).
 * state: int32 per cell (CHECK) or per counter (COUNTER); out: int32 per task. */
int32_t orc_run(int32_t ndim, const int64_t* dom_lo, const int64_t* dom_hi, int32_t n,
                const int32_t* req_off, const int64_t* lo, const int64_t* hi, const uint8_t* priv,
                const int32_t* body_arg, int32_t body, int32_t spin_iters, int32_t* state,
                int32_t* out, const int32_t* order, int64_t count) {
  dom_t d;
  dom_init(&d, ndim, dom_lo, dom_hi);
  int32_t* stamp = NULL;
  uint8_t* comb = NULL;
  int64_t* cells = NULL;
  int64_t ncell = 0, capcell = 0;
  if (body == BODY_CHECK) {
    stamp = (int32_t*)malloc((size_t)d.ncells * sizeof(int32_t));
    comb = (uint8_t*)malloc((size_t)d.ncells);
    if (!stamp || !comb) {
      free(stamp);
      free(comb);
      return -1;
    }
    for (int64_t c = 0; c < d.ncells; ++c) stamp[c] = -1;
  }
  if (order == NULL) count = n;
  for (int64_t q = 0; q < count; ++q) {
    int32_t j = order ? order[q] : (int32_t)q;
    if (body == BODY_SPIN) {
      out[j] = (int32_t)orc_spin((uint32_t)j, spin_iters);
    } else if (body == BODY_FMA) {
      out[j] = (int32_t)orc_fma((uint32_t)j, spin_iters);
    } else if (body == BODY_COUNTER) {
      int32_t k = body_arg[j];
      state[k] = (int32_t)((uint32_t)state[k] + 1u);
    } else if (body == BODY_CHECK) {
      /* the task's stamp must be fresh even when a task runs twice (replays) */
      for (int64_t c = 0; c < ncell; ++c) stamp[cells[c]] = -1;
      if (gather_task_cells(&d, j, req_off, lo, hi, priv, stamp, comb, &cells, &ncell, &capcell)) {
        free(stamp);
        free(comb);
        free(cells);
        return -1;
      }
      uint32_t sum = 0;
      for (int64_t c = 0; c < ncell; ++c)
        if (comb[cells[c]] == P_READ) sum += (uint32_t)state[cells[c]];
      uint32_t acc = orc_mix32((uint32_t)j, sum);
      for (int64_t c = 0; c < ncell; ++c) {
        int64_t cell = cells[c];
        if (comb[cell] == P_WRITE) state[cell] = (int32_t)orc_mix32(acc, (uint32_t)cell);
        else if (comb[cell] == P_REDUCE)
          state[cell] = (int32_t)((uint32_t)state[cell] + orc_mix32((uint32_t)j, (uint32_t)cell));
      }
      out[j] = (int32_t)acc;
    }
  }
  free(stamp);
  free(comb);
  free(cells);
  return 0;
}
