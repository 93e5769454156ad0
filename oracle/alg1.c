/*
 * alg1.c -- Algorithm 1's interpreter on host threads.
 *
 * TEST INFRASTRUCTURE ONLY (like oracle.c): the timed CPU executor baseline of
 * the benchmark and a CPU check of the countdown scheme. Nothing in the
 * product path links or calls it, and it shares no code with the CUDA
 * sources.
 *
 * Section 4.2, Algorithm 1, with the paper's worker actors as host threads
 * over one shared graph:
 *  - INIT: every task's countdown is set to its number of incoming edges, and
 *    every task without incoming edges is put in the ready queue;
 *  - EXECUTE_OP: a worker takes the next ready task from the shared queue and
 *    runs its body;
 *  - COMPLETED_EDGE: for each out-edge the worker atomically decrements the
 *    successor's countdown; the decrement that finds 1 (the last pending
 *    edge) queues the successor.
 * A worker that makes successors ready keeps the first of them and runs it
 * next (Algorithm 1's EXECUTE_OP message a worker sends itself); the others
 * go to the shared queue, an array of n slots: producers reserve a slot with
 * one atomic add on the tail and publish the task with a release store;
 * consumers claim the next reserved slot with a compare-and-swap on the head
 * (never past the tail) and wait for the producer's store, which follows its
 * reservation at once. A worker adds the tasks it ran to the shared completion
 * count when it finds no work, and every worker leaves once that count is n.
 *
 * Bodies: EMPTY (nothing), SPIN (out[v] = the LCG x = 1664525 x + 1013904223
 * iterated spin_iters times from x = v), COUNTER (state[body_arg[v]] += 1,
 * ordered only by the edges). Tickets (optional): per task a start and a
 * finish number drawn from one atomic counter, so a test can check that every
 * edge's source finished before its target started.
 */
#include <pthread.h>
#include <sched.h>
#include <stdatomic.h>
#include <stdint.h>
#include <stdlib.h>
#include <time.h>

#define A1_EMPTY 0
#define A1_SPIN 1
#define A1_COUNTER 2

typedef struct {
  int32_t n;
  const int64_t* row_ptr;
  const int32_t* col;
  atomic_int* count;
  atomic_int* slot;
  atomic_int head, tail, ticket, done;
  int32_t body, spin_iters;
  const int32_t* body_arg;
  int32_t* state;
  int32_t* out;
  int32_t* tickets;
  atomic_int go; /* set once INIT is done */
} a1_job;

static uint32_t a1_spin(uint32_t x, int32_t iters) {
  for (int32_t k = 0; k < iters; ++k) x = x * 1664525u + 1013904223u;
  return x;
}

static void* a1_worker(void* arg) {
  a1_job* J = (a1_job*)arg;
  unsigned wait = 0;
  while (!atomic_load_explicit(&J->go, memory_order_acquire))
    if (++wait > 256) sched_yield();
  int local = -1; /* a ready successor this worker runs next */
  int ran = 0;    /* tasks run, not yet added to the completion count */
  unsigned idle = 0;
  for (;;) {
    int v = local;
    local = -1;
    if (v < 0) {
      int h = atomic_load_explicit(&J->head, memory_order_relaxed);
      if (h >= atomic_load_explicit(&J->tail, memory_order_relaxed)) {
        if (ran) {
          atomic_fetch_add_explicit(&J->done, ran, memory_order_relaxed);
          ran = 0;
        }
        if (atomic_load_explicit(&J->done, memory_order_relaxed) >= J->n) break;
        if (++idle > 64) sched_yield();
        continue;
      }
      if (!atomic_compare_exchange_weak_explicit(&J->head, &h, h + 1, memory_order_relaxed,
                                                 memory_order_relaxed))
        continue;
      while ((v = atomic_load_explicit(&J->slot[h], memory_order_acquire)) < 0) {
      }
    }
    idle = 0;
    if (J->tickets) J->tickets[2 * (int64_t)v] = atomic_fetch_add(&J->ticket, 1);
    if (J->body == A1_SPIN) {
      J->out[v] = (int32_t)a1_spin((uint32_t)v, J->spin_iters);
    } else if (J->body == A1_COUNTER) {
      int32_t k = J->body_arg[v];
      J->state[k] = (int32_t)((uint32_t)J->state[k] + 1u);
    }
    if (J->tickets) J->tickets[2 * (int64_t)v + 1] = atomic_fetch_add(&J->ticket, 1);
    ++ran;
    for (int64_t e = J->row_ptr[v]; e < J->row_ptr[v + 1]; ++e) {
      const int s = J->col[e];
      if (atomic_fetch_sub_explicit(&J->count[s], 1, memory_order_acq_rel) == 1) {
        if (local < 0) {
          local = s;
        } else {
          const int t = atomic_fetch_add_explicit(&J->tail, 1, memory_order_relaxed);
          atomic_store_explicit(&J->slot[t], s, memory_order_release);
        }
      }
    }
  }
  return NULL;
}

static int64_t a1_now_ns(void) {
  struct timespec ts;
  clock_gettime(CLOCK_MONOTONIC, &ts);
  return (int64_t)ts.tv_sec * 1000000000LL + ts.tv_nsec;
}

/* Runs the graph (CSR by source; every column > its row, as the analysis
 * produces) once on `threads` threads (fewer if some cannot be started).
 * Returns 0, or -1 on allocation failure. *ns receives the time from INIT to the last completion
 * (thread start-up excluded). tickets: NULL or int32[2n]. */
int32_t orc_alg1_run(int32_t n, const int64_t* row_ptr, const int32_t* col, int32_t threads, int32_t body,
                     int32_t spin_iters, const int32_t* body_arg, int32_t* state, int32_t* out,
                     int32_t* tickets, int64_t* ns) {
  if (threads < 1) threads = 1;
  a1_job J;
  J.n = n;
  J.row_ptr = row_ptr;
  J.col = col;
  J.body = body;
  J.spin_iters = spin_iters;
  J.body_arg = body_arg;
  J.state = state;
  J.out = out;
  J.tickets = tickets;
  J.count = (atomic_int*)malloc((size_t)(n ? n : 1) * sizeof(atomic_int));
  J.slot = (atomic_int*)malloc((size_t)(n ? n : 1) * sizeof(atomic_int));
  pthread_t* tid = (pthread_t*)malloc((size_t)threads * sizeof(pthread_t));
  if (!J.count || !J.slot || !tid) {
    free(J.count);
    free(J.slot);
    free(tid);
    return -1;
  }
  atomic_init(&J.go, 0);
  int started = 0;
  for (int t = 0; t < threads; ++t) {
    if (pthread_create(&tid[t], NULL, a1_worker, &J)) break;
    started++;
  }
  /* INIT: countdowns and roots, timed from here (the workers are up) */
  const int64_t t0 = a1_now_ns();
  for (int32_t v = 0; v < n; ++v) {
    atomic_init(&J.count[v], 0);
    atomic_init(&J.slot[v], -1);
  }
  for (int64_t e = 0; e < (n ? row_ptr[n] : 0); ++e)
    atomic_fetch_add_explicit(&J.count[col[e]], 1, memory_order_relaxed);
  int roots = 0;
  for (int32_t v = 0; v < n; ++v)
    if (atomic_load_explicit(&J.count[v], memory_order_relaxed) == 0)
      atomic_store_explicit(&J.slot[roots++], v, memory_order_relaxed);
  atomic_init(&J.head, 0);
  atomic_init(&J.tail, roots);
  atomic_init(&J.ticket, 0);
  atomic_init(&J.done, 0);
  atomic_store_explicit(&J.go, 1, memory_order_release);
  if (started == 0) a1_worker(&J); /* no thread could start: run on the caller's */
  for (int t = 0; t < started; ++t) pthread_join(tid[t], NULL);
  const int64_t t1 = a1_now_ns();
  if (ns) *ns = t1 - t0;
  free(J.count);
  free(J.slot);
  free(tid);
  return 0;
}
