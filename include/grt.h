/*
 * grt.h -- C ABI of libgrt, a GPU-resident task-graph runtime for GB300.
 *
 * The library covers the data-parallel path behind per-task runtime overhead
 * in "On the Duality of Task and Actor Programming Models" (arXiv 2508.16522):
 *
 *  - implicit dependence analysis: a program-ordered stream of task launches,
 *    each with region requirements (inclusive int64 rectangles plus a read,
 *    write or reduce-sum privilege), is turned into the task DAG on the GPU
 *    (Section 2.2, implicitly-parallel task systems; Section 5);
 *  - compiled-graph execution: the DAG runs actor-style, each task holding a
 *    countdown of pending incoming edges and its out-edge (trigger) list, with
 *    one atomic decrement per edge instead of events (Section 4.2,
 *    Algorithm 1);
 *  - trace replay: a captured DAG is re-executed without re-analysis
 *    (Section 5, tracing);
 *  - batched execution of many captured graphs in one persistent launch, and a
 *    serving loop that admits graphs as they arrive (Section 4.1: a whole
 *    graph is launched as a single operation).
 *
 * Edge rule (the paper does not define one; this is the library's reading):
 *  (1) a task's rectangles on one cell combine into one privilege:
 *      read+read = read, reduce+reduce = reduce, anything else = write;
 *  (2) per cell, the accesses in program order form runs -- a write is a run
 *      of its own, consecutive reads form one run, consecutive reduces form
 *      one run -- and every member of a run gets an edge from every member of
 *      the run before it;
 *  (3) explicit predecessor lists (Fig. 3, launch(..., pre)) add their edges.
 *  Edges are deduplicated; the DAG is stored as CSR by source with ascending
 *  columns, which is the canonical form every result is compared in.
 *
 * Conventions
 *  - Every call returns rt_status; nothing is thrown across the ABI. On an
 *    error, rt_last_error() returns a thread-local message.
 *  - Device work is ordered on the stream given at creation (a cudaStream_t
 *    passed as void*); calls are asynchronous unless stated otherwise.
 *  - Calls on distinct graphs (batches, servers) may run concurrently from
 *    different host threads; calls on one graph must not overlap. A graph's
 *    rt_analyze blocks only its own thread, so analyses of graphs on their
 *    own streams overlap on the GPU when their threads run them together.
 *  - The library owns everything it allocates (CSR, counters, ring, scratch);
 *    the caller owns `state`/`out` buffers and every array it passes in.
 *  - A task id is the position of its launch in the graph's program order
 *    (0-based, across all rt_launch_batch calls).
 *  - Every device wait is bounded: an executor that sees no progress for
 *    timeout_ns gives up and reports RT_ERR_TIMEOUT; the context stays usable.
 */
#ifndef GRT_H
#define GRT_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct rt_graph* rt_graph_t;
typedef struct rt_batch* rt_batch_t;

typedef enum {
  RT_OK = 0,
  RT_ERR_INVALID = 1, /* bad argument or launch data (nothing was appended) */
  RT_ERR_OOM = 2,     /* device or host allocation failed, or a size limit was hit */
  RT_ERR_CUDA = 3,    /* a CUDA call failed (e.g. no device) */
  RT_ERR_TIMEOUT = 4, /* the executor made no progress for timeout_ns */
  RT_ERR_STATE = 5,   /* call out of order (e.g. execute before analyze) */
  RT_ERR_BUDGET = 6   /* serving: a request does not fit the memory budget */
} rt_status;

/* privileges of a region requirement */
enum { RT_READ = 0, RT_WRITE = 1, RT_REDUCE_SUM = 2 };

/* task bodies run in place by the executor (integer sums wrap mod 2^32)
 *  EMPTY   nothing (pure runtime overhead)
 *  SPIN    x = task id; spin_iters times x = x*1664525 + 1013904223; out[task] = x
 *  FMA     x = (float)task id; spin_iters times x = fma(x, 0.999f, 0.25f) in IEEE
 *          binary32, round to nearest even; out[task] = the bits of x (the
 *          floating-point loop of Task Bench's compute-bound kernel)
 *  COUNTER state[body_arg[task]] += 1 (plain, non-atomic read-modify-write)
 *  CHECK   acc = mix32(task, sum of state over the task's read cells);
 *          state[c] = mix32(acc, c) on its write cells;
 *          state[c] += mix32(task, c) on its reduce cells (atomic);
 *          out[task] = acc.  mix32(a, b) = fmix32(a ^ (b * 0x9E3779B1)),
 *          fmix32 = murmur3's finaliser; c = row-major cell index.            */
enum { RT_BODY_EMPTY = 0, RT_BODY_SPIN = 1, RT_BODY_COUNTER = 2, RT_BODY_CHECK = 3, RT_BODY_FMA = 4 };

/* rt_launch_batch flags */
enum {
  RT_LAUNCH_HOST = 0,      /* arrays are host pointers, validated on the host */
  RT_LAUNCH_DEVICE = 1,    /* arrays are device pointers, validated on the device
                              (a bad batch is reported by rt_analyze) */
  RT_LAUNCH_DEFER_CHECK = 2 /* with host pointers: validate on the device instead */
};

/* executor policies of a single graph (rt_graph_exec_policy) */
enum {
  RT_EXEC_RING = 0,  /* ready tasks go through a global ring that any warp claims from */
  RT_EXEC_OWNED = 1  /* every warp owns fixed chunks of consecutive tasks and polls their countdowns */
};

/* rt_graph_desc.flags */
enum {
  RT_GRAPH_TICKETS = 1, /* record per-task (start, finish) tickets of the last run */
  RT_GRAPH_PROFILE = 2  /* time each analysis/execution kernel with CUDA events */
};

typedef struct {
  int32_t ndim;                   /* 1 or 2 */
  int64_t dom_lo[2], dom_hi[2];   /* inclusive domain bounds (index 1 unused for 1-D) */
  int32_t body;                   /* RT_BODY_* */
  int32_t spin_iters;             /* SPIN, FMA: iteration count (>= 0) */
  void* state;                    /* int32 device buffer, caller-owned: one per cell
                                     (CHECK, row-major) or per counter (COUNTER) */
  int64_t state_elems;
  void* out;                      /* int32 device buffer, one per task (SPIN, FMA, CHECK) */
  int64_t out_elems;
  void* stream;                   /* cudaStream_t; NULL = legacy default stream */
  int32_t tile_w, tile_h;         /* analysis tile in cells; 0 = library default */
  int64_t timeout_ns;             /* executor no-progress limit; 0 = 2 s. Warps report progress
                                     in batches (up to 4096 tasks each), so a serial chain of
                                     very long bodies needs a limit above their total time */
  int32_t flags;                  /* RT_GRAPH_* */
} rt_graph_desc;

/* Per-phase statistics of the last rt_analyze / execution (rt_graph_stats). */
typedef struct {
  int64_t n_tasks, n_rects, n_preds;
  int64_t n_entries;      /* (rect, tile) pairs after binning */
  int64_t n_pairs;        /* candidate (src, dst) pairs the sweep wrote, before deduplication
                             (with the pair-key filter: those it did not drop) */
  int64_t n_edges;        /* distinct edges */
  int64_t n_roots;
  int32_t tile_w, tile_h;
  float ms_analyze;       /* whole analysis, CUDA events (RT_GRAPH_PROFILE) */
  float ms_bin, ms_sort_entries, ms_sweep, ms_sort_pairs, ms_csr;
  float ms_execute;       /* last execution launch (seed + executor) */
  float ms_exec_kernel;   /* the persistent executor kernel alone */
  int32_t exec_blocks, exec_threads;
  float ms_sweep_kernel;  /* the interference sweep kernel alone */
  int32_t csr_by_buckets; /* 1: the CSR was built from per-source buckets (every row held at most
                             1024 candidate pairs), 0: from a radix sort of all the pairs */
  int32_t pair_filter_bits; /* dense inputs (16+ binned entries per task): log2 of the slots of the
                               pair-key filter the first sweep wrote through (a pair found again in
                               another tile is not written again); 0: no filter */
  int32_t pad1;
  /* diagnostic counters of the last executor launch: batches, tasks, edges,
   * ring claims, failed claim CASes, items published to the ring, idle polls,
   * waits for a reserved slot, ready successors kept by their warp */
  int64_t exec_counters[9];
} rt_graph_stats_t;

/* Creates an empty graph. Makes no CUDA call (device buffers are allocated on
 * first use), so argument errors are reported without a GPU.
 * Errors: RT_ERR_INVALID (NULL args, ndim not 1/2, dom_lo > dom_hi, unknown
 * body, tile larger than the supported maximum, negative sizes). */
rt_status rt_graph_create(const rt_graph_desc* desc, rt_graph_t* out);

/* Frees every library-owned buffer of the graph (waits for its stream). */
rt_status rt_graph_destroy(rt_graph_t g);

/* Drops all launches (keeps device buffers for reuse); the graph returns to
 * the state right after rt_graph_create. */
rt_status rt_graph_clear(rt_graph_t g);

/* Appends n launches in program order (Fig. 3, launch(p, tid, args, pre);
 * Section 2.2). Launch i of the batch gets task id (previous count + i).
 *  req_off  int32[n+1], req_off[0] == 0, non-decreasing: launch i owns
 *           rectangles [req_off[i], req_off[i+1]) of this batch
 *  lo, hi   int64[R][ndim] inclusive bounds, R = req_off[n]; lo <= hi and
 *           inside the domain
 *  priv     uint8[R], RT_READ / RT_WRITE / RT_REDUCE_SUM
 *  pred_off int32[n+1] and pred (optional, both NULL or both set): explicit
 *           predecessor ids, each in [0, own id) -- backward edges only, so
 *           the graph cannot have a cycle
 *  body_arg int32[n] (optional; required for COUNTER): per-task body argument
 *  flags    RT_LAUNCH_HOST / RT_LAUNCH_DEVICE / RT_LAUNCH_DEFER_CHECK
 * The arrays are copied; the caller keeps ownership (pinned host arrays are
 * copied asynchronously and must stay valid until rt_analyze returns). Errors: RT_ERR_INVALID
 * (with host validation nothing is appended), RT_ERR_STATE (graph already
 * analyzed: call rt_graph_clear first), RT_ERR_OOM, RT_ERR_CUDA. */
rt_status rt_launch_batch(rt_graph_t g, int32_t n, const int32_t* req_off, const int64_t* lo,
                          const int64_t* hi, const uint8_t* priv, const int32_t* pred_off,
                          const int32_t* pred, const int32_t* body_arg, int32_t flags);

/* rt_launch_batch with the rectangle bounds as int32[R][ndim]: the same
 * launches (Section 2.2), half the coordinate bytes on the host link. The
 * bounds are copied as they are and widened to int64 on the device, into the
 * graph's own arrays; arguments, ownership, validation (host or device, as
 * the flags say) and errors are those of rt_launch_batch. */
rt_status rt_launch_batch32(rt_graph_t g, int32_t n, const int32_t* req_off, const int32_t* lo,
                            const int32_t* hi, const uint8_t* priv, const int32_t* pred_off,
                            const int32_t* pred, const int32_t* body_arg, int32_t flags);

/* Infers the DAG of all launches so far (tile binning, per-tile interference
 * sweep, CSR construction) and prepares the countdown counters (Algorithm 1,
 * Compile). Synchronises the stream a few times to size buffers. Errors:
 * RT_ERR_INVALID (a device-validated batch was bad), RT_ERR_OOM, RT_ERR_CUDA. */
rt_status rt_analyze(rt_graph_t g);

/* Device pointers (library-owned, valid until the next analyze/clear/destroy)
 * to the canonical CSR: row_ptr int32[n+1], col int32[E] (ascending within a
 * row), indeg int32[n]. Synchronises the stream. RT_ERR_STATE before analyze. */
rt_status rt_get_csr(rt_graph_t g, const int32_t** row_ptr, const int32_t** col,
                     const int32_t** indeg, int64_t* n_tasks, int64_t* n_edges);

/* Copies the canonical CSR into caller-owned buffers (host or device
 * pointers, any of them may be NULL): row_ptr int32[n+1], col int32[E],
 * indeg int32[n]. Synchronous. RT_ERR_STATE before analyze. */
rt_status rt_copy_csr(rt_graph_t g, int32_t* row_ptr, int32_t* col, int32_t* indeg);

/* Runs the DAG once (Algorithm 1: INIT seeds every task without incoming
 * edges; each completion decrements its successors' counters and a counter
 * reaching zero makes the task ready). Asynchronous: the status is reported by
 * rt_sync. RT_ERR_STATE before rt_analyze. */
rt_status rt_execute(rt_graph_t g);

/* Replays the captured DAG `times` times without re-analysis (Section 5):
 * counters are restored on the device and the runs happen back to back in one
 * persistent launch (relaunched from a cached CUDA graph). Asynchronous. */
rt_status rt_replay(rt_graph_t g, int32_t times);

/* Runs the analysed graph once through the STANDARD, event-based executor
 * instead of the compiled one, for comparison (the paper's generic task
 * runtime, Fig. task-to-rt-actor reduction, against its compiled actors,
 * Section 4.2): every run starts with fresh events; each launch registers as a
 * waiter on its preconditions' events (built from the CSR's in-edges, as the
 * application would state them), and a finished task triggers its event and
 * notifies the waiters. Bodies and results are those of rt_execute.
 * Synchronous; *ms_kernel (may be NULL) receives the kernel time. Errors:
 * RT_ERR_STATE (not analyzed), RT_ERR_INVALID, RT_ERR_TIMEOUT (no progress for
 * timeout_ns), RT_ERR_OOM, RT_ERR_CUDA. */
rt_status rt_execute_events(rt_graph_t g, float* ms_kernel);

/* Stitched replay (Section 4.1's external pre/post-condition vertices, which
 * join a compiled graph to the work around it; Section 5 joins the graphs of a
 * sharded trace with them). `g` holds one trace launched TWICE in a row (2n
 * tasks, analysed; the second copy must repeat the first's rectangles, and
 * any explicit predecessors shifted by n). Edges inside the first copy are
 * the compiled graph; edges from the first copy to the second are the
 * conditions that join replay r to replay r + 1. Runs `replays` replays of
 * the trace in one persistent launch with no barrier between them: a task of
 * replay r + 1 starts once its predecessors in replays r and r + 1 are done.
 * Task (r, v) writes out[r * n + v] (SPIN: the SPIN value of v; CHECK: its
 * output word, the state evolving as if the trace ran `replays` times in
 * program order; `out` must hold replays * n int32 for those bodies); COUNTER
 * bodies act on state as in rt_execute. With RT_GRAPH_TICKETS the start and
 * end tickets of (r, v) are kept for rt_copy_stitched_tickets. Synchronous;
 * *ms_kernel (may be NULL) receives the launch's time (counter init plus the
 * executor). Errors: RT_ERR_STATE (not analyzed), RT_ERR_INVALID (odd task
 * count, halves that differ in rectangles or internal edges, replays < 1,
 * replays * n >= 2^31 - 16, missing `out`), RT_ERR_TIMEOUT (no progress for
 * timeout_ns, default 2 s), RT_ERR_OOM, RT_ERR_CUDA. */
rt_status rt_execute_stitched(rt_graph_t g, int32_t replays, float* ms_kernel);

/* Copies the tickets of the last stitched run made with RT_GRAPH_TICKETS:
 * int32[replays][n][2] (start, end), into host or device memory. Synchronous.
 * RT_ERR_STATE if there is none. */
rt_status rt_copy_stitched_tickets(rt_graph_t g, int32_t* out);

/* Runs the analysed graph with every task as its own GPU kernel (Section
 * 4.3, optimisations for accelerators): one block of `threads` threads
 * (32..1024), each running `iters` dependent FMAs, after which the task writes
 * out[v] = 1 + the largest out[] of its predecessors (its depth, right only if
 * every predecessor finished first). mode 0 = lifted: the host launches a task
 * once it has seen, by polling, its predecessors' completion events; 1 = async
 * edges: every kernel enqueued up front on a pool of streams, predicated on its
 * predecessors' events; 2 = a CUDA graph of kernel nodes with the DAG's edges,
 * instantiated once per (iters, threads) and relaunched. Needs `out` (one
 * int32 per task), at most 131072 tasks. Synchronous; *ms (may be NULL)
 * receives the host wall time of the run. Errors: RT_ERR_STATE, RT_ERR_INVALID,
 * RT_ERR_TIMEOUT (mode 0 saw no completion for timeout_ns, default 10 s),
 * RT_ERR_CUDA. */
rt_status rt_execute_kernels(rt_graph_t g, int32_t mode, int32_t iters, int32_t threads, float* ms);

/* Launch shape of this graph's executor runs (0 = library default): number of
 * persistent blocks, warps per block (1..8), how many published ring slots a
 * warp claims at once (1..32; default 8) and how many newly ready successors a
 * warp keeps for its own next batch instead of publishing them (0..64). These
 * are the autotuner's knobs; results do not depend on them. The event-based
 * executor (rt_execute_events) takes the same claim width. */
rt_status rt_graph_exec_config(rt_graph_t g, int32_t blocks, int32_t warps, int32_t claim, int32_t keep);

/* How rt_execute / rt_replay find ready tasks (Algorithm 1's EXECUTE_OP):
 * RT_EXEC_RING (default) publishes every task made ready that its warp does
 * not keep to a global ring that any warp claims from; RT_EXEC_OWNED gives
 * every warp fixed chunks of consecutive tasks (chunk c to warp c mod the
 * grid's warps, taken in increasing order) and lets it poll their countdowns,
 * the predecessors decrementing them with reductions that need no answer --
 * the operations compiled to their worker of Algorithm 1. OWNED suits graphs
 * whose tasks become ready roughly in task order (the wavefronts of Task
 * Bench); RING suits irregular ones. Under OWNED the claim width of
 * rt_graph_exec_config is the number of lanes that hold one task (1, 2 or 4;
 * default 1; a chunk is 32 / that many tasks, and the task's successors are
 * split between its lanes) and keep is unused. The first OWNED run after an
 * analysis of a graph with a task of more than 5 successors builds 32 more
 * bytes of trigger record per task (successors 6 to 13 inline). Results never
 * depend on the policy. Errors: RT_ERR_INVALID. */
rt_status rt_graph_exec_policy(rt_graph_t g, int32_t policy);

/* Waits for the graph's stream; returns RT_OK, RT_ERR_TIMEOUT (the executor
 * gave up; the next execution re-initialises the counters) or RT_ERR_CUDA. */
rt_status rt_sync(rt_graph_t g);

/* Statistics of the last analysis / execution (synchronises the stream). */
rt_status rt_graph_stats(rt_graph_t g, rt_graph_stats_t* out);

/* Device pointer to int32[2*n] (start, finish) tickets of the last run, drawn
 * from one global counter (RT_GRAPH_TICKETS only; synchronises). */
rt_status rt_get_tickets(rt_graph_t g, const int32_t** tickets);

/* Copies the tickets of the last run into a caller buffer int32[2*n] (host or
 * device). Synchronous. */
rt_status rt_copy_tickets(rt_graph_t g, int32_t* out);

/* Test hook for bounded waits: the next execution adds `extra` to the
 * countdown of `task`, so that task never becomes ready and the executor must
 * give up with RT_ERR_TIMEOUT after timeout_ns (no trap, no fault). */
rt_status rt_debug_hold_task(rt_graph_t g, int32_t task, int32_t extra);

/* ---- batched execution (Section 4.1: a registered graph runs as one op) --
 * Builds one disjoint union of already-analyzed graphs: their CSRs, counters
 * and roots are copied into batch-owned buffers (the captured traces), with
 * task ids shifted so graph g's tasks follow graph g-1's. The batch still
 * refers to each graph's body buffers (state/out) and launch data (CHECK
 * body), so the graphs must outlive it. At most 2^20 - 1 graphs. Errors:
 * RT_ERR_STATE if a graph is not analyzed, RT_ERR_INVALID, RT_ERR_OOM,
 * RT_ERR_CUDA. */
rt_status rt_batch_create(const rt_graph_t* graphs, int32_t n_graphs, void* stream,
                          rt_batch_t* out);

/* A batch from ONE analysed graph whose tasks [task_off[k], task_off[k+1])
 * form graph k (task_off: host int32[n_graphs+1], from 0 to the graph's task
 * count). The caller places the graphs in disjoint parts of the domain (for
 * instance stacked bands), so that one analysis captures all of them; the
 * batch then runs each graph and replays it independently, as rt_batch_create
 * does. A body sees its graph's own tasks (ids from 0); state-carrying bodies
 * share the graph's state buffer, in which the graphs' parts are disjoint.
 * The graph must outlive the batch. Errors: RT_ERR_STATE (not analyzed),
 * RT_ERR_INVALID (bad offsets, or an edge joins two graphs: checked on the
 * device), RT_ERR_OOM, RT_ERR_CUDA. */
rt_status rt_batch_create_stacked(rt_graph_t g, const int32_t* task_off, int32_t n_graphs, void* stream,
                                  rt_batch_t* out);

/* Captures a batch of independent graphs with ONE analysis, placing them in
 * bands of one domain itself (Section 4.1: each graph is then launched as one
 * operation; Section 5: the analysis is done once and replayed). Graph k owns
 * launches [task_off[k], task_off[k+1]) of the arrays (host task_off
 * int32[n_graphs+1], from 0), and its rectangles are in its OWN domain
 * [graph_lo[k], graph_hi[k]] (host int64[n_graphs][ndim], inclusive). The
 * library stacks the domains along the last dimension -- graph k's band starts
 * where graph k-1's ends, at 0 across the other dimension -- so that the
 * graphs share no cell, copies the launches (req_off int32[n+1] over all
 * launches, lo/hi int64[R][ndim], priv uint8[R], R = req_off[n]; host arrays,
 * or device arrays with RT_LAUNCH_DEVICE), checks on the device that every
 * rectangle lies in its own graph's domain and moves it into the graph's band,
 * analyses the stacked graph and builds the batch as
 * rt_batch_create_stacked does. desc gives ndim, body, spin_iters, the body
 * buffers, stream, tile, timeout and flags (its domain is ignored): `out`
 * holds one int32 per task of all graphs, and a CHECK body's `state` one int32
 * per cell of the stacked domain, [0, W-1] x [0, H-1] in 2-D with W the
 * widest graph and H the sum of the graphs' heights ([0, sum of lengths - 1]
 * in 1-D). The batch owns the stacked graph; *graph_out (may be NULL)
 * receives it for rt_copy_csr and rt_graph_stats, valid until the batch is
 * destroyed. Errors: RT_ERR_INVALID (bad offsets or domains, a rectangle
 * outside its graph's domain -- reported by the analysis), RT_ERR_OOM,
 * RT_ERR_CUDA. */
rt_status rt_batch_capture(const rt_graph_desc* desc, int32_t n_graphs, const int32_t* task_off,
                           const int64_t* graph_lo, const int64_t* graph_hi, const int32_t* req_off, const int64_t* lo,
                           const int64_t* hi, const uint8_t* priv, int32_t flags, rt_batch_t* out,
                           rt_graph_t* graph_out);

/* One persistent launch in which every graph of the batch runs `replays` times
 * (1..4096); graph g's replay r+1 starts as soon as its replay r has finished,
 * independently of the other graphs. exec_blocks/exec_warps/claim/keep (0 =
 * default) are the launch shape of rt_graph_exec_config. The batch's counters
 * are reset at the start of every launch. The launch {counter reset, seed,
 * executor, status read-back} is captured as a CUDA graph once per launch
 * shape and relaunched from it afterwards (the first launch of a new or
 * grown ring, which clears the whole ring, is issued directly). Asynchronous. */
rt_status rt_batch_execute(rt_batch_t b, int32_t replays, int32_t exec_blocks, int32_t exec_warps,
                           int32_t claim, int32_t keep);

/* How rt_batch_execute runs the batch (Algorithm 1's EXECUTE_OP, as for one
 * graph in rt_graph_exec_policy): RT_EXEC_RING (default) as described above;
 * RT_EXEC_OWNED runs the batch's graphs as ONE DAG under the owned-chunk
 * executor (every edge of the batch points to a later task), with count-down
 * counters reset to the in-degrees at every launch and a run barrier between
 * replays: replay r + 1 of every graph starts once replay r of all graphs has
 * finished, a stricter order that gives every graph the same results; each
 * body still sees its own graph's task ids and buffers. Under OWNED the claim
 * width is the lanes per task (1, 2 or 4). The first OWNED launch builds each
 * task's graph index (4 bytes per task) and, when some task has more than 5
 * successors, 32 more bytes of trigger record per task. Errors:
 * RT_ERR_INVALID. */
rt_status rt_batch_exec_policy(rt_batch_t b, int32_t policy);

rt_status rt_batch_sync(rt_batch_t b, float* ms_kernel);

/* out[0] graphs, [1] tasks, [2] edges, [3] launches made from the cached CUDA
 * graph so far (n values; no device work). */
rt_status rt_batch_info(rt_batch_t b, int64_t* out, int32_t n);

/* The first n (<= 9) diagnostic counters of the last batch launch, in the
 * order of rt_graph_stats_t.exec_counters (synchronises). */
rt_status rt_batch_counters(rt_batch_t b, int64_t* out, int32_t n);
rt_status rt_batch_destroy(rt_batch_t b);

/* ---- autotuning -----------------------------------------------------------
 * Results never depend on the analysis tile or the executor's launch shape;
 * speed does, and the best values depend on the workload and the device. The
 * tuners measure candidates on the caller's own workload and keep the fastest.
 * cache_path (may be NULL) names a plain-text cache, one line per workload key
 * (device name and SM count, kind, sizes, an input hash): a key found there is
 * answered without running anything; a new result is appended. The paper
 * fixes no such knobs (its runtime compiles one worker per processor). */
typedef struct {
  int32_t blocks, warps, claim, keep;  /* launch shape (rt_graph_exec_config) */
  float ms;                            /* time of one run with it */
  int32_t trials;                      /* shapes measured (0: from the cache) */
  int32_t policy;                      /* RT_EXEC_RING or RT_EXEC_OWNED (rt_tune_exec) */
} rt_exec_config;

/* Analyses the launches (host arrays, as rt_launch_batch) once per candidate
 * tile -- 8, 16, 32, 64 square and 8x16, 16x8, 32x4, 32x8, 64x4 in 2-D;
 * 128..1024 in 1-D -- in a temporary
 * graph built from desc (body, state, out and flags ignored), and returns the
 * tile whose analysis was fastest (its ms in *ms, may be NULL). Errors:
 * RT_ERR_INVALID (bad arguments, or no candidate could analyse the trace). */
rt_status rt_tune_tile(const rt_graph_desc* desc, int32_t n, const int32_t* req_off, const int64_t* lo,
                       const int64_t* hi, const uint8_t* priv, const char* cache_path, int32_t* tile_w,
                       int32_t* tile_h, float* ms);

/* Runs an analysed graph under candidate launch shapes -- the ring policy by
 * coordinate descent (warps x blocks per SM, then claim, then keep; best of
 * two runs each), the owned policy over its grids and then lanes per task
 * (best of three) -- and
 * configures it with the fastest policy and shape (rt_graph_exec_policy,
 * rt_graph_exec_config). The graph's bodies run once per trial: a
 * state-changing body sees those runs. Synchronous. */
rt_status rt_tune_exec(rt_graph_t g, const char* cache_path, rt_exec_config* best);

/* The same for a batch launch of `replays` replays: the ring policy by
 * coordinate descent, then one run of the owned policy and, only if that run
 * comes within 1.5x of the ring, its grids (1-3 blocks of 4 or 8 warps per SM)
 * and 1, 2 or 4 lanes per task; sets the batch's policy
 * (rt_batch_exec_policy) to the faster one and returns the shape (with its
 * policy) for rt_batch_execute. The bodies run once per trial. Synchronous. */
rt_status rt_tune_batch(rt_batch_t b, int32_t replays, const char* cache_path, rt_exec_config* best);

/* ---- serving (continuous batching) ---------------------------------------
 * A server analyses requests (each a graph of launches with region
 * requirements) as they arrive and executes them in one persistent kernel that
 * admits new graphs while others are still running (Section 4.1: each graph
 * runs as one operation; Section 2.2: dependences inferred from data usage).
 * Requests are admitted in arrival order while a request slot is free and the
 * device memory they would hold fits the budget. A worker thread analyses
 * every admitted request that is waiting (up to max_batch) as ONE graph, each
 * request's rectangles shifted into a band of their own along the domain's
 * last dimension, so the requests' DAGs stay disjoint; analysis runs on the
 * workers' own streams, concurrently with the executing kernel, and each
 * request completes on its own. */
typedef struct rt_server* rt_server_t;

typedef struct {
  int32_t ndim;                  /* every request shares this domain and tiling */
  int64_t dom_lo[2], dom_hi[2];
  int32_t tile_w, tile_h;        /* 0 = library default */
  int32_t body;                  /* RT_BODY_EMPTY, RT_BODY_SPIN or RT_BODY_CHECK. A served body
                                    sees its request alone: task ids from 0 within the request
                                    and, for CHECK, the request's own zeroed state (one int32
                                    per cell of this domain, row-major), so every result equals
                                    that of the request run by itself */
  int32_t spin_iters;
  int64_t budget_bytes;          /* device memory the analysed requests' graphs may hold at
                                    once, retained buffers included (the fixed pool allocated
                                    at creation is apart): each batch graph grows under a cap
                                    that keeps the sum within it */
  int32_t max_inflight;          /* graphs admitted at once, 1..1024 */
  int32_t max_tasks;             /* tasks of the largest request accepted */
  int32_t workers;               /* host threads analysing requests, 1..64 */
  int32_t keep_results;          /* keep each request's CSR (and SPIN outputs) */
  int32_t exec_blocks, exec_warps;  /* serving kernel shape, 0 = default */
  int64_t timeout_ns;            /* stall limit of the serving kernel, 0 = 2 s */
  int32_t max_batch;             /* requests analysed together, 1..1024, 0 = 64;
                                    max_batch x max_tasks < 2^31 */
  int32_t reserved0;             /* 0 */
} rt_server_desc;

typedef struct {
  int32_t state;                 /* 0 queued, 1 analysing, 2 running, 3 done, 4 failed */
  int32_t status;                /* rt_status of a failed request */
  int64_t arrival_ns, admit_ns, posted_ns, done_ns;  /* rt_now_ns clock */
  int64_t n_tasks, n_edges, footprint_bytes;
} rt_request_info;

/* CLOCK_MONOTONIC nanoseconds: the clock of arrival and completion stamps. */
int64_t rt_now_ns(void);

/* Starts a server: allocates its graph pool, ring and mapped mailbox, launches
 * the serving kernel on its own stream and starts the worker threads. Errors:
 * RT_ERR_INVALID, RT_ERR_OOM, RT_ERR_CUDA. */
rt_status rt_server_create(const rt_server_desc* desc, rt_server_t* out);

/* Queues one request: n launches as in rt_launch_batch (host arrays, checked
 * and copied before returning; no explicit preds). arrival_ns stamps its
 * arrival (use rt_now_ns()). Errors: RT_ERR_INVALID (bad offsets, a rectangle
 * empty or outside the domain, a bad privilege, more than max_tasks tasks),
 * RT_ERR_BUDGET (it could never fit the budget), RT_ERR_STATE (stopping). */
rt_status rt_server_submit(rt_server_t s, int32_t n, const int32_t* req_off, const int64_t* lo,
                           const int64_t* hi, const uint8_t* priv, int64_t arrival_ns, int64_t* ticket);

/* State and timings of one request (non-blocking). */
rt_status rt_server_poll(rt_server_t s, int64_t ticket, rt_request_info* info);

/* With keep_results: copies a finished request's canonical CSR (row_ptr
 * int32[n+1], col int32[E]) and, for SPIN and CHECK, its outputs (int32[n])
 * into host buffers (any may be NULL). RT_ERR_STATE if it is not done; a
 * request that failed returns its own status, with the reason in
 * rt_last_error(). */
rt_status rt_server_result(rt_server_t s, int64_t ticket, int32_t* row_ptr, int32_t* col, int32_t* out);

/* With keep_results and the CHECK body: copies a finished request's final
 * state (int32, one per cell of the server's domain, row-major) into a host
 * buffer. The order-sensitive CHECK body makes this the proof that the
 * request's edges were respected while it ran beside others (Algorithm 1:
 * a task runs only after all its predecessors). Errors as rt_server_result;
 * RT_ERR_STATE if the server does not run CHECK bodies or keep results. */
rt_status rt_server_result_state(rt_server_t s, int64_t ticket, int32_t* state);

/* Waits until every submitted request is done or failed (or timeout_ns
 * passes: RT_ERR_TIMEOUT), or the serving kernel reported a stall. */
rt_status rt_server_drain(rt_server_t s, int64_t timeout_ns);

/* Diagnostics: out[0] activations posted, [1] taken by the kernel, [2]
 * finished, [3] kernel status, [4] tasks executed, [5] requests queued, [6]
 * analysing, [7] running, [8] 1 while the serving kernel runs, [9] batches
 * analysed, [10] requests in them; the memory budget: [11] bytes the batch
 * graphs may hold now (caps of batches in analysis, retained buffers of the
 * others; never above budget_bytes), [12] its peak, [13] bytes the batch
 * graphs hold after their last analyses, [14] its peak, [15] bytes of the
 * fixed pool allocated at creation (ring, slot table, per-batch outputs and
 * CHECK states: not request memory), [16] retained graphs trimmed to make
 * room, [17] batches that outgrew their cap and were admitted again. */
rt_status rt_server_stats(rt_server_t s, int64_t* out, int32_t n);

/* Drains (30 s at most), asks the serving kernel to stop once idle (forcing it
 * after 10 s), joins the threads and frees everything. If the kernel cannot be
 * stopped its resources are left to the process exit: RT_ERR_TIMEOUT. */
rt_status rt_server_destroy(rt_server_t s);

/* Message of the last failed call on this thread ("" if none). */
const char* rt_last_error(void);

/* Number of persistent executor blocks per SM and the SM count of the current
 * device (0 on failure); used by the autotuner. */
rt_status rt_device_info(int32_t* num_sms, int32_t* exec_blocks_per_sm);

/* Runs a graph given as a caller-held CSR without allocating anything. The
 * paper has no counterpart: this exists for callers that cannot allocate device
 * memory when they run a graph -- code inside a memory-pool or arena manager
 * that owns all device memory, or a latency-critical loop where cudaMalloc or
 * cudaFree (which synchronises the device) is not allowed. The executor's
 * scratch (countdown counters, ready ring, trigger records, control words)
 * lives in a fixed device array inside the library, about 11 MB, which every
 * GPU that loads the library keeps until the process exits.
 *  row_ptr int32[n_tasks+1], col int32[n_edges], indeg int32[n_tasks]: device
 *          pointers, caller-owned, e.g. filled by rt_copy_csr; every column must
 *          be a later task id (src < dst) and indeg must match the columns
 *  out     int32[n_tasks] device buffer: the SPIN body's result per task
 *          (x = task id; spin_iters times x = x*1664525 + 1013904223)
 *  tickets NULL, or an int32[2*n_tasks] device buffer, caller-owned: task v's
 *          start and finish tickets at [2v] and [2v+1], drawn from one counter,
 *          so the caller can check that every edge's source finished first
 *  stream  cudaStream_t (NULL = legacy default stream)
 * Synchronous: validates the CSR on the device (RT_ERR_INVALID if it is
 * malformed), runs it once and returns the executor's status; it reads flags
 * back into host memory, so it must not be called on a stream that is being
 * captured (RT_ERR_STATE). A CUDA error already pending when it is called is
 * reported as RT_ERR_CUDA before anything is launched. n_tasks may be at most
 * 262144 (2^18); larger graphs get RT_ERR_INVALID. No cudaMalloc, cudaFree or
 * allocating library call is made. The first call on a device looks up the
 * array's device address once. All calls share the one array and it keeps the
 * previous call's contents (each call re-initialises what it needs), so calls
 * whose GPU work overlaps -- from several streams or host threads -- race and
 * corrupt each other: the caller must serialise them. */
rt_status rt_execute_csr_static(const int32_t* row_ptr, const int32_t* col, const int32_t* indeg,
                                int32_t n_tasks, int64_t n_edges, int32_t spin_iters, int32_t* out,
                                int32_t* tickets, void* stream);

/* The executor's rooflines, measured on the current device (synchronous,
 * allocates a 64 MB scratch array): out[0] dependent atomic latency (ns),
 * out[1] dependent L2 load latency (ns), out[2] scattered atomicSub throughput
 * with the result used (G ops/s), out[3] the same without using the result,
 * out[4] contended single-address atomicAdd (G ops/s), out[5] the same
 * warp-aggregated (G thread-ops/s), out[6] the FMA body alone: ns per
 * dependent iteration on one warp (Task Bench's peak for its efficiency).
 * n = how many of the seven to return. */
rt_status rt_microbench_atomics(double* out, int32_t n, void* stream);

/* Total number of kernels this library has launched in the process (for
 * benchmarks that report how much GPU work a timed region issued). */
rt_status rt_kernel_launches(int64_t* count);

#ifdef __cplusplus
}
#endif

#endif /* GRT_H */
