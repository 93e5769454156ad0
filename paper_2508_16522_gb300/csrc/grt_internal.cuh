// grt_internal.cuh -- device helpers and host/device structures of libgrt.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>

#include "grt.h"

namespace grt {

// opt-in host trace (environment GRT_TRACE=1): one timestamped line per step
void trace(const char* what);

// number of kernels this library has launched (reported by rt_kernel_launches)
extern std::atomic<long long> g_kernel_launches;
inline void count_launch(long long k = 1) { g_kernel_launches.fetch_add(k, std::memory_order_relaxed); }

constexpr uint64_t kEmpty64 = ~0ull;   // empty ring slot / sentinel pair key
constexpr uint32_t kPosMask = (1u << 30) - 1;
constexpr int kKindRead = 0, kKindWrite = 1, kKindReduce = 2, kKindNone = 3;

// ---------------------------------------------------------------------------
// analysis tiling limits: a binned entry packs task id (32 bits), privilege
// (2 bits) and the rectangle clipped to its tile in local coordinates
// (4 x 7 bits in 2-D, 2 x 14 bits in 1-D) into one 64-bit word.
// ---------------------------------------------------------------------------
constexpr int kMaxTileSide2D = 128;
constexpr int kMaxTileSide1D = 16384;
constexpr int kMaxClassCells = 1024;  // per-warp cell state (shared memory): class cells swept at once

__host__ __device__ inline uint64_t pack_entry(uint32_t task, uint32_t priv, int ndim, uint32_t x0,
                                               uint32_t x1, uint32_t y0, uint32_t y1) {
  uint64_t p = (uint64_t)task | ((uint64_t)(priv & 3u) << 32);
  if (ndim == 2)
    p |= ((uint64_t)x0 << 34) | ((uint64_t)x1 << 41) | ((uint64_t)y0 << 48) | ((uint64_t)y1 << 55);
  else
    p |= ((uint64_t)x0 << 34) | ((uint64_t)x1 << 48);
  return p;
}

struct Box {
  int task, priv, x0, x1, y0, y1;
};

__device__ __forceinline__ Box unpack_entry(uint64_t p, int ndim) {
  Box b;
  b.task = (int)(uint32_t)(p & 0xffffffffu);
  b.priv = (int)((p >> 32) & 3u);
  if (ndim == 2) {
    b.x0 = (int)((p >> 34) & 127u);
    b.x1 = (int)((p >> 41) & 127u);
    b.y0 = (int)((p >> 48) & 127u);
    b.y1 = (int)((p >> 55) & 127u);
  } else {
    b.x0 = (int)((p >> 34) & 0x3fffu);
    b.x1 = (int)((p >> 48) & 0x3fffu);
    b.y0 = 0;
    b.y1 = 0;
  }
  return b;
}

// ---------------------------------------------------------------------------
// PTX wrappers (memory model: acquire/release at GPU scope)
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint64_t globaltimer_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ void fence_acq_rel_gpu() { asm volatile("fence.acq_rel.gpu;" ::: "memory"); }
__device__ __forceinline__ uint64_t ld_acquire_u64(const uint64_t* p) {
  uint64_t v;
  asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
// one decrement that returns nothing (a reduction, relaxed, GPU scope): the
// SM sends it to L2 and waits for no answer, where an atomicSub whose result
// is unused may still be issued as an atomic that returns the old value
__device__ __forceinline__ void red_dec_s32(int32_t* p) {
  asm volatile("red.relaxed.gpu.global.add.s32 [%0], -1;" ::"l"(p) : "memory");
}
__device__ __forceinline__ void red_add_s32(int32_t* p, int32_t v) {
  asm volatile("red.relaxed.gpu.global.add.s32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ void red_add_u32(uint32_t* p, uint32_t v) {
  asm volatile("red.relaxed.gpu.global.add.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ void red_add_u64(unsigned long long* p, unsigned long long v) {
  asm volatile("red.relaxed.gpu.global.add.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ int32_t ld_relaxed_s32(const int32_t* p) {
  int32_t v;
  asm volatile("ld.relaxed.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ uint32_t ld_relaxed_u32(const uint32_t* p) {
  uint32_t v;
  asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ unsigned long long ld_relaxed_u64(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release_u64(uint64_t* p, uint64_t v) {
  asm volatile("st.release.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ void st_relaxed_u64(uint64_t* p, uint64_t v) {
  asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ unsigned lanemask_lt() {
  unsigned m;
  asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
  return m;
}

// one privilege per task per cell: read+read = read, reduce+reduce = reduce,
// every other mix = write (0xFF = not yet touched)
__device__ __forceinline__ uint32_t combine_priv(uint32_t have, uint32_t add) {
  if (have == 0xFFu) return add;
  return (have == add && add != (uint32_t)kKindWrite) ? add : (uint32_t)kKindWrite;
}

// murmur3's 32-bit finaliser and the CHECK body's mixing function
__device__ __forceinline__ uint32_t fmix32(uint32_t h) {
  h ^= h >> 16;
  h *= 0x85ebca6bu;
  h ^= h >> 13;
  h *= 0xc2b2ae35u;
  h ^= h >> 16;
  return h;
}
__device__ __forceinline__ uint32_t mix32(uint32_t a, uint32_t b) { return fmix32(a ^ (b * 0x9E3779B1u)); }

// ---------------------------------------------------------------------------
// executor structures
// ---------------------------------------------------------------------------
struct ExecGraph {  // one per graph of a launch (1 for rt_execute)
  int32_t task_base, n_tasks, root_base, n_roots;
  int32_t body, spin_iters, ndim, pad0;
  int32_t* state;
  int32_t* out;
  const int32_t* body_arg;
  const int32_t* req_off;  // local rect offsets of the graph's tasks (CHECK body)
  const int64_t* lo;
  const int64_t* hi;
  const uint8_t* priv;
  int64_t dom_lo[2];
  int64_t ext[2];
};

struct ExecCtrl {  // reset before every executor launch; hot words on separate 128-byte lines
  uint32_t head, pad_h[31];        // ring tickets claimed
  uint32_t tail, pad_t[31];        // ring tickets reserved
  uint32_t graphs_done, status;    // status: 0 ok, RT_ERR_TIMEOUT, RT_ERR_OOM (ring)
  uint32_t err_where, err_info, pad_s[28];
  unsigned long long executed;     // progress counter (flushed in batches)
  uint32_t pad_e[30];
  uint32_t ticket, pad_k[31];
  unsigned long long counters[16];  // diagnostics, flushed once per warp at exit (see kCnt*)
};

// executor diagnostic counters (ExecCtrl::counters)
enum { kCntBatches = 0, kCntTasks, kCntEdges, kCntClaims, kCntCasFail, kCntPushed, kCntIdle, kCntSlotWait,
       kCntKept, kCntCount };

// packed trigger record of one task (two int4): {row start, out-degree,
// in-degree, first 5 successors (-1 padded)}
constexpr int kAdjInline = 5;
// the owned-chunk executor's extension record (two more int4 per task):
// successors kAdjInline .. kAdjWide - 1 (-1 padded), so that a task with up to
// kAdjWide successors decrements them all without reading the CSR's columns
constexpr int kAdjWide = 13;

struct ExecParams {
  const int4* adj;        // 2 x int4 per task: packed trigger records
  const int4* adjx;       // optional (owned policy): 2 x int4 per task, successors kAdjInline .. kAdjWide - 1
  const int32_t* row_ptr;
  const int32_t* col;
  const int32_t* indeg;
  int32_t* count;
  uint64_t* ring;
  uint32_t ring_cap;
  int32_t n_graphs;
  const uint64_t* root_items;  // (graph << 32 | global task id), per-graph ranges
  const ExecGraph* graphs;
  uint32_t* done_g;
  ExecCtrl* ctrl;
  int32_t replays;
  int32_t graphs_target;  // graphs with at least one task
  int64_t timeout_ns;
  int32_t claim;          // max ring items a warp claims at once (<= 32)
  int32_t keep;           // ready successors a warp keeps for itself (<= 64)
  int32_t* tickets;       // optional int32[2 * total tasks]
  int32_t total_roots;
  int32_t need_fence;     // some body reads data written by its predecessors
  int32_t policy;         // single graph: RT_EXEC_RING (ready ring) or RT_EXEC_OWNED (owned chunks)
  // the owned policy over a batch (one DAG of all its graphs, a run barrier
  // between replays): its task count and each task's graph, whose table entry
  // (task_base, body, buffers) its body runs with; 0 / null for one graph
  int32_t owned_n;
  const int32_t* task_graph;
};

// ---------------------------------------------------------------------------
// serving: one persistent executor admits analysed graphs while it runs
// ---------------------------------------------------------------------------
struct ServeSlot {         // device table entry of one admitted request
  const int4* adj;         // trigger records of the graph it was analysed in
  const int32_t* col;      // that graph's CSR columns (successors past the inline ones)
  int32_t* count;          // that graph's countdown counters
  const uint64_t* roots;   // the request's roots (low 32 bits: task id in that graph)
  int32_t* out;            // SPIN/CHECK results, one per task of that graph (null for EMPTY)
  int32_t n_tasks, n_roots, body, spin_iters;
  uint32_t gen;            // activation number, echoed at completion
  int32_t base;            // the request's first task in that graph
  uint32_t pad[2];
  // CHECK body only: the batch graph's launch arrays (indexed by batch task
  // id), the request's own state (one int32 per cell of its domain) and the
  // origin of its band in the batch's stacked domain
  const int32_t* req_off;
  const int64_t* lo;
  const int64_t* hi;
  const uint8_t* priv;
  int32_t* state;
  int64_t band_lo[2];
  int64_t ext0;
  int32_t ndim, pad1;
};

struct ServeMailbox {      // host-mapped: written by the host, read by the kernel
  volatile uint32_t posted;  // activations posted so far
  volatile uint32_t stop;    // 1: leave once nothing is admitted or running
  uint32_t pad[30];
  volatile uint32_t queue[1024];  // slot of activation k at queue[k % 1024]
};

struct ServeDone {         // host-mapped: written by the kernel, read by the host
  volatile uint32_t gen[1];  // per slot: gen of its last completed activation
};

struct ServeCtrl {         // device memory, hot words on separate lines
  unsigned long long head, pad_h[15];  // ring tickets claimed
  unsigned long long tail, pad_t[15];  // ring tickets reserved
  uint32_t taken, pad_k[31];           // activations taken from the mailbox
  uint32_t finished, status, pad_f[30];  // completed activations, error status
  unsigned long long executed, pad_e[15];
  unsigned long long counters[16];
};

struct ServeParams {
  ServeSlot* slots;
  uint32_t* done_s;        // per slot: tasks completed in its current activation
  ServeCtrl* ctrl;
  ServeMailbox* mail;      // device view of the mapped mailbox
  uint32_t* done_gen;      // device view of the mapped completion words
  uint64_t* items;         // circular ring, cap slots (power of two)
  unsigned long long* seq; // per ring slot: sequence number
  unsigned long long cap;
  int32_t max_slots;
  int32_t claim, keep;
  int64_t timeout_ns;
};

// ---------------------------------------------------------------------------
// kernels and launchers (defined in scan.cu, radix.cu, analysis.cu, exec.cu)
// ---------------------------------------------------------------------------
template <typename T>
size_t scan_ws_elems(int64_t n);
template <typename T>
void scan_exclusive(const T* in, T* out, int64_t n, T* ws, cudaStream_t s);

size_t radix_ws_bytes(int64_t n);
// sorts (keys, vals) by key bits [0, nbits); ping-pongs between the two
// buffers; returns 1 if the result is in the *_alt buffers
template <typename K>
int radix_sort(K* keys, K* keys_alt, uint64_t* vals, uint64_t* vals_alt, int64_t n, int nbits,
               void* ws, cudaStream_t s);

struct AnalysisDims {
  int ndim;
  int64_t dom_lo[2];
  int64_t ext[2];
  int tw, th;
  int ntx, nty;
};

void launch_validate(const int32_t* req_off, int32_t n, int64_t r_first, const int64_t* lo,
                     const int64_t* hi, const uint8_t* priv, int64_t R, const int32_t* pred_off,
                     const int32_t* pred, int64_t p_first, int64_t p_end, int32_t task_base,
                     const int32_t* body_arg, int64_t body_limit, AnalysisDims d, uint32_t* err,
                     cudaStream_t s);
void launch_add_offset(int32_t* a, int64_t n, int32_t add, cudaStream_t s);
// lo[i] = lo32[i], hi[i] = hi32[i] for i < m
void launch_widen_bounds(const int32_t* lo32, const int32_t* hi32, int64_t m, int64_t* lo, int64_t* hi,
                         cudaStream_t s);
// rt_batch_capture: checks every rectangle against its graph's own domain and
// moves it into the graph's band (box: int64 [G][3][ndim] = lo, hi, shift)
void launch_band_place(const int32_t* req_off, int32_t n, const int32_t* task_first, int32_t G, const int64_t* box,
                       int D, int64_t* lo, int64_t* hi, int64_t R, uint32_t* err, cudaStream_t s);
void launch_bin_count(const int32_t* req_off, int32_t n, const int64_t* lo, const int64_t* hi,
                      int64_t R, AnalysisDims d, int32_t* rect_task, uint64_t* cnt, cudaStream_t s);
void launch_bin_expand(const int32_t* rect_task, const int64_t* lo, const int64_t* hi,
                       const uint8_t* priv, int64_t R, const uint64_t* off, AnalysisDims d,
                       uint32_t* keys, uint64_t* payload, cudaStream_t s);
void launch_segments(const uint32_t* keys, int64_t M, uint32_t* seg_begin, uint32_t* seg_end,
                     cudaStream_t s);
struct SweepOut {
  uint64_t* pairs;
  unsigned long long cap;
  unsigned long long* cursor;
  uint32_t* tile_counter;
  int key_bits;
  uint32_t chunk;  // pairs a warp reserves at a time (its last chunk may keep holes)
  const uint8_t* only;       // non-null: sweep only the tiles flagged here
  uint8_t* flag_out;         // non-null: flag the tiles that dropped a pair
  unsigned long long* rerun; // pairs emitted by the tiles that dropped one
  // optional, dense inputs: a direct-mapped table of 2^filt_bits pair keys
  // (kEmpty64 = free) through which the flushes of a first sweep pass their
  // keys; a key found there was emitted before and is not written again. Lossy
  // only towards keeping duplicates (a slot keeps the last key that reached
  // it); never set for a rerun, whose tiles must write every pair they find.
  unsigned long long* filt;
  int filt_bits;
};
int sweep_warps_per_block(int tw, int th);
size_t sweep_smem_bytes(int tw, int th, int warps);
void launch_sweep(const uint64_t* payload, const uint32_t* seg_begin, const uint32_t* seg_end,
                  AnalysisDims d, SweepOut o, int blocks, cudaStream_t s);
void launch_explicit_pairs(const int32_t* pred_off, const int32_t* pred, int32_t n, int key_bits,
                           uint64_t* pairs, cudaStream_t s);
void launch_unique_flags(const uint64_t* keys, int64_t P, uint32_t* flags, cudaStream_t s);
void launch_emit_csr(const uint64_t* keys, const uint32_t* flags, const uint32_t* upos, int64_t P,
                     int key_bits, int32_t* col, int32_t* rowcnt, int32_t* indeg, cudaStream_t s);
// CSR by buckets (rows of at most kBucketMaxRow candidate pairs): pairs
// counted per source and the longest row found (count reads the pair count on
// the device); then scatter into per-source buckets, sort and deduplicate
// every bucket, compact into col[] and in-degrees, row_ptr = scan of the
// distinct counts
constexpr int kBucketMaxRow = 1024;
void launch_bucket_count(const uint64_t* pairs, const unsigned long long* cursor, unsigned long long cap,
                         int key_bits, uint32_t* cnt, int32_t n, uint32_t* maxrow, cudaStream_t s);
void launch_bucket_build(const uint64_t* pairs, int64_t P, int key_bits, int32_t n, uint32_t* cnt, uint32_t* off,
                         uint32_t* ucnt, uint32_t* big, uint32_t* nbig, uint32_t* bucket, uint32_t* row_ptr,
                         uint32_t* scan_ws, int32_t* col, int32_t* indeg, cudaStream_t s);
void launch_roots(const int32_t* indeg, int32_t n, uint32_t* flags, cudaStream_t s);
void launch_roots_emit(const int32_t* indeg, const uint32_t* pos, int32_t n, int32_t task_base,
                       int32_t graph, uint64_t* root_items, int32_t* count, cudaStream_t s);

// maxdeg (nullable, zeroed by the caller): receives the largest out-degree
void launch_pack_adj(const int32_t* row_ptr, const int32_t* col, const int32_t* indeg, int64_t n, int4* adj,
                     uint32_t* maxdeg, cudaStream_t s);
void launch_pack_adjx(const int32_t* row_ptr, const int32_t* col, int64_t n, int4* adjx, cudaStream_t s);
void launch_fill_task_graph(const ExecGraph* graphs, int32_t G, int32_t* out, cudaStream_t s);
void launch_max_outdeg(const int32_t* row_ptr, int64_t n, uint32_t* out, cudaStream_t s);
void launch_reset_counts(int32_t* count, const int32_t* indeg, int64_t n, int32_t hold_task,
                         int32_t hold_extra, cudaStream_t s);
void launch_rebase_roots(const uint64_t* src, uint64_t* dst, int32_t n, int32_t graph, int32_t task_base,
                         cudaStream_t s);
void launch_seed(ExecParams p, int64_t ring_clear, cudaStream_t s);
void launch_exec(ExecParams p, int blocks, int warps, cudaStream_t s);
int exec_max_blocks_per_sm(int warps);
rt_status microbench(double* out, int n_out, cudaStream_t s, const char** why);
void launch_serve_init(ServeParams p, cudaStream_t s);
void preload_primitives();
// Loads every kernel of the library (cudaFuncGetAttributes on each). With
// CUDA's lazy module loading, a kernel's first launch may wait for the device
// to go idle; a resident kernel (the serving kernel) never lets it, so
// everything is loaded before one starts. Each file's preload_* lists all of
// its kernels (a CPU test checks this against the sources).
void preload_all();
void preload_microbench();
void preload_static();
void preload_stitch();
void preload_analysis();
void preload_sweep();
void preload_exec();
void preload_serve();
// the event-based executor (rt_execute_events)
struct EvCtrl {  // hot words on separate 128-byte lines
  uint32_t reg, pad0[31];    // launches registered (claims of 32)
  uint32_t pool, pad1[31];   // waiter nodes allocated
  uint32_t rhead, pad2[31];  // ring tickets claimed
  uint32_t rtail, pad3[31];  // ring slots filled
  uint32_t done, pad4[31];   // tasks executed
  uint32_t status, pad5[31];
};
struct EvParams {
  const int32_t* pred_off;  // in-edges: pred[pred_off[v] .. pred_off[v+1])
  const int32_t* pred;
  int32_t n;
  uint32_t ring_cap;
  uint32_t* head;           // per task's completion event: its waiter list (or nil / triggered)
  int32_t* pending;         // per task: events not yet triggered (+1 while registering)
  uint32_t* node_task;      // waiter nodes
  uint32_t* node_next;
  uint32_t* ring;           // ready tasks
  EvCtrl* ctrl;
  ExecGraph G;
  int64_t timeout_ns;
  int32_t claim;            // ring tickets a warp claims at once (1..32), one per lane
};
void launch_ev_transpose(const int32_t* row_ptr, const int32_t* col, int32_t n, const int32_t* pred_off,
                         int32_t* cursor, int32_t* pred, cudaStream_t s);
void launch_events(const EvParams& p, int blocks, cudaStream_t s);
void preload_events();
// stitched replay (rt_execute_stitched): R replays of one trace, joined by
// the edges from one copy of it to the next
struct StitchParams {
  const int4* adj;     // trigger records of the two-copy graph (the first copy's are used)
  const int32_t* col;  // its CSR targets (>= n: task target - n of the next replay)
  int32_t* count;      // [R][n] countdown counters
  uint64_t* ring;      // ready items (replay << 32 | task), R * n slots
  uint32_t ring_cap;
  int32_t n, R;        // tasks per replay, replays
  int32_t claim, keep;
  int64_t total;       // R * n
  ExecCtrl* ctrl;
  int32_t* tickets;    // [R][n][2] start / end tickets, or null
  ExecGraph G;         // bodies of the first copy; out indexed by replay * n + task
  int64_t timeout_ns;
};
void launch_stitch_check(const int32_t* req_off, const int64_t* lo, const int64_t* hi, const uint8_t* priv, int D,
                         const int32_t* row_ptr, const int32_t* col, int32_t n, uint32_t* err, cudaStream_t s);
void launch_stitch(const StitchParams& p, const int32_t* indeg, const uint64_t* root_items, const uint32_t* rootpos,
                   int blocks, int warps, bool tickets, bool fence, cudaStream_t s);
// tasks as whole kernels (rt_execute_kernels)
void* task_kernel_fn();
void launch_task_kernel(int32_t v, const int32_t* pred_off, const int32_t* pred, int32_t* depth, float* sink,
                        int32_t iters, int threads, cudaStream_t s);
void preload_task_kernel();
// stacked batches (rt_batch_create_stacked)
void launch_tag_roots(const uint64_t* src, uint64_t* dst, int64_t n, const uint32_t* root_first, int32_t G,
                      cudaStream_t s);
void launch_check_stacked(const int32_t* row_ptr, const int32_t* col, int64_t T, const uint32_t* task_first,
                          int32_t G, uint32_t* bad, cudaStream_t s);
// out[2i] = rootpos[idx[i]], out[2i+1] = row_ptr[idx[i]] for i < k
void launch_serve_gather(const uint32_t* rootpos, const int32_t* row_ptr, const int32_t* idx, int k, uint32_t* out,
                         cudaStream_t s);
void set_last_error(const char* msg);
void launch_serve(ServeParams p, int blocks, int warps, cudaStream_t s);

// what the serving host code needs to know about an analysed graph
struct GraphView {
  const int32_t* req_off;   // the launches as appended (device)
  const int64_t* lo;
  const int64_t* hi;
  const uint8_t* priv;
  const int4* adj;
  const int32_t* col;
  const int32_t* row_ptr;   // int32[n+1]
  const uint32_t* rootpos;  // int32[n+1]: roots before each task (exclusive scan)
  int32_t* count;
  const uint64_t* roots;
  int32_t n, n_roots;
  int64_t n_edges;
  size_t footprint;  // bytes of device memory the graph object holds
};
rt_status graph_view(rt_graph_t g, GraphView* v);
// device bytes the graph's buffers hold (the sum of their capacities)
size_t graph_footprint(rt_graph_t g);
// caps the device bytes the graph may hold while its buffers grow (0 = none):
// a growth past the cap fails with RT_ERR_BUDGET and allocates nothing
void graph_set_mem_cap(rt_graph_t g, size_t cap);
// releases every device buffer of the graph (stream-ordered) and clears it
rt_status graph_trim(rt_graph_t g);
rt_status batch_shape(rt_batch_t b, int64_t* graphs, int64_t* tasks, int64_t* edges);
int32_t static_max_tasks();
rt_status static_execute(const int32_t* row_ptr, const int32_t* col, const int32_t* indeg, int32_t n,
                         int64_t n_edges, int32_t spin_iters, int32_t* out, int32_t* tickets, cudaStream_t s,
                         int64_t timeout_ns, const char** why);

}  // namespace grt
