// api.cu -- host orchestration behind the C ABI of grt.h.
//
// Owns every library buffer, validates inputs, sequences the analysis and
// execution kernels on the graph's stream, caches CUDA graphs for replays and
// builds batches. Nothing here computes the method's results: all of that
// runs in the kernels of analysis.cu, sweep.cu, primitives.cu, exec.cu,
// static_exec.cu, events.cu, kernels.cu and serve.cu.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cstdarg>
#include <mutex>
#include <cstdio>
#include <cstdlib>
#include <time.h>
#include <cstring>
#include <string>
#include <vector>

#include "grt_internal.cuh"

using namespace grt;

namespace {

thread_local std::string g_err;

rt_status fail(rt_status s, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_err = buf;
  return s;
}

#define CK(call)                                                                             \
  do {                                                                                       \
    cudaError_t e_ = (call);                                                                 \
    if (e_ != cudaSuccess) return fail(RT_ERR_CUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
  } while (0)

#define CKR(call)                           \
  do {                                      \
    rt_status r_ = (call);                  \
    if (r_ != RT_OK) return r_;             \
  } while (0)

// A graph whose device bytes are capped (the server gives each batch graph a
// share of its memory budget): while a call grows that graph's buffers on this
// thread, every growth that would take the graph past its cap fails with
// RT_ERR_BUDGET instead of allocating. Null: no cap applies.
thread_local const rt_graph* t_capped = nullptr;
bool over_cap(size_t grow_by);  // defined after rt_graph

// grow-only device buffer, allocated stream-ordered on its owner's stream:
// cudaMallocAsync / cudaFreeAsync never wait for work on other streams (a
// plain cudaFree would wait for the whole device, including a serving kernel
// that runs for the life of a server)
struct DevBuf {
  void* p = nullptr;
  size_t cap = 0;
  rt_status reserve(size_t bytes, cudaStream_t s, size_t keep = 0) {
    if (bytes <= cap && p) return RT_OK;
    size_t nc = std::max<size_t>(bytes, keep ? cap * 2 : bytes);
    nc = std::max<size_t>(nc, 256);
    // the old buffer is freed only after the new one exists (and, with `keep`,
    // after the copy), so the graph briefly holds both
    if (t_capped && over_cap(nc))
      return fail(RT_ERR_BUDGET, "growing a buffer to %zu bytes would pass the graph's memory cap", nc);
    void* np = nullptr;
    cudaError_t e = cudaMallocAsync(&np, nc, s);
    if (e != cudaSuccess) {
      cudaGetLastError();
      return fail(RT_ERR_OOM, "cudaMallocAsync(%zu bytes): %s", nc, cudaGetErrorString(e));
    }
    if (keep && p) {
      e = cudaMemcpyAsync(np, p, keep, cudaMemcpyDeviceToDevice, s);
      if (e != cudaSuccess) return fail(RT_ERR_CUDA, "grow copy: %s", cudaGetErrorString(e));
    }
    if (p) cudaFreeAsync(p, s);  // ordered after the copy on the same stream
    p = np;
    cap = nc;
    return RT_OK;
  }
  void release(cudaStream_t s) {
    if (p) cudaFreeAsync(p, s);
    p = nullptr;
    cap = 0;
  }
  template <class T>
  T* as() const {
    return reinterpret_cast<T*>(p);
  }
};

struct DeviceInfo {
  bool init = false;
  int device = -1, num_sms = 0, exec_bps = 0;
};
DeviceInfo g_dev;
std::mutex g_dev_mu;

rt_status ensure_device() {
  int dev = -1;
  CK(cudaGetDevice(&dev));
  std::lock_guard<std::mutex> lk(g_dev_mu);
  if (g_dev.init && g_dev.device == dev) return RT_OK;
  cudaDeviceProp prop;
  CK(cudaGetDeviceProperties(&prop, dev));
  g_dev.device = dev;
  g_dev.num_sms = prop.multiProcessorCount;
  g_dev.exec_bps = exec_max_blocks_per_sm(8);
  if (g_dev.exec_bps < 1) g_dev.exec_bps = 1;
  g_dev.init = true;
  return RT_OK;
}

int bits_for(uint64_t v) {  // smallest b with 2^b > v
  int b = 0;
  while (b < 63 && (1ull << b) <= v) ++b;
  return b;
}

enum { EV_A0 = 0, EV_BIN, EV_SORTE, EV_SWEEP, EV_SORTP, EV_CSR, EV_X0, EV_XK0, EV_XK1, EV_SW0, EV_SW1, EV_E0, EV_E1,
       EV_COUNT };

}  // namespace

struct rt_graph {
  rt_graph_desc desc{};
  cudaStream_t s = nullptr;
  AnalysisDims dims{};
  int64_t ncells = 0;
  int32_t n = 0;
  int64_t R = 0, P = 0;
  bool has_pred = false, has_body_arg = false;
  DevBuf req_off, lo, hi, priv, pred_off, pred, body_arg;
  DevBuf stage32;  // rt_launch_batch32: the int32 bounds on their way to lo and hi
  DevBuf err;  // uint32 device-side validation bits
  bool pending_validate = false;
  // analysis
  DevBuf rect_task, cnt, keys, keys_alt, pay, pay_alt, seg_b, seg_e, pairs, pairs_alt, flags, upos;
  DevBuf col, row_ptr, indeg, count, rootpos, root_items, ws, misc, adj;
  DevBuf adjx;          // the owned executor's extension records, built on its first run after an analysis
  bool adjx_ok = false;
  int32_t max_outdeg = 0;  // largest out-degree of the analysed graph
  DevBuf tflags;  // per tile: dropped a pair in the first sweep / in the rerun
  DevBuf pfilt;   // dense inputs: the first sweep's pair-key filter
  int pair_filter_bits = 0;  // log2 of its slots in the last analysis (0: not used)
  DevBuf bucket;  // CSR by buckets: per-task counts, offsets, distinct counts, long-row list, control words
  // the event-based executor (rt_execute_events): in-edges, events, waiter nodes
  DevBuf ev_pred_off, ev_pred, ev_head, ev_pending, ev_nodes, ev_ring, ev_ctrl;
  bool ev_preds = false;  // in-edges built for the current analysis
  // rt_execute_kernels: the DAG on the host, events and streams, the CUDA graph
  std::vector<int32_t> kh_rp, kh_col, kh_poff, kh_pred;
  bool kh_valid = false;
  std::vector<cudaEvent_t> kevents;
  std::vector<cudaStream_t> kstreams;
  cudaGraph_t kg = nullptr;
  cudaGraphExec_t kg_exec = nullptr;
  int32_t kg_iters = -1, kg_threads = -1;
  DevBuf ksink;
  // rt_execute_stitched: per-replay counters, ready ring, control, tickets
  DevBuf st_count, st_ring, st_ctrl, st_tickets, st_err;
  int32_t st_R = 0;  // replays of the last stitched run with tickets
  // execution
  DevBuf ring, ctrl, gtable, done_g, tickets;
  uint32_t* hpin = nullptr;  // pinned readback area (64 words)
  bool analyzed = false, dirty = false, status_pending = false;
  int64_t n_edges = 0, n_roots = 0, n_entries = 0, n_pairs = 0;
  int32_t hold_task = -1, hold_extra = 0;
  cudaGraphExec_t replay_exec = nullptr;
  int32_t replay_times = 0;
  cudaStream_t cap_stream = nullptr;
  cudaEvent_t ev[EV_COUNT] = {};
  bool ev_ok = false, analyze_timed = false, exec_timed = false;
  ExecGraph gt_host{};  // last table entry written to gtable
  bool gt_valid = false;
  int exec_blocks = 0, exec_warps = 8;
  int cfg_blocks = 0, cfg_warps = 0, cfg_claim = 0, cfg_keep = 0;  // rt_graph_exec_config
  size_t mem_cap = 0;  // device bytes the graph may hold while it grows (0 = no cap; set by a server)
  int cfg_policy = RT_EXEC_RING;  // rt_graph_exec_policy
  bool csr_by_buckets = false;    // the last analysis built its CSR from buckets, not the pair sort
};

namespace {
// every device buffer a graph holds (its footprint is the sum of their capacities)
template <class G, class F>
void for_each_buf(G* g, F f) {
  auto bufs = {&g->req_off, &g->lo, &g->hi, &g->priv, &g->pred_off, &g->pred, &g->body_arg, &g->stage32, &g->err,
                &g->rect_task, &g->cnt, &g->keys, &g->keys_alt, &g->pay, &g->pay_alt, &g->seg_b, &g->seg_e,
                &g->pairs, &g->pairs_alt, &g->flags, &g->upos, &g->col, &g->row_ptr, &g->indeg, &g->count,
                &g->rootpos, &g->root_items, &g->ws, &g->misc, &g->adj, &g->adjx, &g->bucket, &g->ring, &g->ctrl,
                &g->gtable, &g->done_g, &g->tickets, &g->tflags, &g->pfilt, &g->ev_pred_off, &g->ev_pred,
                &g->ev_head, &g->ev_pending, &g->ev_nodes, &g->ev_ring, &g->ev_ctrl, &g->ksink, &g->st_count,
                &g->st_ring, &g->st_ctrl, &g->st_tickets, &g->st_err};
  for (auto* b : bufs) f(*b);
}

size_t footprint_of(const rt_graph* g) {
  size_t f = 0;
  for_each_buf(g, [&](const DevBuf& b) { f += b.cap; });
  return f;
}

bool over_cap(size_t grow_by) { return footprint_of(t_capped) + grow_by > t_capped->mem_cap; }

// applies the graph's memory cap to the buffers this thread grows until the
// scope ends
struct CapScope {
  const rt_graph* saved;
  explicit CapScope(const rt_graph* g) : saved(t_capped) { t_capped = g->mem_cap ? g : nullptr; }
  ~CapScope() { t_capped = saved; }
};
}  // namespace

struct rt_batch {
  cudaStream_t s = nullptr;
  int32_t G = 0, G_nonempty = 0;
  int64_t T = 0, E = 0, Rtot = 0;
  DevBuf row_ptr, col, indeg, count, root_items, gtable, done_g, ring, ctrl, adj;
  uint32_t* hpin = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  bool dirty = false;
  int need_fence = 0;
  // the launch as a CUDA graph {counter reset, seed, executor, status
  // read-back}, instantiated once per launch shape and relaunched
  cudaGraphExec_t gexec = nullptr;
  int64_t gkey[7] = {0, 0, 0, 0, 0, 0, 0};
  cudaStream_t cap_stream = nullptr;
  int64_t graph_launches = 0;  // launches that went through the cached CUDA graph
  rt_graph* owned = nullptr;   // rt_batch_capture: the stacked graph it analysed
  // the owned-chunk policy (rt_batch_exec_policy): each task's graph, the
  // extension records (only when some task has more than kAdjInline
  // successors), built on the first owned launch
  int policy = RT_EXEC_RING;
  DevBuf task_graph, adjx, scratch;
  bool owned_ready = false;
  int32_t max_outdeg = 0;
};

namespace {

rt_status graph_events(rt_graph* g) {
  if (g->ev_ok) return RT_OK;
  for (int i = 0; i < EV_COUNT; ++i) CK(cudaEventCreate(&g->ev[i]));
  g->ev_ok = true;
  return RT_OK;
}

void drop_replay_graph(rt_graph* g) {
  if (g->replay_exec) cudaGraphExecDestroy(g->replay_exec);
  g->replay_exec = nullptr;
  g->replay_times = 0;
}

void drop_kernel_graph(rt_graph* g) {
  if (g->kg_exec) cudaGraphExecDestroy(g->kg_exec);
  if (g->kg) cudaGraphDestroy(g->kg);
  g->kg_exec = nullptr;
  g->kg = nullptr;
  g->kg_iters = g->kg_threads = -1;
}

rt_status check_desc(const rt_graph_desc* d, AnalysisDims* out, int64_t* ncells) {
  if (!d) return fail(RT_ERR_INVALID, "desc is NULL");
  if (d->ndim != 1 && d->ndim != 2) return fail(RT_ERR_INVALID, "ndim must be 1 or 2 (got %d)", d->ndim);
  AnalysisDims a{};
  a.ndim = d->ndim;
  for (int k = 0; k < 2; ++k) {
    if (k < d->ndim) {
      if (d->dom_lo[k] > d->dom_hi[k]) return fail(RT_ERR_INVALID, "dom_lo[%d] > dom_hi[%d]", k, k);
      a.dom_lo[k] = d->dom_lo[k];
      a.ext[k] = d->dom_hi[k] - d->dom_lo[k] + 1;
      if (a.ext[k] <= 0 || a.ext[k] > (1ll << 40)) return fail(RT_ERR_INVALID, "domain extent out of range");
    } else {
      a.dom_lo[k] = 0;
      a.ext[k] = 1;
    }
  }
  if (d->body < RT_BODY_EMPTY || d->body > RT_BODY_FMA) return fail(RT_ERR_INVALID, "unknown body %d", d->body);
  if (d->spin_iters < 0) return fail(RT_ERR_INVALID, "spin_iters < 0");
  if (d->state_elems < 0 || d->out_elems < 0 || d->timeout_ns < 0)
    return fail(RT_ERR_INVALID, "negative size");
  if (d->tile_w < 0 || d->tile_h < 0) return fail(RT_ERR_INVALID, "negative tile");
  if (d->ndim == 2) {
    a.tw = d->tile_w ? d->tile_w : 16;
    a.th = d->tile_h ? d->tile_h : 16;
    if (a.tw > kMaxTileSide2D || a.th > kMaxTileSide2D)
      return fail(RT_ERR_INVALID, "2-D tile sides must be <= %d", kMaxTileSide2D);
  } else {
    a.tw = d->tile_w ? d->tile_w : 1024;
    a.th = 1;
    if (d->tile_h > 1) return fail(RT_ERR_INVALID, "1-D graphs have tile_h 1");
    if (a.tw > kMaxTileSide1D) return fail(RT_ERR_INVALID, "1-D tile must be <= %d", kMaxTileSide1D);
  }
  // 2-D tiles larger than the per-warp cell state are swept in strips of
  // column/row classes; a 1-D tile's classes must fit it at once
  if (a.th == 1 && a.tw > kMaxClassCells) return fail(RT_ERR_INVALID, "1-D tile must be <= %d", kMaxClassCells);
  int64_t ntx = (a.ext[0] + a.tw - 1) / a.tw, nty = (a.ext[1] + a.th - 1) / a.th;
  if (ntx * nty > (1ll << 26)) return fail(RT_ERR_INVALID, "domain has more than 2^26 tiles; use a larger tile");
  a.ntx = (int)ntx;
  a.nty = (int)nty;
  int64_t cells = a.ext[0] * a.ext[1];
  if (d->body == RT_BODY_CHECK) {
    if (!d->state || d->state_elems < cells)
      return fail(RT_ERR_INVALID, "CHECK body needs state with one int32 per cell (%lld)", (long long)cells);
    if (cells > (1ll << 32)) return fail(RT_ERR_INVALID, "CHECK body needs at most 2^32 cells");
  }
  if (d->body == RT_BODY_COUNTER && (!d->state || d->state_elems <= 0))
    return fail(RT_ERR_INVALID, "COUNTER body needs a state buffer");
  *out = a;
  *ncells = cells;
  return RT_OK;
}

}  // namespace

extern "C" {

const char* rt_last_error(void) { return g_err.c_str(); }

rt_status rt_device_info(int32_t* num_sms, int32_t* exec_blocks_per_sm) {
  CKR(ensure_device());
  if (num_sms) *num_sms = g_dev.num_sms;
  if (exec_blocks_per_sm) *exec_blocks_per_sm = g_dev.exec_bps;
  return RT_OK;
}

rt_status rt_graph_create(const rt_graph_desc* desc, rt_graph_t* out) {
  if (!out) return fail(RT_ERR_INVALID, "out is NULL");
  *out = nullptr;
  AnalysisDims a;
  int64_t cells;
  CKR(check_desc(desc, &a, &cells));
  rt_graph* g = new (std::nothrow) rt_graph();
  if (!g) return fail(RT_ERR_OOM, "host allocation failed");
  g->desc = *desc;
  if (g->desc.timeout_ns == 0) g->desc.timeout_ns = 2000000000ll;
  g->s = (cudaStream_t)desc->stream;
  g->dims = a;
  g->ncells = cells;
  *out = g;
  return RT_OK;
}

rt_status rt_graph_clear(rt_graph_t g) {
  if (!g) return fail(RT_ERR_INVALID, "graph is NULL");
  g->n = 0;
  g->R = 0;
  g->P = 0;
  g->has_pred = g->has_body_arg = false;
  g->pending_validate = false;
  g->analyzed = false;
  g->dirty = false;
  g->n_edges = g->n_roots = g->n_entries = g->n_pairs = 0;
  g->hold_task = -1;
  drop_replay_graph(g);
  return RT_OK;
}

rt_status rt_graph_destroy(rt_graph_t g) {
  if (!g) return RT_OK;
  if (g->ev_ok || g->ring.p || g->req_off.p) cudaStreamSynchronize(g->s);
  drop_replay_graph(g);
  drop_kernel_graph(g);
  for (cudaStream_t st : g->kstreams) {
    cudaStreamSynchronize(st);
    cudaStreamDestroy(st);
  }
  for (cudaEvent_t e : g->kevents) cudaEventDestroy(e);
  for_each_buf(g, [&](DevBuf& b) { b.release(g->s); });
  cudaStreamSynchronize(g->s);
  if (g->hpin) cudaFreeHost(g->hpin);
  if (g->ev_ok)
    for (int i = 0; i < EV_COUNT; ++i) cudaEventDestroy(g->ev[i]);
  if (g->cap_stream) cudaStreamDestroy(g->cap_stream);
  delete g;
  return RT_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// launch ingest
// ---------------------------------------------------------------------------
namespace {

// T: the coordinate type of lo and hi (int64_t, or int32_t for rt_launch_batch32)
template <class T>
rt_status host_validate(const rt_graph* g, int32_t n, const int32_t* req_off, const T* lo, const T* hi,
                        const uint8_t* priv, const int32_t* pred_off, const int32_t* pred,
                        const int32_t* body_arg) {
  const AnalysisDims& d = g->dims;
  if (req_off[0] != 0) return fail(RT_ERR_INVALID, "req_off[0] must be 0 (got %d)", req_off[0]);
  for (int32_t i = 0; i < n; ++i)
    if (req_off[i + 1] < req_off[i]) return fail(RT_ERR_INVALID, "req_off decreases at launch %d", i);
  const int64_t R = req_off[n];
  for (int64_t r = 0; r < R; ++r) {
    for (int k = 0; k < d.ndim; ++k) {
      const int64_t a = lo[r * d.ndim + k], b = hi[r * d.ndim + k];
      if (a > b) return fail(RT_ERR_INVALID, "rect %lld: lo > hi in dim %d", (long long)r, k);
      if (a < d.dom_lo[k] || b > d.dom_lo[k] + d.ext[k] - 1)
        return fail(RT_ERR_INVALID, "rect %lld outside the domain in dim %d", (long long)r, k);
    }
    if (priv[r] > 2) return fail(RT_ERR_INVALID, "rect %lld: privilege %d", (long long)r, (int)priv[r]);
  }
  if (pred_off) {
    if (pred_off[0] != 0) return fail(RT_ERR_INVALID, "pred_off[0] must be 0");
    for (int32_t i = 0; i < n; ++i) {
      if (pred_off[i + 1] < pred_off[i]) return fail(RT_ERR_INVALID, "pred_off decreases at launch %d", i);
      for (int32_t k = pred_off[i]; k < pred_off[i + 1]; ++k)
        if (pred[k] < 0 || pred[k] >= g->n + i)
          return fail(RT_ERR_INVALID, "launch %d: predecessor %d is not an earlier task", g->n + i, pred[k]);
    }
  }
  if (body_arg && g->desc.body == RT_BODY_COUNTER)
    for (int32_t i = 0; i < n; ++i)
      if (body_arg[i] < 0 || (int64_t)body_arg[i] >= g->desc.state_elems)
        return fail(RT_ERR_INVALID, "launch %d: body_arg %d outside the state buffer", g->n + i, body_arg[i]);
  return RT_OK;
}

rt_status copy_in(void* dst, const void* src, size_t bytes, cudaStream_t s) {
  if (!bytes) return RT_OK;
  CK(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDefault, s));
  return RT_OK;
}

rt_status ensure_pinned(rt_graph* g) {
  if (g->hpin) return RT_OK;
  CK(cudaMallocHost(&g->hpin, 1024));
  return RT_OK;
}

}  // namespace

namespace {
// rt_batch_capture's placement of graphs in bands, applied to the launches of
// a fresh graph between their copy and their validation
struct BandPlace {
  const int32_t* task_first;  // device int32[G+1]: graph k owns tasks [task_first[k], task_first[k+1])
  int32_t G;
  const int64_t* box;         // device int64[G][3][ndim]: its domain's lo, hi and its shift
};

// lo and hi are int64[R][ndim], or int32[R][ndim] with c32 (widened on the device)
rt_status append_launches(rt_graph_t g, int32_t n, const int32_t* req_off, const void* lo, const void* hi,
                          const uint8_t* priv, const int32_t* pred_off, const int32_t* pred, const int32_t* body_arg,
                          int32_t flags, const BandPlace* bp, bool c32 = false);
}  // namespace

extern "C" rt_status rt_launch_batch(rt_graph_t g, int32_t n, const int32_t* req_off, const int64_t* lo,
                                     const int64_t* hi, const uint8_t* priv, const int32_t* pred_off,
                                     const int32_t* pred, const int32_t* body_arg, int32_t flags) {
  return append_launches(g, n, req_off, lo, hi, priv, pred_off, pred, body_arg, flags, nullptr);
}

extern "C" rt_status rt_launch_batch32(rt_graph_t g, int32_t n, const int32_t* req_off, const int32_t* lo,
                                       const int32_t* hi, const uint8_t* priv, const int32_t* pred_off,
                                       const int32_t* pred, const int32_t* body_arg, int32_t flags) {
  return append_launches(g, n, req_off, lo, hi, priv, pred_off, pred, body_arg, flags, nullptr, true);
}

namespace {
rt_status append_launches(rt_graph_t g, int32_t n, const int32_t* req_off, const void* lo, const void* hi,
                          const uint8_t* priv, const int32_t* pred_off, const int32_t* pred, const int32_t* body_arg,
                          int32_t flags, const BandPlace* bp, bool c32) {
  if (!g) return fail(RT_ERR_INVALID, "graph is NULL");
  if (g->analyzed) return fail(RT_ERR_STATE, "graph already analyzed; call rt_graph_clear first");
  if (n < 0) return fail(RT_ERR_INVALID, "n < 0");
  CapScope cap_scope(g);
  if (n == 0) return RT_OK;
  if (!req_off) return fail(RT_ERR_INVALID, "req_off is NULL");
  if ((pred_off == nullptr) != (pred == nullptr))
    return fail(RT_ERR_INVALID, "pred_off and pred must both be set or both be NULL");
  if (g->desc.body == RT_BODY_COUNTER && !body_arg)
    return fail(RT_ERR_INVALID, "COUNTER body needs body_arg");
  if (flags & ~(RT_LAUNCH_DEVICE | RT_LAUNCH_DEFER_CHECK)) return fail(RT_ERR_INVALID, "unknown flags");
  if ((int64_t)g->n + n >= (int64_t)INT32_MAX) return fail(RT_ERR_INVALID, "too many tasks");
  const bool dev = (flags & RT_LAUNCH_DEVICE) != 0;
  const bool on_device_check = dev || (flags & RT_LAUNCH_DEFER_CHECK);
  const int D = g->dims.ndim;
  int64_t R = 0, Pb = 0;
  int32_t first[2] = {0, 0};
  if (!dev) {
    R = req_off[n];
    Pb = pred_off ? pred_off[n] : 0;
    first[0] = req_off[0];
    first[1] = pred_off ? pred_off[0] : 0;
    if (R < 0 || Pb < 0) return fail(RT_ERR_INVALID, "negative rect or pred count");
    if (R > 0 && (!lo || !hi || !priv)) return fail(RT_ERR_INVALID, "rect arrays are NULL");
    if (!on_device_check) {
      if (c32)
        CKR(host_validate(g, n, req_off, static_cast<const int32_t*>(lo), static_cast<const int32_t*>(hi), priv,
                          pred_off, pred, body_arg));
      else
        CKR(host_validate(g, n, req_off, static_cast<const int64_t*>(lo), static_cast<const int64_t*>(hi), priv,
                          pred_off, pred, body_arg));
    }
  }
  CKR(ensure_device());
  CKR(ensure_pinned(g));
  cudaStream_t s = g->s;
  if (dev) {
    // the batch's sizes live on the device: read both ends of the offset arrays
    CK(cudaMemcpyAsync(g->hpin + 0, req_off, 4, cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(g->hpin + 1, req_off + n, 4, cudaMemcpyDeviceToHost, s));
    if (pred_off) {
      CK(cudaMemcpyAsync(g->hpin + 2, pred_off, 4, cudaMemcpyDeviceToHost, s));
      CK(cudaMemcpyAsync(g->hpin + 3, pred_off + n, 4, cudaMemcpyDeviceToHost, s));
    }
    CK(cudaStreamSynchronize(s));
    first[0] = (int32_t)g->hpin[0];
    R = (int32_t)g->hpin[1];
    first[1] = pred_off ? (int32_t)g->hpin[2] : 0;
    Pb = pred_off ? (int32_t)g->hpin[3] : 0;
    if (R < 0 || Pb < 0) return fail(RT_ERR_INVALID, "negative rect or pred count");
    if (R > 0 && (!lo || !hi || !priv)) return fail(RT_ERR_INVALID, "rect arrays are NULL");
  }
  if (first[0] != 0) return fail(RT_ERR_INVALID, "req_off[0] must be 0");
  if (first[1] != 0) return fail(RT_ERR_INVALID, "pred_off[0] must be 0");
  if (g->R + R >= (int64_t)INT32_MAX || g->P + Pb >= (int64_t)INT32_MAX)
    return fail(RT_ERR_INVALID, "too many rects or preds");
  trace("launch_batch: validated");

  const int32_t n0 = g->n;
  const int64_t R0 = g->R, P0 = g->P;
  // offsets: position 0 of the batch is the previous end, so copy [1..n]
  CKR(g->req_off.reserve((size_t)(n0 + n + 1) * 4, s, (size_t)(n0 + 1) * 4));
  if (n0 == 0) CK(cudaMemsetAsync(g->req_off.p, 0, 4, s));
  CKR(copy_in(g->req_off.as<int32_t>() + n0 + 1, req_off + 1, (size_t)n * 4, s));
  launch_add_offset(g->req_off.as<int32_t>() + n0 + 1, n, (int32_t)R0, s);
  if (R > 0) {
    CKR(g->lo.reserve((size_t)(R0 + R) * D * 8, s, (size_t)R0 * D * 8));
    CKR(g->hi.reserve((size_t)(R0 + R) * D * 8, s, (size_t)R0 * D * 8));
    CKR(g->priv.reserve((size_t)(R0 + R), s, (size_t)R0));
    if (c32) {
      // the int32 bounds through a staging buffer, widened into the graph's arrays
      CKR(g->stage32.reserve((size_t)R * D * 8, s));
      int32_t* st = g->stage32.as<int32_t>();
      CKR(copy_in(st, lo, (size_t)R * D * 4, s));
      CKR(copy_in(st + R * D, hi, (size_t)R * D * 4, s));
      launch_widen_bounds(st, st + R * D, R * D, g->lo.as<int64_t>() + R0 * D, g->hi.as<int64_t>() + R0 * D, s);
    } else {
      CKR(copy_in(g->lo.as<int64_t>() + R0 * D, lo, (size_t)R * D * 8, s));
      CKR(copy_in(g->hi.as<int64_t>() + R0 * D, hi, (size_t)R * D * 8, s));
    }
    CKR(copy_in(g->priv.as<uint8_t>() + R0, priv, (size_t)R, s));
  }
  if (pred_off || g->has_pred) {
    CKR(g->pred_off.reserve((size_t)(n0 + n + 1) * 4, s, g->has_pred ? (size_t)(n0 + 1) * 4 : 0));
    if (!g->has_pred) CK(cudaMemsetAsync(g->pred_off.p, 0, (size_t)(n0 + 1) * 4, s));
    int32_t* po = g->pred_off.as<int32_t>() + n0 + 1;
    if (pred_off) {
      CKR(copy_in(po, pred_off + 1, (size_t)n * 4, s));
    } else {
      CK(cudaMemsetAsync(po, 0, (size_t)n * 4, s));
    }
    launch_add_offset(po, n, (int32_t)P0, s);
    if (Pb > 0) {
      CKR(g->pred.reserve((size_t)(P0 + Pb) * 4, s, (size_t)P0 * 4));
      CKR(copy_in(g->pred.as<int32_t>() + P0, pred, (size_t)Pb * 4, s));
    }
    g->has_pred = true;
  }
  if (body_arg || g->has_body_arg) {
    CKR(g->body_arg.reserve((size_t)(n0 + n) * 4, s, g->has_body_arg ? (size_t)n0 * 4 : 0));
    if (!g->has_body_arg && n0) CK(cudaMemsetAsync(g->body_arg.p, 0, (size_t)n0 * 4, s));
    if (body_arg) {
      CKR(copy_in(g->body_arg.as<int32_t>() + n0, body_arg, (size_t)n * 4, s));
    } else {
      CK(cudaMemsetAsync(g->body_arg.as<int32_t>() + n0, 0, (size_t)n * 4, s));
    }
    g->has_body_arg = true;
  }
  if (on_device_check) {
    if (!g->err.p) {
      CKR(g->err.reserve(256, s));
      CK(cudaMemsetAsync(g->err.p, 0, 4, s));
    }
    if (bp)  // each rectangle checked against its own graph's domain, then moved into its band
      launch_band_place(g->req_off.as<int32_t>() + n0, n, bp->task_first, bp->G, bp->box, D,
                        g->lo.as<int64_t>() + R0 * D, g->hi.as<int64_t>() + R0 * D, R, g->err.as<uint32_t>(), s);
    const int64_t limit = g->desc.body == RT_BODY_COUNTER ? g->desc.state_elems : -1;
    launch_validate(g->req_off.as<int32_t>() + n0, n, R0, g->lo.as<int64_t>() + R0 * D,
                    g->hi.as<int64_t>() + R0 * D, g->priv.as<uint8_t>() + R0, R,
                    g->has_pred ? g->pred_off.as<int32_t>() + n0 : nullptr, g->pred.as<int32_t>(), P0,
                    P0 + Pb, n0, body_arg ? g->body_arg.as<int32_t>() + n0 : nullptr, limit, g->dims,
                    g->err.as<uint32_t>(), s);
    g->pending_validate = true;
  }
  CK(cudaGetLastError());
  trace("launch_batch: copies enqueued");
  g->n += n;
  g->R += R;
  g->P += Pb;
  return RT_OK;
}
}  // namespace

// ---------------------------------------------------------------------------
// analysis
// ---------------------------------------------------------------------------
namespace {

const char* err_bits_text(uint32_t e) {
  if (e & 32u) return "a rectangle lies outside its own graph's domain";
  if (e & 2u) return "a rectangle has lo > hi or lies outside the domain";
  if (e & 4u) return "a privilege is not read/write/reduce";
  if (e & 1u) return "req_off does not start at 0, decreases, or does not end at the rect count";
  if (e & 8u) return "a predecessor is not an earlier task (or pred_off is malformed)";
  if (e & 16u) return "a body_arg lies outside the state buffer";
  return "invalid launch data";
}

rt_status reserve_ws(rt_graph* g, size_t bytes) { return g->ws.reserve(bytes + 1024, g->s); }

rt_status run_analysis(rt_graph* g) {
  cudaStream_t s = g->s;
  const AnalysisDims& d = g->dims;
  const int32_t n = g->n;
  const int64_t R = g->R;
  const bool prof = (g->desc.flags & RT_GRAPH_PROFILE) != 0;
  if (prof) {
    CKR(graph_events(g));
    CK(cudaEventRecord(g->ev[EV_A0], s));
  }
  const int B = std::max(bits_for((uint64_t)n), 1);  // pair key = src << B | dst
  if (2 * B > 62) return fail(RT_ERR_OOM, "too many tasks for 64-bit pair keys");
  const int64_t ntiles = (int64_t)d.ntx * d.nty;
  trace("analyze: start");
  CKR(g->misc.reserve(256, s));
  trace("analyze: misc reserved");
  unsigned long long* cursor = reinterpret_cast<unsigned long long*>(g->misc.p);
  uint32_t* tile_counter = reinterpret_cast<uint32_t*>(g->misc.as<char>() + 64);
  volatile uint64_t* h64 = reinterpret_cast<volatile uint64_t*>(g->hpin);  // 32 x u64

  // ---- 1-3: binning ------------------------------------------------------
  int64_t M = 0;
  const uint32_t* skeys = nullptr;
  const uint64_t* spay = nullptr;
  if (R > 0) {
    CKR(g->rect_task.reserve((size_t)R * 4, s));
    CKR(g->cnt.reserve((size_t)(R + 1) * 8, s));
    CKR(reserve_ws(g, scan_ws_elems<uint64_t>(R) * 8));
    launch_bin_count(g->req_off.as<int32_t>(), n, g->lo.as<int64_t>(), g->hi.as<int64_t>(), R, d,
                     g->rect_task.as<int32_t>(), g->cnt.as<uint64_t>(), s);
    scan_exclusive<uint64_t>(g->cnt.as<uint64_t>(), g->cnt.as<uint64_t>(), R, g->ws.as<uint64_t>(), s);
    CK(cudaMemcpyAsync((void*)&h64[0], g->cnt.as<uint64_t>() + R, 8, cudaMemcpyDeviceToHost, s));
  }
  h64[1] = 0;
  if (g->pending_validate) CK(cudaMemcpyAsync((void*)&h64[1], g->err.p, 4, cudaMemcpyDeviceToHost, s));
  trace("analyze: bin count enqueued");
  if (R > 0 || g->pending_validate) CK(cudaStreamSynchronize(s));
  trace("analyze: bin count synced");
  if (g->pending_validate && (uint32_t)h64[1] != 0u)
    return fail(RT_ERR_INVALID, "device validation: %s", err_bits_text((uint32_t)h64[1]));
  g->pending_validate = false;
  if (R > 0) M = (int64_t)h64[0];
  if (M >= (1ll << 30)) return fail(RT_ERR_OOM, "%lld tile entries (limit 2^30); use a larger tile", (long long)M);
  g->n_entries = M;
  if (M > 0) {
    CKR(g->keys.reserve((size_t)M * 4, s));
    CKR(g->keys_alt.reserve((size_t)M * 4, s));
    CKR(g->pay.reserve((size_t)M * 8, s));
    CKR(g->pay_alt.reserve((size_t)M * 8, s));
    CKR(g->seg_b.reserve((size_t)ntiles * 4, s));
    CKR(g->seg_e.reserve((size_t)ntiles * 4, s));
    CKR(reserve_ws(g, radix_ws_bytes(M)));
    trace("analyze: entry buffers reserved");
    launch_bin_expand(g->rect_task.as<int32_t>(), g->lo.as<int64_t>(), g->hi.as<int64_t>(),
                      g->priv.as<uint8_t>(), R, g->cnt.as<uint64_t>(), d, g->keys.as<uint32_t>(),
                      g->pay.as<uint64_t>(), s);
    if (prof) CK(cudaEventRecord(g->ev[EV_BIN], s));
    const int tbits = std::max(bits_for((uint64_t)(ntiles - 1)), 1);
    const int flip = radix_sort<uint32_t>(g->keys.as<uint32_t>(), g->keys_alt.as<uint32_t>(),
                                          g->pay.as<uint64_t>(), g->pay_alt.as<uint64_t>(), M, tbits,
                                          g->ws.p, s);
    skeys = flip ? g->keys_alt.as<uint32_t>() : g->keys.as<uint32_t>();
    spay = flip ? g->pay_alt.as<uint64_t>() : g->pay.as<uint64_t>();
    CK(cudaMemsetAsync(g->seg_b.p, 0, (size_t)ntiles * 4, s));
    CK(cudaMemsetAsync(g->seg_e.p, 0, (size_t)ntiles * 4, s));
    launch_segments(skeys, M, g->seg_b.as<uint32_t>(), g->seg_e.as<uint32_t>(), s);
    if (prof) CK(cudaEventRecord(g->ev[EV_SORTE], s));
  } else if (prof) {
    CK(cudaEventRecord(g->ev[EV_BIN], s));
    CK(cudaEventRecord(g->ev[EV_SORTE], s));
  }

  // ---- 4: sweep (+ explicit preds) ---------------------------------------
  const int64_t Pe = g->has_pred ? g->P : 0;
  // Each sweep warp leaves holes in at most its last chunk, so the cursor ends
  // below (pairs written) + (warps x chunk). The chunk is sized to keep that
  // slack near half the first guess. If the buffer overflows, the sweep has
  // flagged the tiles that dropped a pair and counted the pairs they emit;
  // the buffer grows by that much plus the slack (the part already written is
  // kept, the reserved tail past the old end becomes sentinels) and only the
  // flagged tiles are swept again, appending. Their pairs written before the
  // overflow are kept too: duplicates vanish in the dedupe.
  const int sweep_warps = sweep_warps_per_block(d.tw, d.th);
  const int sweep_blocks =
      (int)std::max<int64_t>(std::min<int64_t>((ntiles + sweep_warps - 1) / sweep_warps, (int64_t)g_dev.num_sms * 8), 1);
  const unsigned long long W = (unsigned long long)sweep_blocks * (unsigned long long)sweep_warps;
  const unsigned long long guess = M > 0 ? std::max<unsigned long long>(2ull * M, 1ull << 16) : 0ull;
  uint32_t chunk = 32;
  while (chunk < 512 && 2ull * chunk * W <= guess) chunk <<= 1;
  unsigned long long cap = (unsigned long long)Pe + (M > 0 ? guess + W * chunk : 0ull);
  CKR(g->pairs.reserve((size_t)std::max<unsigned long long>(cap, 1) * 8, s));
  if (Pe > 0)
    launch_explicit_pairs(g->pred_off.as<int32_t>(), g->pred.as<int32_t>(), n, B, g->pairs.as<uint64_t>(), s);
  int64_t Ptot = Pe;
  // CSR by buckets: counts [n+1], offsets [n+1], distinct counts [n+1], long
  // rows [n+1], the longest row and the long-row count
  CKR(g->bucket.reserve(((size_t)4 * (n + 1) + 64) * 4, s));
  uint32_t* bcnt = g->bucket.as<uint32_t>();
  uint32_t* boff = bcnt + (n + 1);
  uint32_t* bucnt = boff + (n + 1);
  uint32_t* bbig = bucnt + (n + 1);
  uint32_t* bmax = bbig + (n + 1);
  uint32_t* bnbig = bmax + 16;
  const bool counted = M > 0;  // the sweep's pairs are counted per source before its sync
  h64[6] = 0;
  if (M > 0) {
    unsigned long long* rerun = reinterpret_cast<unsigned long long*>(g->misc.as<char>() + 128);
    CKR(g->tflags.reserve((size_t)ntiles * 2, s));
    uint8_t* flags1 = g->tflags.as<uint8_t>();
    uint8_t* flags2 = flags1 + ntiles;
    CK(cudaMemsetAsync(flags1, 0, (size_t)ntiles * 2, s));
    h64[2] = (uint64_t)Pe;
    CK(cudaMemcpyAsync(cursor, (const void*)&h64[2], 8, cudaMemcpyHostToDevice, s));
    CK(cudaMemsetAsync(tile_counter, 0, 4, s));
    CK(cudaMemsetAsync(rerun, 0, 8, s));
    // dense inputs (16 or more binned entries per task): the first sweep passes
    // its pair keys through a direct-mapped filter of about one slot per entry
    // (2^16 .. 2^26 slots), so that a pair found again in other tiles is not
    // written again; skipped when it would pass the graph's memory cap
    int fbits = 0;
    if (M >= (int64_t)16 * n) {
      fbits = 16;
      while (fbits < 26 && (1ll << fbits) < M) ++fbits;
      const size_t fbytes = (size_t)8 << fbits;
      if (fbytes > g->pfilt.cap && t_capped && over_cap(fbytes - g->pfilt.cap)) {
        fbits = 0;
      } else {
        CKR(g->pfilt.reserve(fbytes, s));
        CK(cudaMemsetAsync(g->pfilt.p, 0xFF, fbytes, s));
      }
    }
    g->pair_filter_bits = fbits;
    SweepOut o{g->pairs.as<uint64_t>(), cap, cursor, tile_counter, B, chunk, nullptr, flags1, rerun,
               fbits ? g->pfilt.as<unsigned long long>() : nullptr, fbits};
    if (prof) CK(cudaEventRecord(g->ev[EV_SW0], s));
    launch_sweep(spay, g->seg_b.as<uint32_t>(), g->seg_e.as<uint32_t>(), d, o, sweep_blocks, s);
    if (prof) CK(cudaEventRecord(g->ev[EV_SW1], s));
    CK(cudaGetLastError());
    trace("analyze: sweep enqueued");
    // the pairs per source and the longest row, before the sync the sweep
    // needs anyway: they decide between the bucket CSR and the pair sort
    CK(cudaMemsetAsync(bcnt, 0, (size_t)(n + 1) * 4, s));
    CK(cudaMemsetAsync(bmax, 0, 4, s));
    launch_bucket_count(g->pairs.as<uint64_t>(), cursor, cap, B, bcnt, n, bmax, s);
    CK(cudaMemcpyAsync((void*)&h64[6], bmax, 4, cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync((void*)&h64[3], cursor, 8, cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync((void*)&h64[5], rerun, 8, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    trace("analyze: sweep synced");
    Ptot = (int64_t)h64[3];
    if ((unsigned long long)Ptot > cap) {
      const unsigned long long old_cap = cap;
      cap = (unsigned long long)Ptot + (unsigned long long)h64[5] + W * chunk;
      CKR(g->pairs.reserve((size_t)cap * 8, s, (size_t)old_cap * 8));
      CK(cudaMemsetAsync(g->pairs.as<uint64_t>() + old_cap, 0xFF, (size_t)(Ptot - old_cap) * 8, s));
      CK(cudaMemsetAsync(tile_counter, 0, 4, s));
      // the rerun writes every pair its tiles find: no filter (a pair whose
      // first write fell past the buffer's end may already sit in it)
      SweepOut o2{g->pairs.as<uint64_t>(), cap, cursor, tile_counter, B, chunk, flags1, flags2, rerun, nullptr, 0};
      launch_sweep(spay, g->seg_b.as<uint32_t>(), g->seg_e.as<uint32_t>(), d, o2, sweep_blocks, s);
      if (prof) CK(cudaEventRecord(g->ev[EV_SW1], s));
      CK(cudaGetLastError());
      // the rerun appended pairs: count again
      CK(cudaMemsetAsync(bcnt, 0, (size_t)(n + 1) * 4, s));
      CK(cudaMemsetAsync(bmax, 0, 4, s));
      launch_bucket_count(g->pairs.as<uint64_t>(), cursor, cap, B, bcnt, n, bmax, s);
      CK(cudaMemcpyAsync((void*)&h64[6], bmax, 4, cudaMemcpyDeviceToHost, s));
      CK(cudaMemcpyAsync((void*)&h64[3], cursor, 8, cudaMemcpyDeviceToHost, s));
      CK(cudaStreamSynchronize(s));
      Ptot = (int64_t)h64[3];
      if ((unsigned long long)Ptot > cap) return fail(RT_ERR_OOM, "pair buffer overflowed in the rerun");
    }
  }
  CKR(g->pairs_alt.reserve((size_t)std::max<int64_t>(Ptot, 1) * 8, s));
  if (Ptot >= (1ll << 31) - 1) return fail(RT_ERR_OOM, "%lld candidate pairs (limit 2^31)", (long long)Ptot);
  if (prof) CK(cudaEventRecord(g->ev[EV_SWEEP], s));
  g->n_pairs = Ptot;

  // ---- 5: dedupe + CSR -----------------------------------------------------
  CKR(g->flags.reserve((size_t)(Ptot + 1) * 4, s));
  CKR(g->upos.reserve((size_t)(Ptot + 1) * 4, s));
  CKR(g->col.reserve((size_t)std::max<int64_t>(Ptot, 1) * 4, s));
  CKR(g->row_ptr.reserve((size_t)(n + 1) * 4, s));
  CKR(g->indeg.reserve((size_t)n * 4, s));
  CKR(g->count.reserve((size_t)n * 4, s));
  CKR(g->rootpos.reserve((size_t)(n + 1) * 4, s));
  CKR(g->root_items.reserve((size_t)n * 8, s));
  CKR(reserve_ws(g, std::max(radix_ws_bytes(Ptot),
                             scan_ws_elems<uint32_t>(std::max<int64_t>(Ptot, n) + 1) * 4)));
  // rows of at most kBucketMaxRow pairs: buckets per source, each sorted and
  // deduplicated in place; longer rows: an LSD radix sort of all the pairs
  const bool by_buckets = counted && (uint32_t)(h64[6] & 0xffffffffull) <= (uint32_t)kBucketMaxRow;
  const uint32_t* n_edges_at;
  if (by_buckets) {
    launch_bucket_build(g->pairs.as<uint64_t>(), Ptot, B, n, bcnt, boff, bucnt, bbig, bnbig, g->flags.as<uint32_t>(),
                        g->row_ptr.as<uint32_t>(), g->ws.as<uint32_t>(), g->col.as<int32_t>(), g->indeg.as<int32_t>(),
                        s);
    if (prof) CK(cudaEventRecord(g->ev[EV_SORTP], s));
    n_edges_at = g->row_ptr.as<uint32_t>() + n;
  } else {
    const int flip = radix_sort<uint64_t>(g->pairs.as<uint64_t>(), g->pairs_alt.as<uint64_t>(), nullptr,
                                          nullptr, Ptot, 2 * B, g->ws.p, s);
    const uint64_t* sp = flip ? g->pairs_alt.as<uint64_t>() : g->pairs.as<uint64_t>();
    if (prof) CK(cudaEventRecord(g->ev[EV_SORTP], s));
    launch_unique_flags(sp, Ptot, g->flags.as<uint32_t>(), s);
    scan_exclusive<uint32_t>(g->flags.as<uint32_t>(), g->upos.as<uint32_t>(), Ptot, g->ws.as<uint32_t>(), s);
    CK(cudaMemsetAsync(g->row_ptr.p, 0, (size_t)(n + 1) * 4, s));
    CK(cudaMemsetAsync(g->indeg.p, 0, (size_t)n * 4, s));
    launch_emit_csr(sp, g->flags.as<uint32_t>(), g->upos.as<uint32_t>(), Ptot, B, g->col.as<int32_t>(),
                    g->row_ptr.as<int32_t>(), g->indeg.as<int32_t>(), s);
    scan_exclusive<uint32_t>(g->row_ptr.as<uint32_t>(), g->row_ptr.as<uint32_t>(), n, g->ws.as<uint32_t>(), s);
    n_edges_at = g->upos.as<uint32_t>() + Ptot;
  }
  g->csr_by_buckets = by_buckets;
  launch_roots(g->indeg.as<int32_t>(), n, g->rootpos.as<uint32_t>(), s);
  scan_exclusive<uint32_t>(g->rootpos.as<uint32_t>(), g->rootpos.as<uint32_t>(), n, g->ws.as<uint32_t>(), s);
  launch_roots_emit(g->indeg.as<int32_t>(), g->rootpos.as<uint32_t>(), n, 0, 0, g->root_items.as<uint64_t>(),
                    g->count.as<int32_t>(), s);
  CKR(g->adj.reserve((size_t)n * 32, s));
  uint32_t* maxdeg = reinterpret_cast<uint32_t*>(g->misc.as<char>() + 192);
  CK(cudaMemsetAsync(maxdeg, 0, 4, s));
  launch_pack_adj(g->row_ptr.as<int32_t>(), g->col.as<int32_t>(), g->indeg.as<int32_t>(), n, g->adj.as<int4>(),
                  maxdeg, s);
  g->adjx_ok = false;
  if (prof) CK(cudaEventRecord(g->ev[EV_CSR], s));
  CK(cudaMemcpyAsync(g->hpin + 8, n_edges_at, 4, cudaMemcpyDeviceToHost, s));
  CK(cudaMemcpyAsync(g->hpin + 9, g->rootpos.as<uint32_t>() + n, 4, cudaMemcpyDeviceToHost, s));
  CK(cudaMemcpyAsync(g->hpin + 10, maxdeg, 4, cudaMemcpyDeviceToHost, s));
  trace("analyze: csr enqueued");
  CK(cudaStreamSynchronize(s));
  trace("analyze: csr synced");
  CK(cudaGetLastError());
  g->n_edges = g->hpin[8];
  g->n_roots = g->hpin[9];
  g->max_outdeg = (int32_t)g->hpin[10];
  g->analyze_timed = prof;
  return RT_OK;
}

}  // namespace

extern "C" rt_status rt_analyze(rt_graph_t g) {
  if (!g) return fail(RT_ERR_INVALID, "graph is NULL");
  if (g->analyzed) return RT_OK;
  CapScope cap_scope(g);
  const int body = g->desc.body;
  if ((body == RT_BODY_SPIN || body == RT_BODY_FMA || body == RT_BODY_CHECK) && (!g->desc.out || g->desc.out_elems < g->n))
    return fail(RT_ERR_INVALID, "SPIN/FMA/CHECK bodies need `out` with one int32 per task (%d)", g->n);
  if (g->n > 0 && body == RT_BODY_COUNTER && !g->has_body_arg) return fail(RT_ERR_INVALID, "COUNTER needs body_arg");
  CKR(ensure_device());
  CKR(ensure_pinned(g));
  drop_replay_graph(g);
  g->ev_preds = false;
  g->kh_valid = false;
  drop_kernel_graph(g);
  if (g->n > 0) CKR(run_analysis(g));
  else g->n_edges = g->n_roots = g->n_entries = g->n_pairs = 0;
  g->analyzed = true;
  g->dirty = false;
  return RT_OK;
}

extern "C" rt_status rt_get_csr(rt_graph_t g, const int32_t** row_ptr, const int32_t** col,
                                const int32_t** indeg, int64_t* n_tasks, int64_t* n_edges) {
  if (!g) return fail(RT_ERR_INVALID, "graph is NULL");
  if (!g->analyzed) return fail(RT_ERR_STATE, "graph not analyzed");
  if (g->n > 0) CK(cudaStreamSynchronize(g->s));
  if (row_ptr) *row_ptr = g->row_ptr.as<int32_t>();
  if (col) *col = g->col.as<int32_t>();
  if (indeg) *indeg = g->indeg.as<int32_t>();
  if (n_tasks) *n_tasks = g->n;
  if (n_edges) *n_edges = g->n_edges;
  return RT_OK;
}

// ---------------------------------------------------------------------------
// execution
// ---------------------------------------------------------------------------
namespace {

constexpr int kStatusWord = 40;
constexpr int32_t kMaxKernelTasks = 1 << 17;  // rt_execute_kernels: one event per task
constexpr int kKernelStreams = 16;     // hpin word receiving the executor status
constexpr int kCountersByte = 512;  // hpin byte offset of the executor's diagnostic counters

rt_status prepare_run(rt_graph* g, int32_t replays, ExecParams* out, int64_t* ring_clear) {
  cudaStream_t s = g->s;
  const bool owned = g->cfg_policy == RT_EXEC_OWNED;  // no ring: every warp polls the countdowns it owns
  const uint64_t cap = (uint64_t)g->n * (uint64_t)replays + 64;
  if (cap >= 0xFFFFFFF0ull) return fail(RT_ERR_INVALID, "tasks x replays must stay below 2^32 per launch");
  const bool grow = !owned && (cap * 8 > g->ring.cap || !g->ring.p);
  if (grow) {
    drop_replay_graph(g);
    CKR(g->ring.reserve((size_t)cap * 8, s));
  }
  *ring_clear = owned ? 0 : ((grow || g->dirty) ? (int64_t)(g->ring.cap / 8) : 0);
  CKR(g->ctrl.reserve(sizeof(ExecCtrl), s));
  CKR(g->done_g.reserve(64, s));
  const bool wide = owned && g->max_outdeg > kAdjInline;  // some task has successors past its record
  if (wide && !g->adjx_ok) {
    CKR(g->adjx.reserve((size_t)g->n * 32, s));
    launch_pack_adjx(g->row_ptr.as<int32_t>(), g->col.as<int32_t>(), g->n, g->adjx.as<int4>(), s);
    g->adjx_ok = true;
  }
  if (!g->gtable.p) {
    CKR(g->gtable.reserve(sizeof(ExecGraph), s));
  }
  ExecGraph G{};
  G.task_base = 0;
  G.n_tasks = g->n;
  G.root_base = 0;
  G.n_roots = (int32_t)g->n_roots;
  G.body = g->desc.body;
  G.spin_iters = g->desc.spin_iters;
  G.ndim = g->dims.ndim;
  G.state = (int32_t*)g->desc.state;
  G.out = (int32_t*)g->desc.out;
  G.body_arg = g->body_arg.as<int32_t>();
  G.req_off = g->req_off.as<int32_t>();
  G.lo = g->lo.as<int64_t>();
  G.hi = g->hi.as<int64_t>();
  G.priv = g->priv.as<uint8_t>();
  G.dom_lo[0] = g->dims.dom_lo[0];
  G.dom_lo[1] = g->dims.dom_lo[1];
  G.ext[0] = g->dims.ext[0];
  G.ext[1] = g->dims.ext[1];
  // the table lives in device memory; rewritten (synchronously) only when it changes
  if (!g->gt_valid || memcmp(&G, &g->gt_host, sizeof G) != 0) {
    CK(cudaStreamSynchronize(s));
    CK(cudaMemcpy(g->gtable.p, &G, sizeof G, cudaMemcpyHostToDevice));
    g->gt_host = G;
    g->gt_valid = true;
  }
  if (g->desc.flags & RT_GRAPH_TICKETS) CKR(g->tickets.reserve((size_t)g->n * 8, s));
  ExecParams p{};
  p.adj = g->adj.as<int4>();
  p.adjx = wide ? g->adjx.as<int4>() : nullptr;
  p.row_ptr = g->row_ptr.as<int32_t>();
  p.col = g->col.as<int32_t>();
  p.indeg = g->indeg.as<int32_t>();
  p.count = g->count.as<int32_t>();
  p.ring = g->ring.as<uint64_t>();
  p.ring_cap = (uint32_t)std::min<uint64_t>(g->ring.cap / 8, 0xFFFFFFF0ull);
  p.n_graphs = 1;
  p.root_items = g->root_items.as<uint64_t>();
  p.graphs = g->gtable.as<ExecGraph>();
  p.done_g = g->done_g.as<uint32_t>();
  p.ctrl = g->ctrl.as<ExecCtrl>();
  p.replays = replays;
  p.graphs_target = 1;
  p.timeout_ns = g->desc.timeout_ns;
  p.claim = g->cfg_claim > 0 ? g->cfg_claim : (owned ? 1 : 8);  // owned: chunks a warp holds at once
  p.keep = g->cfg_keep > 0 ? g->cfg_keep : 16;
  p.tickets = (g->desc.flags & RT_GRAPH_TICKETS) ? g->tickets.as<int32_t>() : nullptr;
  p.total_roots = owned ? 0 : (int32_t)g->n_roots;
  p.need_fence = g->desc.body == RT_BODY_COUNTER || g->desc.body == RT_BODY_CHECK;
  p.policy = g->cfg_policy;
  *out = p;
  return RT_OK;
}

rt_status enqueue_run(rt_graph* g, const ExecParams& p, int64_t ring_clear, cudaStream_t s, bool timed) {
  if (g->dirty || g->hold_task >= 0)
    launch_reset_counts(g->count.as<int32_t>(), g->indeg.as<int32_t>(), g->n, g->hold_task, g->hold_extra, s);
  if (timed) CK(cudaEventRecord(g->ev[EV_X0], s));
  launch_seed(p, ring_clear, s);
  const int warps = g->cfg_warps > 0 ? g->cfg_warps : 2;
  const int blocks = g->cfg_blocks > 0 ? g->cfg_blocks : g_dev.num_sms;
  if (timed) CK(cudaEventRecord(g->ev[EV_XK0], s));
  launch_exec(p, blocks, warps, s);
  if (timed) CK(cudaEventRecord(g->ev[EV_XK1], s));
  CK(cudaMemcpyAsync(g->hpin + kStatusWord, &p.ctrl->status, 4, cudaMemcpyDeviceToHost, s));
  CK(cudaMemcpyAsync(reinterpret_cast<char*>(g->hpin) + kCountersByte, p.ctrl->counters,
                     kCntCount * sizeof(unsigned long long), cudaMemcpyDeviceToHost, s));
  g->exec_blocks = blocks;
  g->exec_warps = warps;
  return RT_OK;
}

rt_status start_run(rt_graph* g, int32_t replays) {
  if (!g) return fail(RT_ERR_INVALID, "graph is NULL");
  if (!g->analyzed) return fail(RT_ERR_STATE, "execute before analyze");
  if (replays <= 0) return fail(RT_ERR_INVALID, "replays must be positive");
  if (g->n == 0) {
    g->hpin[kStatusWord] = 0;
    g->status_pending = false;
    return RT_OK;
  }
  if (g->hold_task >= g->n) return fail(RT_ERR_INVALID, "held task out of range");
  CKR(ensure_device());
  const bool timed = (g->desc.flags & RT_GRAPH_PROFILE) != 0;
  if (timed) CKR(graph_events(g));
  ExecParams p;
  int64_t ring_clear = 0;
  CKR(prepare_run(g, replays, &p, &ring_clear));
  cudaStream_t s = g->s;
  const bool special = g->dirty || g->hold_task >= 0 || ring_clear > 0 || timed ||
                       (g->desc.flags & RT_GRAPH_TICKETS);
  if (special || replays == 1) {
    CKR(enqueue_run(g, p, ring_clear, s, timed));
  } else {
    // replay: a cached CUDA graph of {seed, executor, status read-back}
    if (!g->replay_exec || g->replay_times != replays) {
      drop_replay_graph(g);
      if (!g->cap_stream) CK(cudaStreamCreateWithFlags(&g->cap_stream, cudaStreamNonBlocking));
      CK(cudaStreamBeginCapture(g->cap_stream, cudaStreamCaptureModeThreadLocal));
      rt_status st = enqueue_run(g, p, 0, g->cap_stream, false);
      cudaGraph_t graph = nullptr;
      cudaError_t e = cudaStreamEndCapture(g->cap_stream, &graph);
      if (st != RT_OK) {
        if (graph) cudaGraphDestroy(graph);
        return st;
      }
      if (e != cudaSuccess) return fail(RT_ERR_CUDA, "capture: %s", cudaGetErrorString(e));
      e = cudaGraphInstantiate(&g->replay_exec, graph, 0);
      cudaGraphDestroy(graph);
      if (e != cudaSuccess) return fail(RT_ERR_CUDA, "instantiate: %s", cudaGetErrorString(e));
      g->replay_times = replays;
    }
    CK(cudaGraphLaunch(g->replay_exec, s));
  }
  CK(cudaGetLastError());
  g->exec_timed = timed;
  g->status_pending = true;
  if (g->hold_task >= 0) {
    g->hold_task = -1;
    g->dirty = true;  // the held run cannot finish: re-arm every counter next time
  } else {
    g->dirty = false;
  }
  return RT_OK;
}

}  // namespace

extern "C" {

rt_status rt_execute(rt_graph_t g) { return start_run(g, 1); }

rt_status rt_replay(rt_graph_t g, int32_t times) { return start_run(g, times); }

}  // extern "C"

namespace grt {
// The analysed graph's in-edges (each task's preconditions, as the application
// would state them at launch): pred[pred_off[v] .. pred_off[v+1]), built once
// per analysis on the device.
rt_status ensure_in_edges(rt_graph* g) {
  if (g->ev_preds) return RT_OK;
  cudaStream_t s = g->s;
  const int32_t n = g->n;
  const int64_t E = g->n_edges;
  CKR(g->ev_pred_off.reserve((size_t)(n + 1) * 4, s));
  CKR(g->ev_pred.reserve((size_t)std::max<int64_t>(E, 1) * 4, s));
  CKR(g->ev_pending.reserve((size_t)std::max<int32_t>(n, 1) * 4, s));
  CKR(reserve_ws(g, scan_ws_elems<uint32_t>(n + 1) * 4));
  CK(cudaMemcpyAsync(g->ev_pred_off.p, g->indeg.p, (size_t)n * 4, cudaMemcpyDeviceToDevice, s));
  scan_exclusive<uint32_t>(g->ev_pred_off.as<uint32_t>(), g->ev_pred_off.as<uint32_t>(), n, g->ws.as<uint32_t>(), s);
  CK(cudaMemsetAsync(g->ev_pending.p, 0, (size_t)n * 4, s));  // cursors for the transpose
  launch_ev_transpose(g->row_ptr.as<int32_t>(), g->col.as<int32_t>(), n, g->ev_pred_off.as<int32_t>(),
                      g->ev_pending.as<int32_t>(), g->ev_pred.as<int32_t>(), s);
  g->ev_preds = true;
  return RT_OK;
}
}  // namespace grt

extern "C" {

rt_status rt_execute_kernels(rt_graph_t g, int32_t mode, int32_t iters, int32_t threads, float* ms) {
  if (!g) return fail(RT_ERR_INVALID, "graph is NULL");
  if (!g->analyzed) return fail(RT_ERR_STATE, "graph not analyzed");
  if (mode < 0 || mode > 2) return fail(RT_ERR_INVALID, "mode must be 0 (lifted), 1 (async edges) or 2 (CUDA graph)");
  if (iters < 0 || threads < 32 || threads > 1024) return fail(RT_ERR_INVALID, "iters >= 0, threads in 32..1024");
  if (g->n > kMaxKernelTasks) return fail(RT_ERR_INVALID, "at most %d tasks run as kernels", kMaxKernelTasks);
  if (!g->desc.out || g->desc.out_elems < g->n) return fail(RT_ERR_INVALID, "needs `out` with one int32 per task");
  if (ms) *ms = 0.f;
  const int32_t n = g->n;
  if (n == 0) return RT_OK;
  CKR(ensure_device());
  cudaStream_t s = g->s;
  CKR(ensure_in_edges(g));
  if (!g->kh_valid) {
    g->kh_rp.resize((size_t)n + 1);
    g->kh_col.resize((size_t)std::max<int64_t>(g->n_edges, 1));
    g->kh_poff.resize((size_t)n + 1);
    g->kh_pred.resize((size_t)std::max<int64_t>(g->n_edges, 1));
    CK(cudaMemcpyAsync(g->kh_rp.data(), g->row_ptr.p, ((size_t)n + 1) * 4, cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(g->kh_col.data(), g->col.p, (size_t)g->n_edges * 4, cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(g->kh_poff.data(), g->ev_pred_off.p, ((size_t)n + 1) * 4, cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(g->kh_pred.data(), g->ev_pred.p, (size_t)g->n_edges * 4, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    g->kh_valid = true;
  }
  while ((int32_t)g->kevents.size() < n) {
    cudaEvent_t e;
    CK(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    g->kevents.push_back(e);
  }
  while (g->kstreams.size() < (size_t)kKernelStreams) {
    cudaStream_t st;
    CK(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
    g->kstreams.push_back(st);
  }
  CKR(g->ksink.reserve(4096, s));
  int32_t* depth = (int32_t*)g->desc.out;
  const int32_t* poff = g->ev_pred_off.as<int32_t>();
  const int32_t* pred = g->ev_pred.as<int32_t>();
  float* sink = g->ksink.as<float>();
  if (mode == 2 && (!g->kg_exec || g->kg_iters != iters || g->kg_threads != threads)) {
    // one kernel node per task, its dependencies the nodes of its predecessors
    drop_kernel_graph(g);
    CK(cudaGraphCreate(&g->kg, 0));
    std::vector<cudaGraphNode_t> nodes((size_t)n);
    std::vector<cudaGraphNode_t> deps;
    for (int32_t v = 0; v < n; ++v) {
      deps.clear();
      for (int32_t k = g->kh_poff[(size_t)v]; k < g->kh_poff[(size_t)v + 1]; ++k)
        deps.push_back(nodes[(size_t)g->kh_pred[(size_t)k]]);
      int32_t vv = v, it = iters;
      void* args[] = {&vv, (void*)&poff, (void*)&pred, &depth, &sink, &it};
      cudaKernelNodeParams kp{};
      kp.func = task_kernel_fn();
      kp.gridDim = dim3(1);
      kp.blockDim = dim3((unsigned)threads);
      kp.kernelParams = args;
      CK(cudaGraphAddKernelNode(&nodes[(size_t)v], g->kg, deps.data(), deps.size(), &kp));
    }
    CK(cudaGraphInstantiate(&g->kg_exec, g->kg, 0));
    g->kg_iters = iters;
    g->kg_threads = threads;
  }
  // depths start at 0, so a task run before a predecessor shows
  CK(cudaMemsetAsync(depth, 0, (size_t)n * 4, s));
  CK(cudaStreamSynchronize(s));
  const auto t0 = std::chrono::steady_clock::now();
  if (mode == 2) {
    count_launch(n);
    CK(cudaGraphLaunch(g->kg_exec, s));
    CK(cudaStreamSynchronize(s));
  } else if (mode == 1) {
    // async edges: every launch enqueued now, each predicated on its
    // predecessors' events (program order is a topological order)
    for (int32_t v = 0; v < n; ++v) {
      cudaStream_t st = g->kstreams[(size_t)v % kKernelStreams];
      for (int32_t k = g->kh_poff[(size_t)v]; k < g->kh_poff[(size_t)v + 1]; ++k)
        CK(cudaStreamWaitEvent(st, g->kevents[(size_t)g->kh_pred[(size_t)k]], 0));
      launch_task_kernel(v, poff, pred, depth, sink, iters, threads, st);
      CK(cudaEventRecord(g->kevents[(size_t)v], st));
    }
    for (cudaStream_t st : g->kstreams) CK(cudaStreamSynchronize(st));
  } else {
    // lifted: the host launches a task once it has seen, by polling, that the
    // events of all its predecessors have completed
    std::vector<int32_t> pending((size_t)n);
    std::vector<int32_t> ready, flight;
    for (int32_t v = 0; v < n; ++v) {
      pending[(size_t)v] = g->kh_poff[(size_t)v + 1] - g->kh_poff[(size_t)v];
      if (pending[(size_t)v] == 0) ready.push_back(v);
    }
    const int64_t limit = g->desc.timeout_ns > 0 ? g->desc.timeout_ns : 10000000000ll;
    int32_t done = 0;
    auto last = std::chrono::steady_clock::now();
    while (done < n) {
      for (int32_t v : ready) {
        cudaStream_t st = g->kstreams[(size_t)v % kKernelStreams];
        launch_task_kernel(v, poff, pred, depth, sink, iters, threads, st);
        CK(cudaEventRecord(g->kevents[(size_t)v], st));
        flight.push_back(v);
      }
      ready.clear();
      for (size_t i = 0; i < flight.size();) {
        const int32_t v = flight[i];
        const cudaError_t q = cudaEventQuery(g->kevents[(size_t)v]);
        if (q == cudaErrorNotReady) {
          ++i;
          continue;
        }
        if (q != cudaSuccess) return fail(RT_ERR_CUDA, "task kernel: %s", cudaGetErrorString(q));
        flight[i] = flight.back();
        flight.pop_back();
        ++done;
        last = std::chrono::steady_clock::now();
        for (int32_t e = g->kh_rp[(size_t)v]; e < g->kh_rp[(size_t)v + 1]; ++e)
          if (--pending[(size_t)g->kh_col[(size_t)e]] == 0) ready.push_back(g->kh_col[(size_t)e]);
      }
      if (std::chrono::duration_cast<std::chrono::nanoseconds>(std::chrono::steady_clock::now() - last).count() >
          limit)
        return fail(RT_ERR_TIMEOUT, "task kernels made no progress");
    }
  }
  CK(cudaGetLastError());
  if (ms) *ms = (float)std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  return RT_OK;
}

rt_status rt_execute_events(rt_graph_t g, float* ms_kernel) {
  if (!g) return fail(RT_ERR_INVALID, "graph is NULL");
  if (!g->analyzed) return fail(RT_ERR_STATE, "graph not analyzed");
  if (ms_kernel) *ms_kernel = 0.f;
  if (g->n == 0) return RT_OK;
  const int body = g->desc.body;
  if ((body == RT_BODY_SPIN || body == RT_BODY_FMA || body == RT_BODY_CHECK) && (!g->desc.out || g->desc.out_elems < g->n))
    return fail(RT_ERR_INVALID, "SPIN/CHECK bodies need `out` with one int32 per task");
  CKR(ensure_device());
  CKR(ensure_pinned(g));
  cudaStream_t s = g->s;
  const int32_t n = g->n;
  const int64_t E = g->n_edges;
  CKR(ensure_in_edges(g));
  const uint32_t ring_cap = (uint32_t)n + 64u;
  CKR(g->ev_head.reserve((size_t)n * 4, s));
  CKR(g->ev_pending.reserve((size_t)n * 4, s));
  CKR(g->ev_nodes.reserve((size_t)(E + 1) * 8, s));
  CKR(g->ev_ring.reserve((size_t)ring_cap * 4, s));
  CKR(g->ev_ctrl.reserve(sizeof(EvCtrl), s));
  CK(cudaMemsetAsync(g->ev_ctrl.p, 0, sizeof(EvCtrl), s));
  EvParams p{};
  p.claim = std::min(std::max(g->cfg_claim > 0 ? g->cfg_claim : 8, 1), 32);  // as the compiled executor's
  p.pred_off = g->ev_pred_off.as<int32_t>();
  p.pred = g->ev_pred.as<int32_t>();
  p.n = n;
  p.ring_cap = ring_cap;
  p.head = g->ev_head.as<uint32_t>();
  p.pending = g->ev_pending.as<int32_t>();
  p.node_task = g->ev_nodes.as<uint32_t>();
  p.node_next = g->ev_nodes.as<uint32_t>() + (E + 1);
  p.ring = g->ev_ring.as<uint32_t>();
  p.ctrl = g->ev_ctrl.as<EvCtrl>();
  ExecGraph& G = p.G;
  G.n_tasks = n;
  G.body = body;
  G.spin_iters = g->desc.spin_iters;
  G.ndim = g->dims.ndim;
  G.state = (int32_t*)g->desc.state;
  G.out = (int32_t*)g->desc.out;
  G.body_arg = g->body_arg.as<int32_t>();
  G.req_off = g->req_off.as<int32_t>();
  G.lo = g->lo.as<int64_t>();
  G.hi = g->hi.as<int64_t>();
  G.priv = g->priv.as<uint8_t>();
  G.dom_lo[0] = g->dims.dom_lo[0];
  G.dom_lo[1] = g->dims.dom_lo[1];
  G.ext[0] = g->dims.ext[0];
  G.ext[1] = g->dims.ext[1];
  p.timeout_ns = g->desc.timeout_ns > 0 ? g->desc.timeout_ns : 2000000000ll;
  CKR(graph_events(g));
  CK(cudaEventRecord(g->ev[EV_E0], s));
  launch_events(p, g_dev.num_sms * 2, s);
  CK(cudaEventRecord(g->ev[EV_E1], s));
  CK(cudaMemcpyAsync(g->hpin + kStatusWord, &p.ctrl->status, 4, cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  CK(cudaGetLastError());
  if (ms_kernel) cudaEventElapsedTime(ms_kernel, g->ev[EV_E0], g->ev[EV_E1]);
  const uint32_t st = g->hpin[kStatusWord];
  if (st == (uint32_t)RT_ERR_TIMEOUT) return fail(RT_ERR_TIMEOUT, "event executor made no progress");
  if (st == (uint32_t)RT_ERR_OOM) return fail(RT_ERR_OOM, "event executor ring overflow");
  return RT_OK;
}

rt_status rt_execute_stitched(rt_graph_t g, int32_t replays, float* ms_kernel) {
  if (!g) return fail(RT_ERR_INVALID, "graph is NULL");
  if (!g->analyzed) return fail(RT_ERR_STATE, "graph not analyzed");
  if (ms_kernel) *ms_kernel = 0.f;
  if (replays < 1) return fail(RT_ERR_INVALID, "replays must be positive (got %d)", replays);
  if (g->n % 2 != 0)
    return fail(RT_ERR_INVALID, "a stitched graph holds two copies of one trace (got %d tasks)", g->n);
  const int32_t n = g->n / 2;
  if (n == 0) return RT_OK;
  const int64_t total = (int64_t)replays * n;
  if (total > 0x7FFFFFF0ll) return fail(RT_ERR_INVALID, "replays x tasks = %lld (limit 2^31 - 16)", (long long)total);
  const int body = g->desc.body;
  if ((body == RT_BODY_SPIN || body == RT_BODY_FMA || body == RT_BODY_CHECK) && (!g->desc.out || g->desc.out_elems < total))
    return fail(RT_ERR_INVALID, "SPIN/CHECK bodies need `out` with one int32 per task and replay (%lld)",
                (long long)total);
  CKR(ensure_device());
  CKR(ensure_pinned(g));
  cudaStream_t s = g->s;
  // the second copy must repeat the first
  CKR(g->st_err.reserve(4, s));
  CK(cudaMemsetAsync(g->st_err.p, 0, 4, s));
  launch_stitch_check(g->req_off.as<int32_t>(), g->lo.as<int64_t>(), g->hi.as<int64_t>(), g->priv.as<uint8_t>(),
                      g->dims.ndim, g->row_ptr.as<int32_t>(), g->col.as<int32_t>(), n, g->st_err.as<uint32_t>(), s);
  CK(cudaMemcpyAsync(g->hpin + kStatusWord, g->st_err.p, 4, cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  CK(cudaGetLastError());
  if (g->hpin[kStatusWord] & 1u)
    return fail(RT_ERR_INVALID, "the graph's second half does not repeat the first one's rectangles");
  if (g->hpin[kStatusWord] & 2u)
    return fail(RT_ERR_INVALID, "the graph's two halves have different internal edges");
  const bool tickets = (g->desc.flags & RT_GRAPH_TICKETS) != 0;
  CKR(g->st_count.reserve((size_t)total * 4, s));
  CKR(g->st_ring.reserve((size_t)total * 8, s));
  CKR(g->st_ctrl.reserve(sizeof(ExecCtrl), s));
  if (tickets) CKR(g->st_tickets.reserve((size_t)total * 8, s));
  StitchParams p{};
  p.adj = g->adj.as<int4>();
  p.col = g->col.as<int32_t>();
  p.count = g->st_count.as<int32_t>();
  p.ring = g->st_ring.as<uint64_t>();
  p.ring_cap = (uint32_t)total;
  p.n = n;
  p.R = replays;
  p.claim = std::min(g->cfg_claim > 0 ? g->cfg_claim : 8, 32);
  p.keep = std::min(g->cfg_keep > 0 ? g->cfg_keep : 16, 64);  // the kernel keeps at most 64 per warp
  p.total = total;
  p.ctrl = g->st_ctrl.as<ExecCtrl>();
  p.tickets = tickets ? g->st_tickets.as<int32_t>() : nullptr;
  ExecGraph& G = p.G;
  G.n_tasks = n;
  G.body = body;
  G.spin_iters = g->desc.spin_iters;
  G.ndim = g->dims.ndim;
  G.state = (int32_t*)g->desc.state;
  G.out = (int32_t*)g->desc.out;
  G.body_arg = g->body_arg.as<int32_t>();
  G.req_off = g->req_off.as<int32_t>();
  G.lo = g->lo.as<int64_t>();
  G.hi = g->hi.as<int64_t>();
  G.priv = g->priv.as<uint8_t>();
  G.dom_lo[0] = g->dims.dom_lo[0];
  G.dom_lo[1] = g->dims.dom_lo[1];
  G.ext[0] = g->dims.ext[0];
  G.ext[1] = g->dims.ext[1];
  p.timeout_ns = g->desc.timeout_ns > 0 ? g->desc.timeout_ns : 2000000000ll;
  const int warps = std::min(g->cfg_warps > 0 ? g->cfg_warps : 2, 8);
  const int blocks = g->cfg_blocks > 0 ? g->cfg_blocks : g_dev.num_sms;
  CK(cudaMemsetAsync(p.ring, 0xFF, (size_t)total * 8, s));
  CK(cudaMemsetAsync(p.ctrl, 0, sizeof(ExecCtrl), s));
  CKR(graph_events(g));
  CK(cudaEventRecord(g->ev[EV_E0], s));
  launch_stitch(p, g->indeg.as<int32_t>(), g->root_items.as<uint64_t>(), g->rootpos.as<uint32_t>(), blocks, warps,
                tickets, body == RT_BODY_CHECK || body == RT_BODY_COUNTER, s);
  CK(cudaEventRecord(g->ev[EV_E1], s));
  CK(cudaMemcpyAsync(g->hpin + kStatusWord, &p.ctrl->status, 4, cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  CK(cudaGetLastError());
  if (ms_kernel) cudaEventElapsedTime(ms_kernel, g->ev[EV_E0], g->ev[EV_E1]);
  g->st_R = tickets ? replays : 0;
  const uint32_t st = g->hpin[kStatusWord];
  if (st == (uint32_t)RT_ERR_TIMEOUT) return fail(RT_ERR_TIMEOUT, "stitched replay made no progress");
  if (st == (uint32_t)RT_ERR_OOM) return fail(RT_ERR_OOM, "stitched replay ring overflow");
  return RT_OK;
}

rt_status rt_copy_stitched_tickets(rt_graph_t g, int32_t* out) {
  if (!g) return fail(RT_ERR_INVALID, "graph is NULL");
  if (!out) return fail(RT_ERR_INVALID, "out is NULL");
  if (g->st_R == 0) return fail(RT_ERR_STATE, "no stitched run with RT_GRAPH_TICKETS yet");
  CK(cudaMemcpy(out, g->st_tickets.p, (size_t)g->st_R * (g->n / 2) * 8, cudaMemcpyDefault));
  return RT_OK;
}

rt_status rt_sync(rt_graph_t g) {
  if (!g) return fail(RT_ERR_INVALID, "graph is NULL");
  if (!g->hpin && !g->status_pending) return RT_OK;
  CK(cudaStreamSynchronize(g->s));
  CK(cudaGetLastError());
  if (g->status_pending) {
    g->status_pending = false;
    const uint32_t st = g->hpin[kStatusWord];
    if (st == (uint32_t)RT_ERR_TIMEOUT) {
      g->dirty = true;
      return fail(RT_ERR_TIMEOUT, "executor made no progress for %lld ns", (long long)g->desc.timeout_ns);
    }
    if (st != 0u) {
      g->dirty = true;
      return fail(RT_ERR_OOM, "executor ring overflow (status %u)", st);
    }
  }
  return RT_OK;
}

rt_status rt_graph_stats(rt_graph_t g, rt_graph_stats_t* out) {
  if (!g || !out) return fail(RT_ERR_INVALID, "NULL argument");
  memset(out, 0, sizeof *out);
  if (g->ev_ok || g->hpin) CK(cudaStreamSynchronize(g->s));
  out->n_tasks = g->n;
  out->n_rects = g->R;
  out->n_preds = g->P;
  out->n_entries = g->n_entries;
  out->n_pairs = g->n_pairs;
  out->csr_by_buckets = g->csr_by_buckets ? 1 : 0;
  out->pair_filter_bits = g->pair_filter_bits;
  out->n_edges = g->n_edges;
  out->n_roots = g->n_roots;
  out->tile_w = g->dims.tw;
  out->tile_h = g->dims.th;
  out->exec_blocks = g->exec_blocks;
  out->exec_threads = g->exec_warps * 32;
  if (g->ev_ok && g->analyze_timed) {
    cudaEventElapsedTime(&out->ms_analyze, g->ev[EV_A0], g->ev[EV_CSR]);
    cudaEventElapsedTime(&out->ms_bin, g->ev[EV_A0], g->ev[EV_BIN]);
    cudaEventElapsedTime(&out->ms_sort_entries, g->ev[EV_BIN], g->ev[EV_SORTE]);
    cudaEventElapsedTime(&out->ms_sweep, g->ev[EV_SORTE], g->ev[EV_SWEEP]);
    cudaEventElapsedTime(&out->ms_sort_pairs, g->ev[EV_SWEEP], g->ev[EV_SORTP]);
    cudaEventElapsedTime(&out->ms_csr, g->ev[EV_SORTP], g->ev[EV_CSR]);
    if (g->n_entries > 0) cudaEventElapsedTime(&out->ms_sweep_kernel, g->ev[EV_SW0], g->ev[EV_SW1]);
  }
  if (g->hpin) {
    const unsigned long long* c = reinterpret_cast<const unsigned long long*>(reinterpret_cast<char*>(g->hpin) + 512);
    for (int k = 0; k < kCntCount && k < 9; ++k) out->exec_counters[k] = (int64_t)c[k];
  }
  if (g->ev_ok && g->exec_timed) {
    cudaEventElapsedTime(&out->ms_execute, g->ev[EV_X0], g->ev[EV_XK1]);
    cudaEventElapsedTime(&out->ms_exec_kernel, g->ev[EV_XK0], g->ev[EV_XK1]);
  }
  cudaGetLastError();
  return RT_OK;
}

rt_status rt_get_tickets(rt_graph_t g, const int32_t** tickets) {
  if (!g || !tickets) return fail(RT_ERR_INVALID, "NULL argument");
  if (!(g->desc.flags & RT_GRAPH_TICKETS) || !g->tickets.p) return fail(RT_ERR_STATE, "no tickets recorded");
  CK(cudaStreamSynchronize(g->s));
  *tickets = g->tickets.as<int32_t>();
  return RT_OK;
}

rt_status rt_graph_exec_config(rt_graph_t g, int32_t blocks, int32_t warps, int32_t claim, int32_t keep) {
  if (!g) return fail(RT_ERR_INVALID, "graph is NULL");
  if (blocks < 0 || warps < 0 || warps > 8 || claim < 0 || claim > 32 || keep < 0 || keep > 64)
    return fail(RT_ERR_INVALID, "exec config out of range (warps 0..8, claim 0..32, keep 0..64)");
  if (blocks > 0) {
    CKR(ensure_device());
    const int w = warps > 0 ? warps : 8;
    if (blocks > g_dev.num_sms * std::max(exec_max_blocks_per_sm(w), 1))
      return fail(RT_ERR_INVALID, "more persistent blocks than can be resident");
  }
  g->cfg_blocks = blocks;
  g->cfg_warps = warps;
  g->cfg_claim = claim;
  g->cfg_keep = keep;
  drop_replay_graph(g);
  return RT_OK;
}

rt_status rt_graph_exec_policy(rt_graph_t g, int32_t policy) {
  if (!g) return fail(RT_ERR_INVALID, "graph is NULL");
  if (policy != RT_EXEC_RING && policy != RT_EXEC_OWNED) return fail(RT_ERR_INVALID, "unknown policy %d", policy);
  if (policy != g->cfg_policy) drop_replay_graph(g);
  g->cfg_policy = policy;
  return RT_OK;
}

rt_status rt_debug_hold_task(rt_graph_t g, int32_t task, int32_t extra) {
  if (!g) return fail(RT_ERR_INVALID, "graph is NULL");
  if (task < 0 || extra <= 0) return fail(RT_ERR_INVALID, "task must be >= 0 and extra > 0");
  g->hold_task = task;
  g->hold_extra = extra;
  return RT_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// batches: many captured graphs, one persistent launch
// ---------------------------------------------------------------------------
namespace {
int exec_bps_for(int warps) {
  static int cache[9] = {0};
  if (warps < 1 || warps > 8) return 1;
  if (!cache[warps]) cache[warps] = std::max(exec_max_blocks_per_sm(warps), 1);
  return cache[warps];
}
}  // namespace

extern "C" {

rt_status rt_batch_create(const rt_graph_t* graphs, int32_t n_graphs, void* stream, rt_batch_t* out) {
  if (!out) return fail(RT_ERR_INVALID, "out is NULL");
  *out = nullptr;
  if (!graphs || n_graphs <= 0) return fail(RT_ERR_INVALID, "no graphs");
  if (n_graphs >= (1 << 20)) return fail(RT_ERR_INVALID, "a batch holds fewer than 2^20 graphs (got %d)", n_graphs);
  int64_t T = 0, E = 0, Rt = 0;
  int32_t nonempty = 0;
  for (int32_t i = 0; i < n_graphs; ++i) {
    if (!graphs[i]) return fail(RT_ERR_INVALID, "graph %d is NULL", i);
    if (!graphs[i]->analyzed) return fail(RT_ERR_STATE, "graph %d is not analyzed", i);
    T += graphs[i]->n;
    E += graphs[i]->n_edges;
    Rt += graphs[i]->n_roots;
    nonempty += graphs[i]->n > 0;
  }
  if (T >= (1ll << 31) - 1 || E >= (1ll << 31) - 1) return fail(RT_ERR_INVALID, "batch exceeds 2^31 tasks or edges");
  CKR(ensure_device());
  rt_batch* b = new (std::nothrow) rt_batch();
  if (!b) return fail(RT_ERR_OOM, "host allocation failed");
  b->s = (cudaStream_t)stream;
  b->G = n_graphs;
  b->G_nonempty = nonempty;
  b->T = T;
  b->E = E;
  b->Rtot = Rt;
  cudaStream_t s = b->s;
  auto bail = [&](rt_status st) {
    rt_batch_destroy(b);
    return st;
  };
  rt_status st;
  if ((st = b->row_ptr.reserve((size_t)(T + 1) * 4, s)) || (st = b->col.reserve((size_t)std::max<int64_t>(E, 1) * 4, s)) ||
      (st = b->indeg.reserve((size_t)std::max<int64_t>(T, 1) * 4, s)) ||
      (st = b->count.reserve((size_t)std::max<int64_t>(T, 1) * 4, s)) ||
      (st = b->root_items.reserve((size_t)std::max<int64_t>(Rt, 1) * 8, s)) ||
      (st = b->gtable.reserve((size_t)n_graphs * sizeof(ExecGraph), s)) ||
      (st = b->done_g.reserve((size_t)n_graphs * 4, s)) || (st = b->ctrl.reserve(sizeof(ExecCtrl), s)))
    return bail(st);
  if (cudaMallocHost(&b->hpin, 1024) != cudaSuccess || cudaEventCreate(&b->e0) != cudaSuccess ||
      cudaEventCreate(&b->e1) != cudaSuccess)
    return bail(fail(RT_ERR_CUDA, "batch host/event allocation failed"));
  std::vector<ExecGraph> table((size_t)n_graphs);
  int64_t tb = 0, eb = 0, rb = 0;
  cudaMemsetAsync(b->row_ptr.p, 0, 4, s);
  for (int32_t i = 0; i < n_graphs; ++i) {
    rt_graph* g = graphs[i];
    cudaStreamSynchronize(g->s);  // its analysis is complete
    ExecGraph& G = table[(size_t)i];
    G.task_base = (int32_t)tb;
    G.n_tasks = g->n;
    G.root_base = (int32_t)rb;
    G.n_roots = (int32_t)g->n_roots;
    G.body = g->desc.body;
    G.spin_iters = g->desc.spin_iters;
    G.ndim = g->dims.ndim;
    G.state = (int32_t*)g->desc.state;
    G.out = (int32_t*)g->desc.out;
    G.body_arg = g->body_arg.as<int32_t>();
    G.req_off = g->req_off.as<int32_t>();
    G.lo = g->lo.as<int64_t>();
    G.hi = g->hi.as<int64_t>();
    G.priv = g->priv.as<uint8_t>();
    G.dom_lo[0] = g->dims.dom_lo[0];
    G.dom_lo[1] = g->dims.dom_lo[1];
    G.ext[0] = g->dims.ext[0];
    G.ext[1] = g->dims.ext[1];
    if (G.body == RT_BODY_COUNTER || G.body == RT_BODY_CHECK) b->need_fence = 1;
    if (g->n > 0) {
      int32_t* rp = b->row_ptr.as<int32_t>() + tb;
      cudaMemcpyAsync(rp, g->row_ptr.p, (size_t)(g->n + 1) * 4, cudaMemcpyDeviceToDevice, s);
      launch_add_offset(rp, g->n + 1, (int32_t)eb, s);
      if (g->n_edges > 0) {
        int32_t* cl = b->col.as<int32_t>() + eb;
        cudaMemcpyAsync(cl, g->col.p, (size_t)g->n_edges * 4, cudaMemcpyDeviceToDevice, s);
        launch_add_offset(cl, g->n_edges, (int32_t)tb, s);
      }
      cudaMemcpyAsync(b->indeg.as<int32_t>() + tb, g->indeg.p, (size_t)g->n * 4, cudaMemcpyDeviceToDevice, s);
      cudaMemcpyAsync(b->count.as<int32_t>() + tb, g->indeg.p, (size_t)g->n * 4, cudaMemcpyDeviceToDevice, s);
      launch_rebase_roots(g->root_items.as<uint64_t>(), b->root_items.as<uint64_t>() + rb, (int32_t)g->n_roots, i,
                          (int32_t)tb, s);
    }
    tb += g->n;
    eb += g->n_edges;
    rb += g->n_roots;
  }
  if ((st = b->adj.reserve((size_t)std::max<int64_t>(T, 1) * 32, s))) return bail(st);
  launch_pack_adj(b->row_ptr.as<int32_t>(), b->col.as<int32_t>(), b->indeg.as<int32_t>(), T, b->adj.as<int4>(),
                  nullptr, s);
  if (cudaMemcpyAsync(b->gtable.p, table.data(), table.size() * sizeof(ExecGraph), cudaMemcpyHostToDevice, s) !=
          cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess || cudaGetLastError() != cudaSuccess)
    return bail(fail(RT_ERR_CUDA, "batch assembly failed"));
  b->dirty = true;  // ring not yet initialised
  *out = b;
  return RT_OK;
}

rt_status rt_batch_create_stacked(rt_graph_t g, const int32_t* task_off, int32_t n_graphs, void* stream,
                                  rt_batch_t* out) {
  if (!out) return fail(RT_ERR_INVALID, "out is NULL");
  *out = nullptr;
  if (!g || !task_off || n_graphs <= 0) return fail(RT_ERR_INVALID, "NULL graph, offsets or no graphs");
  if (n_graphs >= (1 << 20)) return fail(RT_ERR_INVALID, "a batch holds fewer than 2^20 graphs (got %d)", n_graphs);
  if (!g->analyzed) return fail(RT_ERR_STATE, "graph is not analyzed");
  if (task_off[0] != 0 || task_off[n_graphs] != g->n)
    return fail(RT_ERR_INVALID, "task_off must run from 0 to the graph's %d tasks", g->n);
  int32_t nonempty = 0;
  for (int32_t k = 0; k < n_graphs; ++k) {
    if (task_off[k + 1] < task_off[k]) return fail(RT_ERR_INVALID, "task_off decreases at graph %d", k);
    nonempty += task_off[k + 1] > task_off[k];
  }
  CKR(ensure_device());
  rt_batch* b = new (std::nothrow) rt_batch();
  if (!b) return fail(RT_ERR_OOM, "host allocation failed");
  const int64_t T = g->n, E = g->n_edges, Rt = g->n_roots;
  b->s = (cudaStream_t)stream;
  b->G = n_graphs;
  b->G_nonempty = nonempty;
  b->T = T;
  b->E = E;
  b->Rtot = Rt;
  cudaStream_t s = b->s;
  auto bail = [&](rt_status st) {
    rt_batch_destroy(b);
    return st;
  };
  rt_status st;
  DevBuf tmp;  // task and root starts of the graphs, the check flag
  if ((st = b->row_ptr.reserve((size_t)(T + 1) * 4, s)) || (st = b->col.reserve((size_t)std::max<int64_t>(E, 1) * 4, s)) ||
      (st = b->indeg.reserve((size_t)std::max<int64_t>(T, 1) * 4, s)) ||
      (st = b->count.reserve((size_t)std::max<int64_t>(T, 1) * 4, s)) ||
      (st = b->root_items.reserve((size_t)std::max<int64_t>(Rt, 1) * 8, s)) ||
      (st = b->gtable.reserve((size_t)n_graphs * sizeof(ExecGraph), s)) ||
      (st = b->done_g.reserve((size_t)n_graphs * 4, s)) || (st = b->ctrl.reserve(sizeof(ExecCtrl), s)) ||
      (st = tmp.reserve((size_t)(n_graphs + 1) * 16 + 64, s)))
    return bail(st);
  if (cudaMallocHost(&b->hpin, 1024) != cudaSuccess || cudaEventCreate(&b->e0) != cudaSuccess ||
      cudaEventCreate(&b->e1) != cudaSuccess) {
    tmp.release(s);
    return bail(fail(RT_ERR_CUDA, "batch host/event allocation failed"));
  }
  cudaStreamSynchronize(g->s);  // its analysis is complete
  uint32_t* task_first = tmp.as<uint32_t>();
  uint32_t* gathered = task_first + (n_graphs + 1);          // 2 words per graph start
  uint32_t* root_first = gathered + 2 * (n_graphs + 1);
  uint32_t* bad = root_first + (n_graphs + 1);
  std::vector<uint32_t> h_first((size_t)n_graphs + 1), h_gath(2 * ((size_t)n_graphs + 1)), h_root((size_t)n_graphs + 1);
  for (int32_t k = 0; k <= n_graphs; ++k) h_first[(size_t)k] = (uint32_t)task_off[k];
  cudaError_t e = cudaMemcpyAsync(task_first, h_first.data(), h_first.size() * 4, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(bad, 0, 4, s);
  launch_check_stacked(g->row_ptr.as<int32_t>(), g->col.as<int32_t>(), T, task_first, n_graphs, bad, s);
  launch_serve_gather(g->rootpos.as<uint32_t>(), g->row_ptr.as<int32_t>(), reinterpret_cast<const int32_t*>(task_first),
                      n_graphs + 1, gathered, s);
  uint32_t h_bad = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(h_gath.data(), gathered, h_gath.size() * 4, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&h_bad, bad, 4, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) {
    tmp.release(s);
    return bail(fail(RT_ERR_CUDA, "stacked batch: %s", cudaGetErrorString(e)));
  }
  if (h_bad) {
    tmp.release(s);
    return bail(fail(RT_ERR_INVALID, "an edge joins two graphs of the stacked batch"));
  }
  for (int32_t k = 0; k <= n_graphs; ++k) h_root[(size_t)k] = h_gath[2 * (size_t)k];
  std::vector<ExecGraph> table((size_t)n_graphs);
  for (int32_t k = 0; k < n_graphs; ++k) {
    ExecGraph& G = table[(size_t)k];
    const int32_t tb = task_off[k];
    G.task_base = tb;
    G.n_tasks = task_off[k + 1] - tb;
    G.root_base = (int32_t)h_root[(size_t)k];
    G.n_roots = (int32_t)(h_root[(size_t)k + 1] - h_root[(size_t)k]);
    G.body = g->desc.body;
    G.spin_iters = g->desc.spin_iters;
    G.ndim = g->dims.ndim;
    // a body sees the graph's own tasks: its launch arrays start at its first task
    G.state = (int32_t*)g->desc.state;
    G.out = g->desc.out ? (int32_t*)g->desc.out + tb : nullptr;
    G.body_arg = g->has_body_arg ? g->body_arg.as<int32_t>() + tb : nullptr;
    G.req_off = g->req_off.as<int32_t>() + tb;
    G.lo = g->lo.as<int64_t>();
    G.hi = g->hi.as<int64_t>();
    G.priv = g->priv.as<uint8_t>();
    G.dom_lo[0] = g->dims.dom_lo[0];
    G.dom_lo[1] = g->dims.dom_lo[1];
    G.ext[0] = g->dims.ext[0];
    G.ext[1] = g->dims.ext[1];
  }
  if (g->desc.body == RT_BODY_COUNTER || g->desc.body == RT_BODY_CHECK) b->need_fence = 1;
  if (T > 0) {
    cudaMemcpyAsync(b->row_ptr.p, g->row_ptr.p, (size_t)(T + 1) * 4, cudaMemcpyDeviceToDevice, s);
    if (E > 0) cudaMemcpyAsync(b->col.p, g->col.p, (size_t)E * 4, cudaMemcpyDeviceToDevice, s);
    cudaMemcpyAsync(b->indeg.p, g->indeg.p, (size_t)T * 4, cudaMemcpyDeviceToDevice, s);
    cudaMemcpyAsync(b->count.p, g->indeg.p, (size_t)T * 4, cudaMemcpyDeviceToDevice, s);
    cudaMemcpyAsync(root_first, h_root.data(), h_root.size() * 4, cudaMemcpyHostToDevice, s);
    launch_tag_roots(g->root_items.as<uint64_t>(), b->root_items.as<uint64_t>(), Rt, root_first, n_graphs, s);
  } else {
    cudaMemsetAsync(b->row_ptr.p, 0, 4, s);
  }
  if ((st = b->adj.reserve((size_t)std::max<int64_t>(T, 1) * 32, s))) {
    tmp.release(s);
    return bail(st);
  }
  launch_pack_adj(b->row_ptr.as<int32_t>(), b->col.as<int32_t>(), b->indeg.as<int32_t>(), T, b->adj.as<int4>(),
                  nullptr, s);
  e = cudaMemcpyAsync(b->gtable.p, table.data(), table.size() * sizeof(ExecGraph), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  tmp.release(s);
  if (e != cudaSuccess || cudaGetLastError() != cudaSuccess) return bail(fail(RT_ERR_CUDA, "batch assembly failed"));
  b->dirty = true;  // ring not yet initialised
  *out = b;
  return RT_OK;
}

}  // extern "C"

namespace {
// One batch launch on stream s: the launch's INIT (a batch's counters count up
// from 0 across its replays; the ring is cleared only when it is new or dirty),
// the persistent executor and the status read-back.
rt_status enqueue_batch(rt_batch* b, const ExecParams& p, int64_t ring_clear, int blocks, int warps,
                        cudaStream_t s) {
  CK(cudaMemsetAsync(b->count.p, 0, (size_t)b->T * 4, s));
  launch_seed(p, ring_clear, s);
  launch_exec(p, blocks, warps, s);
  CK(cudaMemcpyAsync(b->hpin, &p.ctrl->status, 4, cudaMemcpyDeviceToHost, s));
  CK(cudaMemcpyAsync(reinterpret_cast<char*>(b->hpin) + 512, p.ctrl->counters, kCntCount * sizeof(unsigned long long),
                     cudaMemcpyDeviceToHost, s));
  return RT_OK;
}

void drop_batch_graph(rt_batch* b) {
  if (b->gexec) cudaGraphExecDestroy(b->gexec);
  b->gexec = nullptr;
}

// The owned-chunk policy's launch: the batch's graphs as one DAG (every edge
// still points to a later task), count-down counters reset to the in-degrees,
// a run barrier between replays; bodies run with their own graph's entry.
rt_status enqueue_batch_owned(rt_batch* b, const ExecParams& p, int blocks, int warps, cudaStream_t s) {
  launch_reset_counts(b->count.as<int32_t>(), b->indeg.as<int32_t>(), b->T, -1, 0, s);
  launch_seed(p, 0, s);  // clears the control block and the completion counters
  launch_exec(p, blocks, warps, s);
  CK(cudaMemcpyAsync(b->hpin, &p.ctrl->status, 4, cudaMemcpyDeviceToHost, s));
  CK(cudaMemcpyAsync(reinterpret_cast<char*>(b->hpin) + 512, p.ctrl->counters, kCntCount * sizeof(unsigned long long),
                     cudaMemcpyDeviceToHost, s));
  return RT_OK;
}

rt_status prepare_batch_owned(rt_batch* b) {
  if (b->owned_ready) return RT_OK;
  cudaStream_t s = b->s;
  CKR(b->task_graph.reserve((size_t)std::max<int64_t>(b->T, 1) * 4, s));
  launch_fill_task_graph(b->gtable.as<ExecGraph>(), b->G, b->task_graph.as<int32_t>(), s);
  CKR(b->scratch.reserve(64, s));
  CK(cudaMemsetAsync(b->scratch.p, 0, 4, s));
  launch_max_outdeg(b->row_ptr.as<int32_t>(), b->T, b->scratch.as<uint32_t>(), s);
  CK(cudaMemcpyAsync(b->hpin + 4, b->scratch.p, 4, cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  b->max_outdeg = (int32_t)b->hpin[4];
  if (b->max_outdeg > kAdjInline) {
    CKR(b->adjx.reserve((size_t)b->T * 32, s));
    launch_pack_adjx(b->row_ptr.as<int32_t>(), b->col.as<int32_t>(), b->T, b->adjx.as<int4>(), s);
  }
  CK(cudaGetLastError());
  b->owned_ready = true;
  return RT_OK;
}
}  // namespace

extern "C" {

rt_status rt_batch_capture(const rt_graph_desc* desc, int32_t n_graphs, const int32_t* task_off,
                           const int64_t* graph_lo, const int64_t* graph_hi, const int32_t* req_off, const int64_t* lo,
                           const int64_t* hi, const uint8_t* priv, int32_t flags, rt_batch_t* out,
                           rt_graph_t* graph_out) {
  if (!out) return fail(RT_ERR_INVALID, "out is NULL");
  *out = nullptr;
  if (graph_out) *graph_out = nullptr;
  if (!desc || !task_off || !graph_lo || !graph_hi || !req_off)
    return fail(RT_ERR_INVALID, "NULL descriptor, offsets, domains or req_off");
  if (n_graphs <= 0 || n_graphs >= (1 << 20))
    return fail(RT_ERR_INVALID, "a batch holds 1 to 2^20 - 1 graphs (got %d)", n_graphs);
  if (desc->ndim != 1 && desc->ndim != 2) return fail(RT_ERR_INVALID, "ndim must be 1 or 2");
  if (flags & ~(RT_LAUNCH_DEVICE | RT_LAUNCH_DEFER_CHECK)) return fail(RT_ERR_INVALID, "unknown flags");
  const int D = desc->ndim, sd = D - 1;  // graphs are stacked along the last dimension
  if (task_off[0] != 0) return fail(RT_ERR_INVALID, "task_off[0] must be 0");
  // the bands: graph k's domain moves to origin 0 across the other dimension
  // and to the sum of the earlier graphs' extents along the stacking one
  std::vector<int64_t> box((size_t)n_graphs * 3 * D);
  int64_t along = 0, across = 1;
  for (int32_t k = 0; k < n_graphs; ++k) {
    if (task_off[k + 1] < task_off[k]) return fail(RT_ERR_INVALID, "task_off decreases at graph %d", k);
    int64_t* b = &box[(size_t)k * 3 * D];
    for (int d = 0; d < D; ++d) {
      const int64_t l = graph_lo[(size_t)k * D + d], h = graph_hi[(size_t)k * D + d];
      if (l > h || h - l >= (1ll << 40)) return fail(RT_ERR_INVALID, "graph %d has an empty or huge domain", k);
      b[d] = l;
      b[D + d] = h;
      b[2 * D + d] = (d == sd ? along : 0) - l;
      if (d != sd) across = std::max<int64_t>(across, h - l + 1);
    }
    along += graph_hi[(size_t)k * D + sd] - graph_lo[(size_t)k * D + sd] + 1;
    if (along >= (1ll << 40)) return fail(RT_ERR_INVALID, "the stacked domain is too long");
  }
  const int32_t n = task_off[n_graphs];
  rt_graph_desc sdesc = *desc;
  sdesc.dom_lo[0] = sdesc.dom_lo[1] = 0;
  sdesc.dom_hi[0] = D == 2 ? across - 1 : along - 1;
  sdesc.dom_hi[1] = D == 2 ? along - 1 : 0;
  rt_graph_t g = nullptr;
  CKR(rt_graph_create(&sdesc, &g));
  auto bail = [&](rt_status st) {
    const std::string msg = g_err;
    rt_graph_destroy(g);
    g_err = msg;
    return st;
  };
  rt_status st = ensure_device();
  if (st != RT_OK) return bail(st);
  // the offsets and bands on the device, for the placement kernel
  DevBuf place;
  const size_t off_bytes = ((size_t)n_graphs + 1) * 4, box_off = (off_bytes + 15) / 16 * 16;
  if ((st = place.reserve(box_off + box.size() * 8, g->s)) != RT_OK) return bail(st);
  if (cudaMemcpyAsync(place.p, task_off, off_bytes, cudaMemcpyHostToDevice, g->s) != cudaSuccess ||
      cudaMemcpyAsync(static_cast<char*>(place.p) + box_off, box.data(), box.size() * 8, cudaMemcpyHostToDevice,
                      g->s) != cudaSuccess) {
    place.release(g->s);
    return bail(fail(RT_ERR_CUDA, "band table copy failed"));
  }
  BandPlace bp{place.as<int32_t>(), n_graphs,
               reinterpret_cast<const int64_t*>(static_cast<char*>(place.p) + box_off)};
  // host arrays are validated on the device too: their coordinates are each
  // graph's own until the placement moves them
  const int32_t fl = (flags & RT_LAUNCH_DEVICE) ? RT_LAUNCH_DEVICE : RT_LAUNCH_DEFER_CHECK;
  st = append_launches(g, n, req_off, lo, hi, priv, nullptr, nullptr, nullptr, fl, &bp);
  if (st == RT_OK) st = rt_analyze(g);
  place.release(g->s);
  if (st != RT_OK) return bail(st);
  std::vector<int32_t> toff(task_off, task_off + n_graphs + 1);
  st = rt_batch_create_stacked(g, toff.data(), n_graphs, desc->stream, out);
  if (st != RT_OK) return bail(st);
  (*out)->owned = g;
  if (graph_out) *graph_out = g;
  return RT_OK;
}

rt_status rt_batch_execute(rt_batch_t b, int32_t replays, int32_t exec_blocks, int32_t exec_warps, int32_t claim,
                           int32_t keep) {
  if (!b) return fail(RT_ERR_INVALID, "batch is NULL");
  if (replays <= 0 || replays > 4096) return fail(RT_ERR_INVALID, "a batch runs 1 to 4096 replays (got %d)", replays);
  const int warps = exec_warps > 0 ? std::min(exec_warps, 8) : 4;
  const uint64_t cap = (uint64_t)b->T * (uint64_t)replays + 64;
  if (cap >= 0xFFFFFFF0ull) return fail(RT_ERR_INVALID, "tasks x replays must stay below 2^32 per launch");
  const int max_blocks = g_dev.num_sms * exec_bps_for(warps);
  if (exec_blocks > max_blocks) return fail(RT_ERR_INVALID, "more persistent blocks than can be resident");
  const int blocks = exec_blocks > 0 ? exec_blocks : g_dev.num_sms * std::min(exec_bps_for(warps), 3);
  cudaStream_t s = b->s;
  if (b->policy == RT_EXEC_OWNED) {
    CKR(prepare_batch_owned(b));
    ExecParams p{};
    p.adj = b->adj.as<int4>();
    p.adjx = b->max_outdeg > kAdjInline ? b->adjx.as<int4>() : nullptr;
    p.row_ptr = b->row_ptr.as<int32_t>();
    p.col = b->col.as<int32_t>();
    p.indeg = b->indeg.as<int32_t>();
    p.count = b->count.as<int32_t>();
    p.n_graphs = b->G;
    p.graphs = b->gtable.as<ExecGraph>();
    p.done_g = b->done_g.as<uint32_t>();
    p.ctrl = b->ctrl.as<ExecCtrl>();
    p.replays = replays;
    p.graphs_target = b->G_nonempty;
    p.timeout_ns = 2000000000ll;
    p.claim = claim > 0 ? claim : 1;  // lanes per task
    p.keep = keep > 0 ? keep : 16;
    p.need_fence = b->need_fence;
    p.policy = RT_EXEC_OWNED;
    p.owned_n = (int32_t)b->T;
    p.task_graph = b->task_graph.as<int32_t>();
    CK(cudaEventRecord(b->e0, s));
    const int64_t key[7] = {replays, blocks, warps, p.claim, p.keep, -1 - (int64_t)RT_EXEC_OWNED, b->T};
    if (!b->gexec || memcmp(key, b->gkey, sizeof key) != 0) {
      drop_batch_graph(b);
      if (!b->cap_stream) CK(cudaStreamCreateWithFlags(&b->cap_stream, cudaStreamNonBlocking));
      CK(cudaStreamBeginCapture(b->cap_stream, cudaStreamCaptureModeThreadLocal));
      rt_status st = enqueue_batch_owned(b, p, blocks, warps, b->cap_stream);
      cudaGraph_t graph = nullptr;
      cudaError_t e = cudaStreamEndCapture(b->cap_stream, &graph);
      if (st != RT_OK) {
        if (graph) cudaGraphDestroy(graph);
        return st;
      }
      if (e != cudaSuccess) return fail(RT_ERR_CUDA, "batch capture: %s", cudaGetErrorString(e));
      e = cudaGraphInstantiate(&b->gexec, graph, 0);
      cudaGraphDestroy(graph);
      if (e != cudaSuccess) return fail(RT_ERR_CUDA, "batch instantiate: %s", cudaGetErrorString(e));
      memcpy(b->gkey, key, sizeof key);
    }
    CK(cudaGraphLaunch(b->gexec, s));
    ++b->graph_launches;
    CK(cudaEventRecord(b->e1, s));
    CK(cudaGetLastError());
    return RT_OK;  // the ring was not touched: it stays as clean as the last ring launch left it
  }
  bool clear = b->dirty;
  if (cap * 8 > b->ring.cap) {
    drop_batch_graph(b);
    CKR(b->ring.reserve((size_t)cap * 8, s));
    clear = true;
  }
  ExecParams p{};
  p.adj = b->adj.as<int4>();
  p.row_ptr = b->row_ptr.as<int32_t>();
  p.col = b->col.as<int32_t>();
  p.indeg = b->indeg.as<int32_t>();
  p.count = b->count.as<int32_t>();
  p.ring = b->ring.as<uint64_t>();
  p.ring_cap = (uint32_t)std::min<uint64_t>(b->ring.cap / 8, 0xFFFFFFF0ull);
  p.n_graphs = b->G;
  p.root_items = b->root_items.as<uint64_t>();
  p.graphs = b->gtable.as<ExecGraph>();
  p.done_g = b->done_g.as<uint32_t>();
  p.ctrl = b->ctrl.as<ExecCtrl>();
  p.replays = replays;
  p.graphs_target = b->G_nonempty;
  p.timeout_ns = 2000000000ll;
  p.claim = claim > 0 ? claim : 32;
  p.keep = keep > 0 ? keep : 32;
  p.tickets = nullptr;
  p.total_roots = (int32_t)b->Rtot;
  p.need_fence = b->need_fence;
  CK(cudaEventRecord(b->e0, s));
  if (clear) {
    // a new or dirty ring is cleared whole: a direct launch
    CKR(enqueue_batch(b, p, (int64_t)(b->ring.cap / 8), blocks, warps, s));
  } else {
    // the launch from a cached CUDA graph, captured once per launch shape
    const int64_t key[7] = {replays, blocks, warps, p.claim, p.keep, (int64_t)(uintptr_t)p.ring, (int64_t)p.ring_cap};
    if (!b->gexec || memcmp(key, b->gkey, sizeof key) != 0) {
      drop_batch_graph(b);
      if (!b->cap_stream) CK(cudaStreamCreateWithFlags(&b->cap_stream, cudaStreamNonBlocking));
      CK(cudaStreamBeginCapture(b->cap_stream, cudaStreamCaptureModeThreadLocal));
      rt_status st = enqueue_batch(b, p, 0, blocks, warps, b->cap_stream);
      cudaGraph_t graph = nullptr;
      cudaError_t e = cudaStreamEndCapture(b->cap_stream, &graph);
      if (st != RT_OK) {
        if (graph) cudaGraphDestroy(graph);
        return st;
      }
      if (e != cudaSuccess) return fail(RT_ERR_CUDA, "batch capture: %s", cudaGetErrorString(e));
      e = cudaGraphInstantiate(&b->gexec, graph, 0);
      cudaGraphDestroy(graph);
      if (e != cudaSuccess) return fail(RT_ERR_CUDA, "batch instantiate: %s", cudaGetErrorString(e));
      memcpy(b->gkey, key, sizeof key);
    }
    CK(cudaGraphLaunch(b->gexec, s));
    ++b->graph_launches;
  }
  CK(cudaEventRecord(b->e1, s));
  CK(cudaGetLastError());
  b->dirty = false;
  return RT_OK;
}

rt_status rt_batch_exec_policy(rt_batch_t b, int32_t policy) {
  if (!b) return fail(RT_ERR_INVALID, "batch is NULL");
  if (policy != RT_EXEC_RING && policy != RT_EXEC_OWNED) return fail(RT_ERR_INVALID, "unknown policy %d", policy);
  if (policy != b->policy) drop_batch_graph(b);
  b->policy = policy;
  return RT_OK;
}

rt_status rt_batch_info(rt_batch_t b, int64_t* out, int32_t n) {
  if (!b || !out || n < 0) return fail(RT_ERR_INVALID, "NULL argument");
  const int64_t v[4] = {b->G, b->T, b->E, b->graph_launches};
  for (int32_t k = 0; k < n; ++k) out[k] = k < 4 ? v[k] : 0;
  return RT_OK;
}

rt_status rt_batch_sync(rt_batch_t b, float* ms_kernel) {
  if (!b) return fail(RT_ERR_INVALID, "batch is NULL");
  CK(cudaStreamSynchronize(b->s));
  CK(cudaGetLastError());
  if (ms_kernel) {
    *ms_kernel = 0.f;
    cudaEventElapsedTime(ms_kernel, b->e0, b->e1);
    cudaGetLastError();
  }
  const uint32_t st = b->hpin[0];
  b->hpin[0] = 0;
  if (st == (uint32_t)RT_ERR_TIMEOUT) {
    b->dirty = true;
    return fail(RT_ERR_TIMEOUT, "batch executor made no progress");
  }
  if (st != 0u) {
    b->dirty = true;
    return fail(RT_ERR_OOM, "batch executor ring overflow");
  }
  return RT_OK;
}

rt_status rt_batch_destroy(rt_batch_t b) {
  if (!b) return RT_OK;
  cudaStreamSynchronize(b->s);
  drop_batch_graph(b);
  DevBuf* bufs[] = {&b->row_ptr, &b->col,  &b->indeg, &b->count, &b->root_items, &b->gtable,  &b->done_g,
                    &b->ring,    &b->ctrl, &b->adj,   &b->adjx,  &b->task_graph, &b->scratch};
  for (DevBuf* x : bufs) x->release(b->s);
  cudaStreamSynchronize(b->s);
  if (b->hpin) cudaFreeHost(b->hpin);
  if (b->e0) cudaEventDestroy(b->e0);
  if (b->e1) cudaEventDestroy(b->e1);
  if (b->cap_stream) cudaStreamDestroy(b->cap_stream);
  if (b->owned) rt_graph_destroy(b->owned);
  delete b;
  return RT_OK;
}

}  // extern "C"

extern "C" rt_status rt_copy_csr(rt_graph_t g, int32_t* row_ptr, int32_t* col, int32_t* indeg) {
  if (!g) return fail(RT_ERR_INVALID, "graph is NULL");
  if (!g->analyzed) return fail(RT_ERR_STATE, "graph not analyzed");
  if (g->n == 0) {
    if (row_ptr) {
      int32_t z = 0;
      CK(cudaMemcpy(row_ptr, &z, 4, cudaMemcpyDefault));
    }
    return RT_OK;
  }
  CK(cudaStreamSynchronize(g->s));
  if (row_ptr) CK(cudaMemcpy(row_ptr, g->row_ptr.p, (size_t)(g->n + 1) * 4, cudaMemcpyDefault));
  if (col && g->n_edges) CK(cudaMemcpy(col, g->col.p, (size_t)g->n_edges * 4, cudaMemcpyDefault));
  if (indeg) CK(cudaMemcpy(indeg, g->indeg.p, (size_t)g->n * 4, cudaMemcpyDefault));
  return RT_OK;
}

extern "C" rt_status rt_copy_tickets(rt_graph_t g, int32_t* out) {
  const int32_t* t = nullptr;
  CKR(rt_get_tickets(g, &t));
  if (out && g->n) CK(cudaMemcpy(out, t, (size_t)g->n * 8, cudaMemcpyDefault));
  return RT_OK;
}

extern "C" rt_status rt_kernel_launches(int64_t* count) {
  if (!count) return fail(RT_ERR_INVALID, "count is NULL");
  *count = grt::g_kernel_launches.load();
  return RT_OK;
}

extern "C" rt_status rt_execute_csr_static(const int32_t* row_ptr, const int32_t* col, const int32_t* indeg,
                                           int32_t n_tasks, int64_t n_edges, int32_t spin_iters, int32_t* out,
                                           int32_t* tickets, void* stream) {
  if (n_tasks < 0 || n_edges < 0 || spin_iters < 0) return fail(RT_ERR_INVALID, "negative size");
  if (n_tasks > grt::static_max_tasks())
    return fail(RT_ERR_INVALID, "rt_execute_csr_static handles at most %d tasks (got %d); use rt_execute",
                grt::static_max_tasks(), n_tasks);
  if (n_edges >= (1ll << 31)) return fail(RT_ERR_INVALID, "too many edges");
  if (n_tasks == 0) return RT_OK;
  if (!row_ptr || !indeg || !out || (n_edges > 0 && !col)) return fail(RT_ERR_INVALID, "NULL array");
  const char* why = "";
  rt_status st = grt::static_execute(row_ptr, col, indeg, n_tasks, n_edges, spin_iters, out, tickets,
                                     (cudaStream_t)stream, 2000000000ll, &why);
  if (st != RT_OK) return fail(st, "rt_execute_csr_static: %s", why);
  return RT_OK;
}

extern "C" rt_status rt_batch_counters(rt_batch_t b, int64_t* out, int32_t n) {
  if (!b || !out || n < 0) return fail(RT_ERR_INVALID, "NULL argument");
  CK(cudaStreamSynchronize(b->s));
  const unsigned long long* c = reinterpret_cast<const unsigned long long*>(reinterpret_cast<char*>(b->hpin) + 512);
  for (int k = 0; k < n; ++k) out[k] = k < kCntCount ? (int64_t)c[k] : 0;
  return RT_OK;
}

extern "C" rt_status rt_microbench_atomics(double* out, int32_t n, void* stream) {
  if (!out || n <= 0) return fail(RT_ERR_INVALID, "out is NULL");
  CKR(ensure_device());
  const char* why = "";
  const rt_status st = grt::microbench(out, n, (cudaStream_t)stream, &why);
  if (st != RT_OK) return fail(st, "microbenchmark: %s", why);
  return RT_OK;
}

namespace grt {
void set_last_error(const char* msg) { g_err = msg ? msg : ""; }

void trace(const char* what) {
  static const bool on = [] {
    const char* e = getenv("GRT_TRACE");
    return e && e[0] == '1';
  }();
  if (!on) return;
  timespec ts;
  clock_gettime(CLOCK_MONOTONIC, &ts);
  fprintf(stderr, "[grt %ld.%06ld] %s\n", (long)ts.tv_sec, ts.tv_nsec / 1000, what);
  fflush(stderr);
}

rt_status batch_shape(rt_batch_t b, int64_t* graphs, int64_t* tasks, int64_t* edges) {
  if (!b) return fail(RT_ERR_INVALID, "batch is NULL");
  *graphs = b->G;
  *tasks = b->T;
  *edges = b->E;
  return RT_OK;
}

rt_status graph_view(rt_graph_t g, GraphView* v) {
  if (!g || !v) return fail(RT_ERR_INVALID, "NULL argument");
  if (!g->analyzed) return fail(RT_ERR_STATE, "graph not analyzed");
  v->req_off = g->req_off.as<int32_t>();
  v->lo = g->lo.as<int64_t>();
  v->hi = g->hi.as<int64_t>();
  v->priv = g->priv.as<uint8_t>();
  v->adj = g->adj.as<int4>();
  v->col = g->col.as<int32_t>();
  v->row_ptr = g->row_ptr.as<int32_t>();
  v->rootpos = g->rootpos.as<uint32_t>();
  v->count = g->count.as<int32_t>();
  v->roots = g->root_items.as<uint64_t>();
  v->n = g->n;
  v->n_roots = (int32_t)g->n_roots;
  v->n_edges = g->n_edges;
  v->footprint = footprint_of(g);
  return RT_OK;
}

size_t graph_footprint(rt_graph_t g) { return g ? footprint_of(g) : 0; }

void graph_set_mem_cap(rt_graph_t g, size_t cap) {
  if (g) g->mem_cap = cap;
}

rt_status graph_trim(rt_graph_t g) {
  if (!g) return fail(RT_ERR_INVALID, "graph is NULL");
  rt_graph_clear(g);
  drop_kernel_graph(g);
  for_each_buf(g, [&](DevBuf& b) { b.release(g->s); });
  g->gt_valid = false;
  g->adjx_ok = false;
  return RT_OK;
}
}  // namespace grt
