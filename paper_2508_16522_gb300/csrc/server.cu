// server.cu -- host side of serving: admission, batched analysis, completion.
//
// Requests queue in arrival order. A worker thread takes every request that is
// waiting (up to max_batch, while request slots are free and their estimated
// device memory fits the budget) and analyses them TOGETHER as one graph: each
// request's rectangles are shifted into a band of their own along the last
// dimension of a stacked domain, so no rectangle of one request meets another's
// and the batch's DAG is the disjoint union of the requests' DAGs (task v of
// request j is task toff_j + v). One analysis, a few tens of kernel launches
// and three host syncs, then serves the whole batch; the per-request costs
// that remain are a table entry and a mailbox post.
//
// Every request keeps its own slot in the device table: the entry points into
// the batch's CSR, countdown counters and trigger records, and at the
// request's own roots. The serving kernel (serve.cu) carries the slot in every
// ready item, so each request completes on its own, as soon as its last task
// runs. A completion thread watches the host-mapped completion words, stamps
// the finish time, copies results back if asked, frees the slot and, when the
// batch's last request has finished, the batch graph and its budget share.
// While one batch executes, workers analyse the next ones: continuous batching.
#include <stdio.h>
#include <time.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "grt_internal.cuh"

using namespace grt;

namespace {

int64_t now_ns() {
  timespec ts;
  clock_gettime(CLOCK_MONOTONIC, &ts);
  return (int64_t)ts.tv_sec * 1000000000ll + ts.tv_nsec;
}

struct Request {
  int64_t ticket = 0;
  int32_t n = 0;
  std::vector<int32_t> req_off;
  std::vector<int64_t> lo, hi;
  std::vector<uint8_t> priv;
  int64_t arrival = 0, admit = 0, posted = 0, done = 0;
  int64_t estimate = 0, footprint = 0, n_edges = 0;
  int state = 0, status = 0, slot = -1, batch = -1;
  int32_t toff = 0;                        // first task in the batch graph
  int32_t band = 0;                        // its band (position) in the batch
  int64_t eoff = 0;                        // first edge in the batch graph's CSR
  std::vector<int32_t> row_ptr, col, out;  // results (keep_results)
  std::vector<int32_t> cells;              // CHECK: final state of its domain (keep_results)
  std::string error;                       // why it failed (state 4)
};

struct Slot {      // one request's entry of the device table
  uint32_t gen = 0;
  Request* req = nullptr;
};

// pinned host memory that only grows; replaced buffers are freed with the
// server (freeing pinned memory may synchronise the device, which the
// resident serving kernel would turn into a wait for the server's end)
struct HostBuf {
  void* p = nullptr;
  size_t cap = 0;
};

struct Batch {     // a pooled graph that analyses one batch of requests
  rt_graph_t g = nullptr;
  cudaStream_t stream = nullptr;
  int32_t* out = nullptr;    // SPIN/CHECK outputs of the whole batch (device)
  int32_t* state = nullptr;  // CHECK: one domain's state per band (device)
  int32_t* gidx = nullptr;   // task offsets of the batch's requests (device)
  uint32_t* gout = nullptr;  // gathered root and edge offsets (device)
  int32_t* hidx = nullptr;   // pinned mirrors of the two
  uint32_t* hout = nullptr;
  HostBuf req_off, lo, hi, priv;
  int live = 0;              // requests of the batch not yet finished
  int64_t footprint = 0;     // device bytes the batch graph holds
};

// error message of a failed library call, kept with the request
std::string last_err() {
  const char* e = rt_last_error();
  return e ? std::string(e) : std::string();
}

}  // namespace

struct rt_server {
  rt_server_desc desc{};
  int device = 0;
  int stack_dim = 0;               // requests are stacked along this dimension
  int64_t band = 0;                // extent of one request's domain along it
  int64_t cells = 0;               // cells of one request's domain (CHECK state)
  std::vector<Slot> slots;
  std::vector<int> free_slots;
  std::vector<Batch> batches;
  std::vector<int> free_batches;
  std::vector<HostBuf> retired;    // outgrown pinned buffers
  // device
  ServeSlot* table = nullptr;
  ServeSlot* table_h = nullptr;    // pinned staging: one entry per slot
  uint32_t* done_s = nullptr;
  ServeCtrl* ctrl = nullptr;
  uint64_t* items = nullptr;
  unsigned long long* seq = nullptr;
  unsigned long long cap = 0;
  // host-mapped
  ServeMailbox* mail = nullptr;
  ServeMailbox* mail_dev = nullptr;
  uint32_t* done_gen = nullptr;
  uint32_t* done_gen_dev = nullptr;
  cudaStream_t exec_stream = nullptr;
  cudaStream_t copy_stream = nullptr;
  // admission
  std::mutex mu;
  std::condition_variable cv;      // workers: something to admit
  std::condition_variable cv_done; // drain: a request finished
  std::deque<Request*> pending;
  std::unordered_map<int64_t, std::unique_ptr<Request>> reqs;
  int64_t next_ticket = 1;
  // Device-memory budget. Every batch graph has a ledger entry: the bytes it
  // may hold. While a batch is analysed that is its cap (the graph cannot grow
  // past it); otherwise it is what the graph holds, retained for reuse. The
  // entries always sum to at most budget_bytes, so the bytes the graphs hold
  // never exceed the budget; free batch graphs are trimmed to make room.
  std::vector<int64_t> ledger;
  int64_t ledger_sum = 0, ledger_peak = 0;
  std::vector<int64_t> held;            // per batch graph: bytes it held after its last analysis
  int64_t held_sum = 0, held_peak = 0;
  int64_t fixed_bytes = 0;              // the pool allocated at creation (not request memory)
  int64_t n_trims = 0, n_retries = 0;
  int64_t outstanding = 0;         // submitted, not yet done or failed
  int64_t n_batches = 0, n_batched = 0;
  std::mutex post_mu;              // serialises mailbox posts
  std::mutex pin_mu;               // guards `retired`
  bool stopping = false;
  std::atomic<bool> quit{false};
  std::vector<std::thread> workers;
  std::thread completer;
  std::vector<int> running;        // slots posted to the kernel (guarded by mu)
  std::string fatal;
};

namespace {

int64_t estimate_bytes(int32_t n, int64_t R) {
  // analysis buffers grow with binned entries (a few tiles per rectangle),
  // candidate pairs and the CSR; this bound is replaced by the real footprint
  // once the request has been analysed
  return (8ll << 20) + (int64_t)n * 256 + R * 2048;
}

bool grow(rt_server* s, HostBuf& b, size_t bytes) {
  if (b.cap >= bytes) return true;
  size_t c = std::max<size_t>(bytes + bytes / 2, 1 << 16);
  void* p = nullptr;
  if (cudaHostAlloc(&p, c, cudaHostAllocDefault) != cudaSuccess) return false;
  if (b.p) {
    std::lock_guard<std::mutex> lk(s->pin_mu);
    s->retired.push_back(b);
  }
  b.p = p;
  b.cap = c;
  return true;
}

void fail_request(Request* r, int status, std::string why) {
  r->error = std::move(why);
  r->state = 4;
  r->status = status;
  r->done = now_ns();
}

// Writes the batch's arrays in pinned memory: request j's launches follow
// request j-1's, and its rectangles move j bands along the stacking dimension.
rt_status build_union(rt_server* s, Batch& b, const std::vector<Request*>& rs, int32_t n_tot, int64_t R_tot) {
  const int D = s->desc.ndim, sd = s->stack_dim;
  if (R_tot > INT32_MAX) return RT_ERR_OOM;  // launch offsets are int32
  if (!grow(s, b.req_off, (size_t)(n_tot + 1) * 4) || !grow(s, b.lo, (size_t)std::max<int64_t>(R_tot, 1) * D * 8) ||
      !grow(s, b.hi, (size_t)std::max<int64_t>(R_tot, 1) * D * 8) ||
      !grow(s, b.priv, (size_t)std::max<int64_t>(R_tot, 1)))
    return RT_ERR_OOM;
  int32_t* ro = static_cast<int32_t*>(b.req_off.p);
  int64_t* lo = static_cast<int64_t*>(b.lo.p);
  int64_t* hi = static_cast<int64_t*>(b.hi.p);
  uint8_t* pv = static_cast<uint8_t*>(b.priv.p);
  int64_t roff = 0;
  for (size_t j = 0; j < rs.size(); ++j) {
    Request* r = rs[j];
    for (int32_t i = 0; i < r->n; ++i) ro[r->toff + i] = (int32_t)(roff + r->req_off[(size_t)i]);
    const int64_t R = r->req_off[(size_t)r->n];
    const int64_t shift = (int64_t)j * s->band;
    int64_t* l = lo + roff * D;
    int64_t* h = hi + roff * D;
    std::memcpy(l, r->lo.data(), (size_t)R * D * 8);
    std::memcpy(h, r->hi.data(), (size_t)R * D * 8);
    if (shift)
      for (int64_t k = 0; k < R; ++k) {
        l[k * D + sd] += shift;
        h[k * D + sd] += shift;
      }
    std::memcpy(pv + roff, r->priv.data(), (size_t)R);
    roff += R;
  }
  ro[n_tot] = (int32_t)R_tot;
  return RT_OK;
}

void set_ledger(rt_server* s, int bi, int64_t bytes) {
  s->ledger_sum += bytes - s->ledger[(size_t)bi];
  s->ledger[(size_t)bi] = bytes;
  s->ledger_peak = std::max(s->ledger_peak, s->ledger_sum);
}

// batch bi's graph now holds `bytes` (measured by the thread that owns it)
void set_held(rt_server* s, int bi, int64_t bytes) {
  s->held_sum += bytes - s->held[(size_t)bi];
  s->held[(size_t)bi] = bytes;
  s->held_peak = std::max(s->held_peak, s->held_sum);
}

// Room for batch bi to hold `need` bytes (its ledger entry included)? Trims
// the other free batch graphs' retained buffers when that makes the room.
// Called with s->mu held.
bool make_room(rt_server* s, int bi, int64_t need) {
  const int64_t others = s->ledger_sum - s->ledger[(size_t)bi];
  if (others + need <= s->desc.budget_bytes) return true;
  for (int f : s->free_batches) {
    if (f == bi || s->ledger[(size_t)f] == 0) continue;
    graph_trim(s->batches[(size_t)f].g);
    set_ledger(s, f, 0);
    set_held(s, f, 0);
    ++s->n_trims;
  }
  return s->ledger_sum - s->ledger[(size_t)bi] + need <= s->desc.budget_bytes;
}

void worker_main(rt_server* s) {
  cudaSetDevice(s->device);
  std::vector<Request*> rs;
  for (;;) {
    rs.clear();
    int bi = -1;
    int64_t est = 0;
    {
      std::unique_lock<std::mutex> lk(s->mu);
      s->cv.wait(lk, [&] {
        if (s->quit) return true;
        if (s->pending.empty() || s->free_slots.empty() || s->free_batches.empty()) return false;
        const int f = s->free_batches.back();
        return make_room(s, f, std::max(s->ledger[(size_t)f], s->pending.front()->estimate));
      });
      if (s->quit) return;
      bi = s->free_batches.back();
      s->free_batches.pop_back();
      const int64_t t = now_ns();
      const int64_t others = s->ledger_sum - s->ledger[(size_t)bi];
      const int64_t room = s->desc.budget_bytes - others;
      // admit in arrival order: everything waiting whose estimates fit, up to max_batch
      while (!s->pending.empty() && (int)rs.size() < s->desc.max_batch && !s->free_slots.empty() &&
             est + s->pending.front()->estimate <= room) {
        Request* r = s->pending.front();
        s->pending.pop_front();
        r->slot = s->free_slots.back();
        s->free_slots.pop_back();
        est += r->estimate;
        r->batch = bi;
        r->state = 1;
        r->admit = t;
        rs.push_back(r);
      }
      // the batch graph may grow to twice the estimate (never past the room
      // left): estimates are not bounds, and a graph that would pass its cap
      // fails cleanly and its requests are admitted again with larger ones
      const int64_t cap = std::min<int64_t>(room, std::max<int64_t>(std::max<int64_t>(2 * est, est + ((int64_t)64 << 20)), s->ledger[(size_t)bi]));
      set_ledger(s, bi, cap);
      graph_set_mem_cap(s->batches[(size_t)bi].g, (size_t)cap);
    }
    Batch& b = s->batches[(size_t)bi];
    trace("worker: batch admitted");
    int32_t n_tot = 0;
    int64_t R_tot = 0;
    for (Request* r : rs) {
      r->toff = n_tot;
      n_tot += r->n;
      R_tot += r->req_off[(size_t)r->n];
    }
    const int B = (int)rs.size();
    rt_status st = build_union(s, b, rs, n_tot, R_tot);
    std::string why = st == RT_OK ? std::string() : std::string("pinned staging for the batch");
    GraphView v{};
    if (st == RT_OK && n_tot > 0) {
      st = rt_graph_clear(b.g);
      if (st == RT_OK)
        st = rt_launch_batch(b.g, n_tot, static_cast<int32_t*>(b.req_off.p), static_cast<int64_t*>(b.lo.p),
                             static_cast<int64_t*>(b.hi.p), static_cast<uint8_t*>(b.priv.p), nullptr, nullptr,
                             nullptr, RT_LAUNCH_DEFER_CHECK);
      if (st == RT_OK) st = rt_analyze(b.g);
      if (st == RT_OK) st = graph_view(b.g, &v);
      if (st != RT_OK) why = last_err();
      if (st == RT_OK) {
        // each request's first root and first edge in the batch graph
        for (int j = 0; j < B; ++j) b.hidx[j] = rs[(size_t)j]->toff;
        b.hidx[B] = n_tot;
        if (cudaMemcpyAsync(b.gidx, b.hidx, (size_t)(B + 1) * 4, cudaMemcpyHostToDevice, b.stream) != cudaSuccess)
          st = RT_ERR_CUDA;
        launch_serve_gather(v.rootpos, v.row_ptr, b.gidx, B + 1, b.gout, b.stream);
        if (st == RT_OK &&
            (cudaMemcpyAsync(b.hout, b.gout, (size_t)(B + 1) * 8, cudaMemcpyDeviceToHost, b.stream) != cudaSuccess ||
             cudaStreamSynchronize(b.stream) != cudaSuccess))
          st = RT_ERR_CUDA;
        if (st != RT_OK) why = "root and edge offsets of the batch";
      }
      if (st == RT_OK) {
        // The entries must be in device memory before the kernel can see the
        // posts. A synchronous copy from pageable memory may return before its
        // DMA has landed, so they are staged in pinned memory and the stream
        // is waited for.
        trace("worker: analysed, writing table");
        for (int j = 0; j < B && st == RT_OK; ++j) {
          Request* r = rs[(size_t)j];
          if (r->n == 0) continue;
          ServeSlot e{};
          e.adj = v.adj;
          e.col = v.col;
          e.count = v.count;
          e.roots = v.roots + b.hout[2 * j];
          e.out = b.out;
          e.n_tasks = r->n;
          e.n_roots = (int32_t)(b.hout[2 * j + 2] - b.hout[2 * j]);
          e.body = s->desc.body;
          e.spin_iters = s->desc.spin_iters;
          e.gen = ++s->slots[(size_t)r->slot].gen;
          e.base = r->toff;
          r->band = j;
          if (s->desc.body == RT_BODY_CHECK) {
            e.req_off = v.req_off;
            e.lo = v.lo;
            e.hi = v.hi;
            e.priv = v.priv;
            e.state = b.state + (size_t)j * (size_t)s->cells;
            e.band_lo[0] = s->desc.dom_lo[0];
            e.band_lo[1] = s->desc.ndim == 2 ? s->desc.dom_lo[1] : 0;
            e.band_lo[s->stack_dim] += (int64_t)j * s->band;
            e.ext0 = s->desc.dom_hi[0] - s->desc.dom_lo[0] + 1;
            e.ndim = s->desc.ndim;
          }
          s->table_h[r->slot] = e;
          if (cudaMemcpyAsync(s->table + r->slot, s->table_h + r->slot, sizeof e, cudaMemcpyHostToDevice,
                              b.stream) != cudaSuccess)
            st = RT_ERR_CUDA;
        }
        // CHECK: every request of the batch starts from a zero state
        if (st == RT_OK && s->desc.body == RT_BODY_CHECK &&
            cudaMemsetAsync(b.state, 0, (size_t)B * (size_t)s->cells * 4, b.stream) != cudaSuccess)
          st = RT_ERR_CUDA;
        if (st == RT_OK && cudaStreamSynchronize(b.stream) != cudaSuccess) st = RT_ERR_CUDA;
        if (st != RT_OK) why = "slot table write";
        trace("worker: table written");
      }
    }
    std::vector<int> post;
    const int64_t fp = (int64_t)graph_footprint(b.g);  // this worker owns the graph until it is posted
    {
      std::lock_guard<std::mutex> lk(s->mu);
      if (st == RT_ERR_BUDGET) {
        // the batch outgrew its cap: release what the graph holds and admit its
        // requests again, first in line, with twice their estimates (a request
        // that failed with the whole budget as its estimate can never fit)
        graph_trim(b.g);
        set_ledger(s, bi, 0);
        set_held(s, bi, 0);
        ++s->n_retries;
        for (size_t j = rs.size(); j-- > 0;) {
          Request* r = rs[j];
          s->free_slots.push_back(r->slot);
          r->slot = -1;
          r->batch = -1;
          if (r->estimate >= s->desc.budget_bytes) {
            fail_request(r, RT_ERR_BUDGET, "request does not fit the memory budget: " + why);
            --s->outstanding;
          } else {
            r->estimate = std::min(2 * r->estimate, s->desc.budget_bytes);
            r->state = 0;
            s->pending.push_front(r);
          }
        }
        s->free_batches.push_back(bi);
      } else if (st != RT_OK) {
        for (Request* r : rs) {
          fail_request(r, st, why);
          s->free_slots.push_back(r->slot);
          --s->outstanding;
        }
        set_ledger(s, bi, fp);
        set_held(s, bi, fp);
        s->free_batches.push_back(bi);
      } else {
        // the graph keeps what it holds (at most its cap) for the next batch
        b.footprint = fp;
        set_ledger(s, bi, fp);
        set_held(s, bi, fp);
        for (Request* r : rs) {  // the batch has its own copy of the launches now
          std::vector<int32_t>().swap(r->req_off);
          std::vector<int64_t>().swap(r->lo);
          std::vector<int64_t>().swap(r->hi);
          std::vector<uint8_t>().swap(r->priv);
        }
        ++s->n_batches;
        s->n_batched += B;
        b.live = 0;
        const int64_t t = now_ns();
        for (int j = 0; j < B; ++j) {
          Request* r = rs[(size_t)j];
          r->posted = t;
          r->footprint = n_tot > 0 ? b.footprint * r->n / n_tot : 0;
          if (r->n == 0) {  // nothing to run: done at once
            r->n_edges = 0;
            r->state = 3;
            r->done = t;
            s->free_slots.push_back(r->slot);
            --s->outstanding;
            continue;
          }
          r->eoff = b.hout[2 * j + 1];
          r->n_edges = (int64_t)b.hout[2 * j + 3] - (int64_t)b.hout[2 * j + 1];
          r->state = 2;
          s->slots[(size_t)r->slot].req = r;
          s->running.push_back(r->slot);
          post.push_back(r->slot);
          ++b.live;
        }
        if (b.live == 0) s->free_batches.push_back(bi);
      }
      s->cv.notify_all();
      s->cv_done.notify_all();
    }
    if (!post.empty()) {
      std::lock_guard<std::mutex> lk(s->post_mu);
      const uint32_t k = s->mail->posted;
      for (size_t i = 0; i < post.size(); ++i) s->mail->queue[(k + (uint32_t)i) % 1024u] = (uint32_t)post[i];
      std::atomic_thread_fence(std::memory_order_seq_cst);
      s->mail->posted = k + (uint32_t)post.size();
      std::atomic_thread_fence(std::memory_order_seq_cst);
    }
  }
}

// Copies one finished request's part of its batch's CSR (and SPIN outputs)
// back, renumbered from its own first task and edge.
void copy_results(rt_server* s, Request* r) {
  Batch& b = s->batches[(size_t)r->batch];
  GraphView v{};
  if (graph_view(b.g, &v) != RT_OK) return;
  r->row_ptr.resize((size_t)r->n + 1);
  r->col.resize((size_t)r->n_edges);
  cudaMemcpyAsync(r->row_ptr.data(), v.row_ptr + r->toff, ((size_t)r->n + 1) * 4, cudaMemcpyDeviceToHost,
                  s->copy_stream);
  if (r->n_edges)
    cudaMemcpyAsync(r->col.data(), v.col + r->eoff, (size_t)r->n_edges * 4, cudaMemcpyDeviceToHost, s->copy_stream);
  if (s->desc.body == RT_BODY_SPIN || s->desc.body == RT_BODY_CHECK) {
    r->out.resize((size_t)r->n);
    cudaMemcpyAsync(r->out.data(), b.out + r->toff, (size_t)r->n * 4, cudaMemcpyDeviceToHost, s->copy_stream);
  }
  if (s->desc.body == RT_BODY_CHECK) {
    r->cells.resize((size_t)s->cells);
    cudaMemcpyAsync(r->cells.data(), b.state + (size_t)r->band * (size_t)s->cells, (size_t)s->cells * 4,
                    cudaMemcpyDeviceToHost, s->copy_stream);
  }
  cudaStreamSynchronize(s->copy_stream);
  const int32_t e0 = r->row_ptr[0];
  for (int32_t& x : r->row_ptr) x -= e0;
  for (int32_t& x : r->col) x -= r->toff;
}

void completer_main(rt_server* s) {
  cudaSetDevice(s->device);
  std::vector<int> done_slots;
  while (!s->quit) {
    done_slots.clear();
    {
      std::lock_guard<std::mutex> lk(s->mu);
      for (size_t i = 0; i < s->running.size();) {
        const int slot = s->running[i];
        if (*(volatile uint32_t*)&s->done_gen[slot] == s->slots[(size_t)slot].gen) {
          done_slots.push_back(slot);
          s->running[i] = s->running.back();
          s->running.pop_back();
        } else {
          ++i;
        }
      }
    }
    const int64_t t = now_ns();
    for (int slot : done_slots) {
      Request* r = s->slots[(size_t)slot].req;
      r->done = t;
      if (s->desc.keep_results) copy_results(s, r);
      std::lock_guard<std::mutex> lk(s->mu);
      r->state = 3;
      s->slots[(size_t)slot].req = nullptr;
      s->free_slots.push_back(slot);
      --s->outstanding;
      Batch& b = s->batches[(size_t)r->batch];
      if (--b.live == 0) s->free_batches.push_back(r->batch);  // its graph is free again (buffers retained)
    }
    if (!done_slots.empty()) {
      std::lock_guard<std::mutex> lk(s->mu);
      s->cv.notify_all();
      s->cv_done.notify_all();
    } else {
      // the serving kernel may have stopped with an error
      if (cudaStreamQuery(s->exec_stream) == cudaSuccess) {
        std::lock_guard<std::mutex> lk(s->mu);
        if (!s->stopping && s->fatal.empty()) s->fatal = "serving kernel ended";
        s->cv_done.notify_all();
      }
      std::this_thread::sleep_for(std::chrono::microseconds(20));
    }
  }
}

rt_status sfail(rt_status st, const std::string& m) {
  set_last_error(m.c_str());
  return st;
}

unsigned long long next_pow2(unsigned long long v) {
  unsigned long long p = 1;
  while (p < v) p <<= 1;
  return p;
}

void free_host(HostBuf& b) {
  if (b.p) cudaFreeHost(b.p);
  b.p = nullptr;
  b.cap = 0;
}

void free_server(rt_server* s) {
  for (Batch& b : s->batches) {
    if (b.g) rt_graph_destroy(b.g);
    if (b.stream) cudaStreamDestroy(b.stream);
    if (b.out) cudaFree(b.out);
    if (b.state) cudaFree(b.state);
    if (b.gidx) cudaFree(b.gidx);
    if (b.gout) cudaFree(b.gout);
    if (b.hidx) cudaFreeHost(b.hidx);
    if (b.hout) cudaFreeHost(b.hout);
    free_host(b.req_off);
    free_host(b.lo);
    free_host(b.hi);
    free_host(b.priv);
  }
  for (HostBuf& h : s->retired) free_host(h);
  if (s->table) cudaFree(s->table);
  if (s->done_s) cudaFree(s->done_s);
  if (s->ctrl) cudaFree(s->ctrl);
  if (s->items) cudaFree(s->items);
  if (s->seq) cudaFree(s->seq);
  if (s->mail) cudaFreeHost(s->mail);
  if (s->done_gen) cudaFreeHost(s->done_gen);
  if (s->table_h) cudaFreeHost(s->table_h);
  if (s->exec_stream) cudaStreamDestroy(s->exec_stream);
  if (s->copy_stream) cudaStreamDestroy(s->copy_stream);
  delete s;
}

}  // namespace

extern "C" {

int64_t rt_now_ns(void) { return now_ns(); }

rt_status rt_server_create(const rt_server_desc* d, rt_server_t* out) {
  if (!d || !out) return sfail(RT_ERR_INVALID, "NULL argument");
  *out = nullptr;
  if (d->body != RT_BODY_EMPTY && d->body != RT_BODY_SPIN && d->body != RT_BODY_CHECK)
    return sfail(RT_ERR_INVALID, "serving supports EMPTY, SPIN and CHECK bodies");
  if (d->ndim < 1 || d->ndim > 2 || d->max_inflight < 1 || d->max_inflight > 1024 || d->workers < 1 ||
      d->workers > 64 || d->max_tasks < 1 || d->budget_bytes <= 0 || d->spin_iters < 0 || d->exec_warps < 0 ||
      d->exec_warps > 8 || d->exec_blocks < 0 || d->max_batch < 0 || d->max_batch > 1024)
    return sfail(RT_ERR_INVALID, "server descriptor out of range");
  const int mb = d->max_batch > 0 ? d->max_batch : 64;
  if ((int64_t)mb * d->max_tasks > (int64_t)INT32_MAX - 1)
    return sfail(RT_ERR_INVALID, "max_batch x max_tasks must stay below 2^31");
  for (int k = 0; k < d->ndim; ++k)
    if (d->dom_hi[k] < d->dom_lo[k]) return sfail(RT_ERR_INVALID, "empty domain");
  const int sd = d->ndim - 1;
  const int64_t band = d->dom_hi[sd] - d->dom_lo[sd] + 1;
  if (band <= 0 || band > ((int64_t)1 << 52) / mb) return sfail(RT_ERR_INVALID, "domain too long to stack");
  rt_server* s = new (std::nothrow) rt_server();
  if (!s) return sfail(RT_ERR_OOM, "host allocation failed");
  s->desc = *d;
  s->desc.max_batch = mb;
  s->stack_dim = sd;
  s->band = band;
  s->cells = (d->dom_hi[0] - d->dom_lo[0] + 1) * (d->ndim == 2 ? d->dom_hi[1] - d->dom_lo[1] + 1 : 1);
  if (d->body == RT_BODY_CHECK && (s->cells > ((int64_t)1 << 31) || s->cells * mb > ((int64_t)1 << 36))) {
    delete s;
    return sfail(RT_ERR_INVALID, "CHECK serving: the domain's state is too large for max_batch bands");
  }
  if (s->desc.timeout_ns == 0) s->desc.timeout_ns = 2000000000ll;
  auto bail = [&](rt_status st, const std::string& m) {
    free_server(s);
    return sfail(st, m);
  };
  if (cudaGetDevice(&s->device) != cudaSuccess) return bail(RT_ERR_CUDA, "no CUDA device");
  const int M = d->max_inflight;
  s->slots.resize((size_t)M);
  for (int i = 0; i < M; ++i) s->free_slots.push_back(M - 1 - i);
  // enough batch graphs that workers analyse while earlier batches execute
  const int P = std::max(1, std::min(M, 2 * d->workers + 2));
  s->batches.resize((size_t)P);
  for (int i = 0; i < P; ++i) {
    Batch& b = s->batches[(size_t)i];
    if (cudaStreamCreateWithFlags(&b.stream, cudaStreamNonBlocking) != cudaSuccess)
      return bail(RT_ERR_CUDA, "streams");
    if (((d->body == RT_BODY_SPIN || d->body == RT_BODY_CHECK) &&
         cudaMalloc(&b.out, (size_t)mb * d->max_tasks * 4) != cudaSuccess) ||
        (d->body == RT_BODY_CHECK && cudaMalloc(&b.state, (size_t)mb * (size_t)s->cells * 4) != cudaSuccess) ||
        cudaMalloc(&b.gidx, (size_t)(mb + 1) * 4) != cudaSuccess ||
        cudaMalloc(&b.gout, (size_t)(mb + 1) * 8) != cudaSuccess ||
        cudaHostAlloc(&b.hidx, (size_t)(mb + 1) * 4, cudaHostAllocDefault) != cudaSuccess ||
        cudaHostAlloc(&b.hout, (size_t)(mb + 1) * 8, cudaHostAllocDefault) != cudaSuccess)
      return bail(RT_ERR_OOM, "batch buffers");
    rt_graph_desc gd{};
    gd.ndim = d->ndim;
    for (int k = 0; k < 2; ++k) {
      gd.dom_lo[k] = d->dom_lo[k];
      gd.dom_hi[k] = d->dom_hi[k];
    }
    gd.dom_hi[sd] = d->dom_lo[sd] + band * mb - 1;  // max_batch bands
    gd.body = RT_BODY_EMPTY;  // the graph object only analyses; the serving kernel runs the bodies
    gd.stream = b.stream;
    gd.tile_w = d->tile_w;
    gd.tile_h = d->tile_h;
    if (rt_graph_create(&gd, &b.g) != RT_OK) return bail(RT_ERR_INVALID, last_err());
    s->free_batches.push_back(P - 1 - i);
  }
  s->cap = next_pow2((unsigned long long)M * (unsigned long long)d->max_tasks + 4096ull);
  if (cudaMalloc(&s->table, (size_t)M * sizeof(ServeSlot)) != cudaSuccess ||
      cudaMalloc(&s->done_s, (size_t)M * 4) != cudaSuccess || cudaMalloc(&s->ctrl, sizeof(ServeCtrl)) != cudaSuccess ||
      cudaMalloc(&s->items, s->cap * 8) != cudaSuccess || cudaMalloc(&s->seq, s->cap * 8) != cudaSuccess)
    return bail(RT_ERR_OOM, "serving buffers");
  if (cudaHostAlloc(&s->mail, sizeof(ServeMailbox), cudaHostAllocMapped) != cudaSuccess ||
      cudaHostAlloc(&s->done_gen, (size_t)M * 4, cudaHostAllocMapped) != cudaSuccess ||
      cudaHostAlloc(&s->table_h, (size_t)M * sizeof(ServeSlot), cudaHostAllocDefault) != cudaSuccess)
    return bail(RT_ERR_OOM, "mapped host memory");
  memset((void*)s->mail, 0, sizeof(ServeMailbox));
  memset(s->done_gen, 0, (size_t)M * 4);
  if (cudaHostGetDevicePointer((void**)&s->mail_dev, (void*)s->mail, 0) != cudaSuccess ||
      cudaHostGetDevicePointer((void**)&s->done_gen_dev, s->done_gen, 0) != cudaSuccess)
    return bail(RT_ERR_CUDA, "mapped pointers");
  if (cudaStreamCreateWithFlags(&s->exec_stream, cudaStreamNonBlocking) != cudaSuccess ||
      cudaStreamCreateWithFlags(&s->copy_stream, cudaStreamNonBlocking) != cudaSuccess)
    return bail(RT_ERR_CUDA, "streams");
  ServeParams p{};
  p.slots = s->table;
  p.done_s = s->done_s;
  p.ctrl = s->ctrl;
  p.mail = s->mail_dev;
  p.done_gen = s->done_gen_dev;
  p.items = s->items;
  p.seq = s->seq;
  p.cap = s->cap;
  p.max_slots = M;
  p.claim = 8;
  p.keep = 16;
  p.timeout_ns = s->desc.timeout_ns;
  int sms = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, s->device);
  // every kernel of the library is loaded before the serving kernel starts: a
  // lazily loaded kernel (one the workers, or the caller on another stream,
  // launch for the first time) could otherwise wait for it to finish
  preload_all();
  // one tiny analysis per batch graph: first-use host allocations (pinned
  // staging words) happen now, not while the serving kernel runs
  {
    const int32_t ro[2] = {0, 1};
    const int64_t c[2] = {d->dom_lo[0], d->dom_lo[1]};
    const uint8_t pw = RT_WRITE;
    for (Batch& b : s->batches) {
      if (rt_launch_batch(b.g, 1, ro, c, c, &pw, nullptr, nullptr, nullptr, RT_LAUNCH_DEFER_CHECK) != RT_OK ||
          rt_analyze(b.g) != RT_OK || rt_graph_clear(b.g) != RT_OK)
        return bail(RT_ERR_CUDA, "pool warm-up: " + last_err());
    }
  }
  if (cudaDeviceSynchronize() != cudaSuccess) return bail(RT_ERR_CUDA, "kernel preload");
  // the batch graphs' warm-up buffers are the first entries of the budget's ledger
  s->ledger.assign((size_t)P, 0);
  s->held.assign((size_t)P, 0);
  for (int i = 0; i < P; ++i) {
    const int64_t fp = (int64_t)graph_footprint(s->batches[(size_t)i].g);
    if (s->ledger_sum + fp > d->budget_bytes) {
      graph_trim(s->batches[(size_t)i].g);
      continue;
    }
    set_ledger(s, i, fp);
    set_held(s, i, fp);
  }
  s->fixed_bytes = (int64_t)M * (int64_t)(sizeof(ServeSlot) + 4) + (int64_t)sizeof(ServeCtrl) + (int64_t)s->cap * 16;
  for (Batch& b : s->batches) {
    s->fixed_bytes += (int64_t)(mb + 1) * 12;
    if (b.out) s->fixed_bytes += (int64_t)mb * d->max_tasks * 4;
    if (b.state) s->fixed_bytes += (int64_t)mb * s->cells * 4;
  }
  launch_serve_init(p, s->exec_stream);
  // Two warps per SM by default: the kernel stays resident beside the workers'
  // analysis, and with more warps its registers would leave room for only two
  // of the sweep's three blocks per SM.
  launch_serve(p, d->exec_blocks > 0 ? d->exec_blocks : sms, d->exec_warps > 0 ? d->exec_warps : 2, s->exec_stream);
  if (cudaGetLastError() != cudaSuccess) return bail(RT_ERR_CUDA, "serving kernel launch");
  for (int i = 0; i < d->workers; ++i) s->workers.emplace_back(worker_main, s);
  s->completer = std::thread(completer_main, s);
  *out = s;
  return RT_OK;
}

rt_status rt_server_submit(rt_server_t s, int32_t n, const int32_t* req_off, const int64_t* lo, const int64_t* hi,
                           const uint8_t* priv, int64_t arrival_ns, int64_t* ticket) {
  if (!s || !ticket || !req_off || n < 0) return sfail(RT_ERR_INVALID, "bad arguments");
  if (n > s->desc.max_tasks) return sfail(RT_ERR_INVALID, "request has more than max_tasks tasks");
  const int64_t R = req_off[n];
  if (req_off[0] != 0 || R < 0 || (R > 0 && (!lo || !hi || !priv)))
    return sfail(RT_ERR_INVALID, "req_off must start at 0 and rect arrays must be set");
  // Checked here, on the host: a batch shares one domain, so a rectangle
  // outside its request's domain would meet another request's rectangles.
  const int D = s->desc.ndim;
  for (int32_t i = 0; i < n; ++i)
    if (req_off[i + 1] < req_off[i]) return sfail(RT_ERR_INVALID, "req_off decreases at launch " + std::to_string(i));
  for (int64_t r = 0; r < R; ++r) {
    for (int k = 0; k < D; ++k) {
      const int64_t a = lo[r * D + k], b = hi[r * D + k];
      if (a > b || a < s->desc.dom_lo[k] || b > s->desc.dom_hi[k])
        return sfail(RT_ERR_INVALID, "rect " + std::to_string(r) + " empty or outside the domain");
    }
    if (priv[r] > RT_REDUCE_SUM) return sfail(RT_ERR_INVALID, "rect " + std::to_string(r) + ": bad privilege");
  }
  auto q = std::make_unique<Request>();
  q->n = n;
  q->req_off.assign(req_off, req_off + n + 1);
  q->lo.assign(lo, lo + R * D);
  q->hi.assign(hi, hi + R * D);
  q->priv.assign(priv, priv + R);
  q->arrival = arrival_ns;
  q->estimate = estimate_bytes(n, R);
  if (q->estimate > s->desc.budget_bytes) return sfail(RT_ERR_BUDGET, "request can never fit the memory budget");
  std::lock_guard<std::mutex> lk(s->mu);
  if (s->stopping) return sfail(RT_ERR_STATE, "server is stopping");
  q->ticket = s->next_ticket++;
  *ticket = q->ticket;
  s->pending.push_back(q.get());
  ++s->outstanding;
  s->reqs.emplace(q->ticket, std::move(q));
  s->cv.notify_one();
  return RT_OK;
}

rt_status rt_server_poll(rt_server_t s, int64_t ticket, rt_request_info* info) {
  if (!s || !info) return sfail(RT_ERR_INVALID, "NULL argument");
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->reqs.find(ticket);
  if (it == s->reqs.end()) return sfail(RT_ERR_INVALID, "unknown ticket");
  const Request* r = it->second.get();
  info->state = r->state;
  info->status = r->status;
  info->arrival_ns = r->arrival;
  info->admit_ns = r->admit;
  info->posted_ns = r->posted;
  info->done_ns = r->done;
  info->n_tasks = r->n;
  info->n_edges = r->n_edges;
  info->footprint_bytes = r->footprint;
  return RT_OK;
}

rt_status rt_server_result(rt_server_t s, int64_t ticket, int32_t* row_ptr, int32_t* col, int32_t* out) {
  if (!s) return sfail(RT_ERR_INVALID, "NULL server");
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->reqs.find(ticket);
  if (it == s->reqs.end()) return sfail(RT_ERR_INVALID, "unknown ticket");
  const Request* r = it->second.get();
  if (r->state == 4) return sfail((rt_status)r->status, "request failed: " + r->error);
  if (r->state != 3) return sfail(RT_ERR_STATE, "request is not done");
  if (!s->desc.keep_results) return sfail(RT_ERR_STATE, "server does not keep results");
  if (row_ptr) {
    if (r->row_ptr.empty()) row_ptr[0] = 0;  // an empty request
    else memcpy(row_ptr, r->row_ptr.data(), r->row_ptr.size() * 4);
  }
  if (col && !r->col.empty()) memcpy(col, r->col.data(), r->col.size() * 4);
  if (out && !r->out.empty()) memcpy(out, r->out.data(), r->out.size() * 4);
  return RT_OK;
}

rt_status rt_server_result_state(rt_server_t s, int64_t ticket, int32_t* state) {
  if (!s || !state) return sfail(RT_ERR_INVALID, "NULL argument");
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->reqs.find(ticket);
  if (it == s->reqs.end()) return sfail(RT_ERR_INVALID, "unknown ticket");
  const Request* r = it->second.get();
  if (r->state == 4) return sfail((rt_status)r->status, "request failed: " + r->error);
  if (r->state != 3) return sfail(RT_ERR_STATE, "request is not done");
  if (!s->desc.keep_results || s->desc.body != RT_BODY_CHECK)
    return sfail(RT_ERR_STATE, "server does not keep CHECK states");
  if (r->cells.empty()) memset(state, 0, (size_t)s->cells * 4);  // an empty request
  else memcpy(state, r->cells.data(), r->cells.size() * 4);
  return RT_OK;
}

rt_status rt_server_drain(rt_server_t s, int64_t timeout_ns) {
  if (!s) return sfail(RT_ERR_INVALID, "NULL server");
  const int64_t until = now_ns() + (timeout_ns > 0 ? timeout_ns : (int64_t)3600 * 1000000000ll);
  std::unique_lock<std::mutex> lk(s->mu);
  while (s->outstanding > 0) {
    if (!s->fatal.empty()) {
      // describe what is still running: completed tasks vs the request's size
      std::string m = "serving kernel stopped: " + s->fatal;
      uint32_t kst = 0;
      cudaMemcpyAsync(&kst, &s->ctrl->status, 4, cudaMemcpyDeviceToHost, s->copy_stream);
      cudaStreamSynchronize(s->copy_stream);
      m += "; kernel status " + std::to_string(kst);
      int shown = 0;
      for (int slot : s->running) {
        uint32_t d = 0;
        ServeSlot e{};
        cudaMemcpyAsync(&d, s->done_s + slot, 4, cudaMemcpyDeviceToHost, s->copy_stream);
        cudaMemcpyAsync(&e, s->table + slot, sizeof e, cudaMemcpyDeviceToHost, s->copy_stream);
        cudaStreamSynchronize(s->copy_stream);
        m += "; slot " + std::to_string(slot) + ": " + std::to_string(d) + "/" + std::to_string(e.n_tasks) +
             " tasks, roots " + std::to_string(e.n_roots) + ", gen " + std::to_string(e.gen) + "/" +
             std::to_string(s->done_gen[slot]);
        if (++shown == 6) break;
      }
      return sfail(RT_ERR_TIMEOUT, m);
    }
    if (now_ns() > until) {
      int by_state[5] = {0, 0, 0, 0, 0};
      for (auto& kv : s->reqs) by_state[std::min(std::max(kv.second->state, 0), 4)]++;
      uint32_t w[2] = {0, 0};
      cudaMemcpyAsync(&w[0], &s->ctrl->taken, 4, cudaMemcpyDeviceToHost, s->copy_stream);
      cudaMemcpyAsync(&w[1], &s->ctrl->finished, 4, cudaMemcpyDeviceToHost, s->copy_stream);
      cudaStreamSynchronize(s->copy_stream);
      char buf[256];
      snprintf(buf, sizeof buf,
               "drain timed out: %d queued, %d analysing, %d running, %d done, %d failed; posted %u, "
               "taken %u, finished %u",
               by_state[0], by_state[1], by_state[2], by_state[3], by_state[4], s->mail->posted, w[0], w[1]);
      return sfail(RT_ERR_TIMEOUT, buf);
    }
    s->cv_done.wait_for(lk, std::chrono::milliseconds(5));
  }
  return RT_OK;
}

rt_status rt_server_stats(rt_server_t s, int64_t* out, int32_t n) {
  if (!s || !out || n < 0) return sfail(RT_ERR_INVALID, "NULL argument");
  uint32_t w[3] = {0, 0, 0};
  unsigned long long ex = 0;
  cudaMemcpyAsync(&w[0], &s->ctrl->taken, 4, cudaMemcpyDeviceToHost, s->copy_stream);
  cudaMemcpyAsync(&w[1], &s->ctrl->finished, 4, cudaMemcpyDeviceToHost, s->copy_stream);
  cudaMemcpyAsync(&w[2], &s->ctrl->status, 4, cudaMemcpyDeviceToHost, s->copy_stream);
  cudaMemcpyAsync(&ex, &s->ctrl->executed, 8, cudaMemcpyDeviceToHost, s->copy_stream);
  if (cudaStreamSynchronize(s->copy_stream) != cudaSuccess) return sfail(RT_ERR_CUDA, "stats copy");
  int64_t v[18];
  v[0] = s->mail->posted;
  v[1] = w[0];
  v[2] = w[1];
  v[3] = w[2];
  v[4] = (int64_t)ex;
  int by_state[5] = {0, 0, 0, 0, 0};
  {
    std::lock_guard<std::mutex> lk(s->mu);
    for (auto& kv : s->reqs) by_state[std::min(std::max(kv.second->state, 0), 4)]++;
    v[9] = s->n_batches;
    v[10] = s->n_batched;
    v[11] = s->ledger_sum;
    v[12] = s->ledger_peak;
    v[13] = s->held_sum;
    v[14] = s->held_peak;
    v[15] = s->fixed_bytes;
    v[16] = s->n_trims;
    v[17] = s->n_retries;
  }
  v[5] = by_state[0];
  v[6] = by_state[1];
  v[7] = by_state[2];
  v[8] = cudaStreamQuery(s->exec_stream) == cudaErrorNotReady ? 1 : 0;
  for (int k = 0; k < n && k < 18; ++k) out[k] = v[k];
  return RT_OK;
}
rt_status rt_server_destroy(rt_server_t s) {
  if (!s) return RT_OK;
  rt_status st = rt_server_drain(s, 30ll * 1000000000ll);
  const std::string drain_msg = st != RT_OK ? std::string(rt_last_error()) : std::string();
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stopping = true;
  }
  // ask the kernel to leave once idle; if it does not within 10 s, force it
  auto wait_kernel = [&](int64_t ns) {
    const int64_t until = now_ns() + ns;
    while (cudaStreamQuery(s->exec_stream) == cudaErrorNotReady) {
      if (now_ns() > until) return false;
      std::this_thread::sleep_for(std::chrono::milliseconds(1));
    }
    return true;
  };
  {
    std::lock_guard<std::mutex> lk(s->post_mu);
    s->mail->stop = 1;
    std::atomic_thread_fence(std::memory_order_seq_cst);
  }
  bool ended = wait_kernel(10ll * 1000000000ll);
  if (!ended) {
    s->mail->stop = 2;
    std::atomic_thread_fence(std::memory_order_seq_cst);
    ended = wait_kernel(10ll * 1000000000ll);
  }
  s->quit = true;
  s->cv.notify_all();
  if (!ended) {
    // the kernel still runs: its buffers cannot be freed; leave them (and the
    // threads) to the process exit instead of blocking here
    for (auto& t : s->workers) t.detach();
    if (s->completer.joinable()) s->completer.detach();
    return sfail(RT_ERR_TIMEOUT, "serving kernel did not stop; resources left to process exit. " + drain_msg);
  }
  uint32_t kst = 0;
  cudaMemcpy(&kst, &s->ctrl->status, 4, cudaMemcpyDeviceToHost);
  for (auto& t : s->workers) t.join();
  if (s->completer.joinable()) s->completer.join();
  free_server(s);
  if (st != RT_OK) return sfail(st, drain_msg);
  if (kst != 0u) return sfail(RT_ERR_TIMEOUT, "serving kernel reported a stall");
  return RT_OK;
}

}  // extern "C"
