// server.cu -- host side of serving: admission, analysis workers, completion.
//
// Requests queue in arrival order. A worker thread admits the oldest request
// when a slot of the graph pool is free and the device memory the request
// would hold fits the budget, analyses it on the slot's own stream (the same
// GPU analysis as rt_analyze), writes the slot's table entry and posts it
// through the host-mapped mailbox to the serving kernel (serve.cu), which is
// running all the time. A completion thread watches the host-mapped completion
// words, stamps the finish time, copies results back if asked, and frees the
// slot and its budget share. Several requests are analysed concurrently (one
// per worker) while earlier ones execute: continuous batching.
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
  int state = 0, status = 0, slot = -1;
  std::vector<int32_t> row_ptr, col, out;  // results (keep_results)
  std::string error;                       // why it failed (state 4)
};

struct Slot {
  rt_graph_t g = nullptr;
  cudaStream_t stream = nullptr;
  int32_t* out = nullptr;  // SPIN results, max_tasks int32 (device)
  uint32_t gen = 0;
  Request* req = nullptr;
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
  std::vector<Slot> slots;
  std::vector<int> free_slots;
  // device
  ServeSlot* table = nullptr;
  ServeSlot* table_h = nullptr;  // pinned staging: one entry per slot
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
  int64_t budget_used = 0;
  int64_t outstanding = 0;         // submitted, not yet done or failed
  std::mutex post_mu;              // serialises mailbox posts
  bool stopping = false;
  std::atomic<bool> quit{false};
  std::vector<std::thread> workers;
  std::thread completer;
  std::vector<int> running;        // slots posted to the kernel (guarded by mu)
  uint32_t kernel_status = 0;
  std::string fatal;
};

namespace {

int64_t estimate_bytes(int32_t n, int64_t R) {
  // analysis buffers grow with binned entries (a few tiles per rectangle),
  // candidate pairs and the CSR; this bound is replaced by the real footprint
  // once the request has been analysed
  return (8ll << 20) + (int64_t)n * 256 + R * 2048;
}

void fail_request(rt_server* s, Request* r, int status, std::string why) {
  r->error = std::move(why);
  r->state = 4;
  r->status = status;
  r->done = now_ns();
}

void worker_main(rt_server* s) {
  cudaSetDevice(s->device);
  for (;;) {
    Request* r = nullptr;
    int slot = -1;
    {
      std::unique_lock<std::mutex> lk(s->mu);
      s->cv.wait(lk, [&] {
        if (s->quit) return true;
        if (s->pending.empty() || s->free_slots.empty()) return false;
        return s->budget_used + s->pending.front()->estimate <= s->desc.budget_bytes;
      });
      if (s->quit) return;
      r = s->pending.front();
      s->pending.pop_front();
      slot = s->free_slots.back();
      s->free_slots.pop_back();
      s->budget_used += r->estimate;
      r->slot = slot;
      r->state = 1;
      r->admit = now_ns();
    }
    Slot& sl = s->slots[(size_t)slot];
    trace("worker: admitted");
    rt_status st = rt_graph_clear(sl.g);
    if (st == RT_OK)
      st = rt_launch_batch(sl.g, r->n, r->req_off.data(), r->lo.data(), r->hi.data(), r->priv.data(), nullptr,
                           nullptr, nullptr, RT_LAUNCH_DEFER_CHECK);
    if (st == RT_OK) st = rt_analyze(sl.g);
    GraphView v{};
    if (st == RT_OK) st = graph_view(sl.g, &v);
    if (st == RT_OK) {
      ServeSlot e{};
      e.adj = v.adj;
      e.col = v.col;
      e.count = v.count;
      e.roots = v.roots;
      e.out = sl.out;
      e.n_tasks = v.n;
      e.n_roots = v.n_roots;
      e.body = s->desc.body;
      e.spin_iters = s->desc.spin_iters;
      e.gen = ++sl.gen;
      // The entry must be in device memory before the kernel can see the
      // post. A synchronous copy from pageable memory may return before its
      // DMA has landed, so stage it in pinned memory and wait for the stream.
      trace("worker: analysed, writing table");
      s->table_h[slot] = e;
      if (cudaMemcpyAsync(s->table + slot, s->table_h + slot, sizeof e, cudaMemcpyHostToDevice, sl.stream) !=
              cudaSuccess ||
          cudaStreamSynchronize(sl.stream) != cudaSuccess)
        st = RT_ERR_CUDA;
      trace("worker: table written");
    }
    if (st != RT_OK) {
      std::lock_guard<std::mutex> lk(s->mu);
      fail_request(s, r, st, last_err());
      s->budget_used -= r->estimate;
      s->free_slots.push_back(slot);
      --s->outstanding;
      s->cv.notify_all();
      s->cv_done.notify_all();
      continue;
    }
    {
      std::lock_guard<std::mutex> lk(s->mu);
      s->budget_used += (int64_t)v.footprint - r->estimate;
      r->footprint = (int64_t)v.footprint;
      r->n_edges = v.n_edges;
      r->posted = now_ns();
      r->state = 2;
      sl.req = r;
      if (v.n == 0) {  // nothing to run: done at once
        r->state = 3;
        r->done = r->posted;
        sl.req = nullptr;
        s->budget_used -= r->footprint;
        s->free_slots.push_back(slot);
        --s->outstanding;
        s->cv.notify_all();
        s->cv_done.notify_all();
        continue;
      }
      s->running.push_back(slot);
    }
    {
      std::lock_guard<std::mutex> lk(s->post_mu);
      const uint32_t k = s->mail->posted;
      s->mail->queue[k % 1024u] = (uint32_t)slot;
      std::atomic_thread_fence(std::memory_order_seq_cst);
      s->mail->posted = k + 1;
      std::atomic_thread_fence(std::memory_order_seq_cst);
    }
  }
}

void completer_main(rt_server* s) {
  cudaSetDevice(s->device);
  while (!s->quit) {
    std::vector<int> done_slots;
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
      Slot& sl = s->slots[(size_t)slot];
      Request* r = sl.req;
      r->done = t;
      if (s->desc.keep_results) {
        r->row_ptr.resize((size_t)r->n + 1);
        r->col.resize((size_t)std::max<int64_t>(r->n_edges, 1));
        rt_copy_csr(sl.g, r->row_ptr.data(), r->col.data(), nullptr);
        r->col.resize((size_t)r->n_edges);
        if (s->desc.body == RT_BODY_SPIN) {
          r->out.resize((size_t)r->n);
          cudaMemcpy(r->out.data(), sl.out, (size_t)r->n * 4, cudaMemcpyDeviceToHost);
        }
      }
      std::lock_guard<std::mutex> lk(s->mu);
      r->state = 3;
      sl.req = nullptr;
      s->budget_used -= r->footprint;
      s->free_slots.push_back(slot);
      --s->outstanding;
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

}  // namespace

namespace {
rt_status sfail(rt_status st, const std::string& m) {
  set_last_error(m.c_str());
  return st;
}

unsigned long long next_pow2(unsigned long long v) {
  unsigned long long p = 1;
  while (p < v) p <<= 1;
  return p;
}

void free_server(rt_server* s) {
  for (Slot& sl : s->slots) {
    if (sl.g) rt_graph_destroy(sl.g);
    if (sl.stream) cudaStreamDestroy(sl.stream);
    if (sl.out) cudaFree(sl.out);
  }
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
  if (d->body != RT_BODY_EMPTY && d->body != RT_BODY_SPIN)
    return sfail(RT_ERR_INVALID, "serving supports EMPTY and SPIN bodies");
  if (d->max_inflight < 1 || d->max_inflight > 1024 || d->workers < 1 || d->workers > 64 || d->max_tasks < 1 ||
      d->budget_bytes <= 0 || d->spin_iters < 0 || d->exec_warps < 0 || d->exec_warps > 8 || d->exec_blocks < 0)
    return sfail(RT_ERR_INVALID, "server descriptor out of range");
  rt_server* s = new (std::nothrow) rt_server();
  if (!s) return sfail(RT_ERR_OOM, "host allocation failed");
  s->desc = *d;
  if (s->desc.timeout_ns == 0) s->desc.timeout_ns = 2000000000ll;
  auto bail = [&](rt_status st, const std::string& m) {
    free_server(s);
    return sfail(st, m);
  };
  if (cudaGetDevice(&s->device) != cudaSuccess) return bail(RT_ERR_CUDA, "no CUDA device");
  const int M = d->max_inflight;
  s->slots.resize((size_t)M);
  for (int i = 0; i < M; ++i) {
    Slot& sl = s->slots[(size_t)i];
    if (d->body == RT_BODY_SPIN && cudaMalloc(&sl.out, (size_t)d->max_tasks * 4) != cudaSuccess)
      return bail(RT_ERR_OOM, "slot output buffers");
    if (cudaStreamCreateWithFlags(&sl.stream, cudaStreamNonBlocking) != cudaSuccess)
      return bail(RT_ERR_CUDA, "streams");
    cudaStream_t st = sl.stream;
    rt_graph_desc gd{};
    gd.ndim = d->ndim;
    for (int k = 0; k < 2; ++k) {
      gd.dom_lo[k] = d->dom_lo[k];
      gd.dom_hi[k] = d->dom_hi[k];
    }
    gd.body = RT_BODY_EMPTY;  // the graph object only analyses; the serving kernel runs the bodies
    gd.stream = st;
    gd.tile_w = d->tile_w;
    gd.tile_h = d->tile_h;
    if (rt_graph_create(&gd, &sl.g) != RT_OK) return bail(RT_ERR_INVALID, last_err());
    s->free_slots.push_back(M - 1 - i);
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
  // every kernel the workers will launch is loaded before the serving kernel
  // starts: a lazily loaded kernel could otherwise wait for it to finish
  preload_primitives();
  preload_analysis();
  preload_sweep();
  preload_exec();
  preload_serve();
  // one tiny analysis per pool graph: first-use host allocations (pinned
  // staging words) happen now, not while the serving kernel runs
  {
    const int32_t ro[2] = {0, 1};
    const int64_t c[2] = {d->dom_lo[0], d->dom_lo[1]};
    const uint8_t pw = RT_WRITE;
    for (Slot& sl : s->slots) {
      if (rt_launch_batch(sl.g, 1, ro, c, c, &pw, nullptr, nullptr, nullptr, RT_LAUNCH_DEFER_CHECK) != RT_OK ||
          rt_analyze(sl.g) != RT_OK || rt_graph_clear(sl.g) != RT_OK)
        return bail(RT_ERR_CUDA, "pool warm-up: " + last_err());
    }
  }
  if (cudaDeviceSynchronize() != cudaSuccess) return bail(RT_ERR_CUDA, "kernel preload");
  launch_serve_init(p, s->exec_stream);
  launch_serve(p, d->exec_blocks > 0 ? d->exec_blocks : sms, d->exec_warps > 0 ? d->exec_warps : 4, s->exec_stream);
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
  const int D = s->desc.ndim;
  auto r = std::make_unique<Request>();
  r->n = n;
  r->req_off.assign(req_off, req_off + n + 1);
  r->lo.assign(lo, lo + R * D);
  r->hi.assign(hi, hi + R * D);
  r->priv.assign(priv, priv + R);
  r->arrival = arrival_ns;
  r->estimate = estimate_bytes(n, R);
  if (r->estimate > s->desc.budget_bytes) return sfail(RT_ERR_BUDGET, "request can never fit the memory budget");
  std::lock_guard<std::mutex> lk(s->mu);
  if (s->stopping) return sfail(RT_ERR_STATE, "server is stopping");
  r->ticket = s->next_ticket++;
  *ticket = r->ticket;
  s->pending.push_back(r.get());
  ++s->outstanding;
  s->reqs.emplace(r->ticket, std::move(r));
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
  if (row_ptr) memcpy(row_ptr, r->row_ptr.data(), r->row_ptr.size() * 4);
  if (col) memcpy(col, r->col.data(), r->col.size() * 4);
  if (out && !r->out.empty()) memcpy(out, r->out.data(), r->out.size() * 4);
  return RT_OK;
}

rt_status rt_server_drain(rt_server_t s, int64_t timeout_ns) {
  if (!s) return sfail(RT_ERR_INVALID, "NULL server");
  const int64_t until = now_ns() + (timeout_ns > 0 ? timeout_ns : (int64_t)3600 * 1000000000ll);
  std::unique_lock<std::mutex> lk(s->mu);
  while (s->outstanding > 0) {
    if (!s->fatal.empty()) {
      // describe what is still running: completed tasks vs the graph's size
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
      unsigned long long info[2] = {0, 0};
      cudaMemcpyAsync(info, &s->ctrl->taken, 4, cudaMemcpyDeviceToHost, s->copy_stream);
      cudaMemcpyAsync(info + 1, &s->ctrl->finished, 4, cudaMemcpyDeviceToHost, s->copy_stream);
      cudaStreamSynchronize(s->copy_stream);
      char buf[256];
      snprintf(buf, sizeof buf,
               "drain timed out: %d queued, %d analysing, %d running, %d done, %d failed; posted %u, "
               "taken %u, finished %u",
               by_state[0], by_state[1], by_state[2], by_state[3], by_state[4], s->mail->posted,
               (unsigned)info[0], (unsigned)info[1]);
      return sfail(RT_ERR_TIMEOUT, buf);
    }
    s->cv_done.wait_for(lk, std::chrono::milliseconds(5));
  }
  return RT_OK;
}

rt_status rt_server_stats(rt_server_t s, int64_t* out, int32_t n) {
  if (!s || !out || n < 0) return sfail(RT_ERR_INVALID, "NULL argument");
  unsigned int w[4] = {0, 0, 0, 0};
  unsigned long long ex = 0;
  cudaMemcpyAsync(&w[0], &s->ctrl->taken, 4, cudaMemcpyDeviceToHost, s->copy_stream);
  cudaMemcpyAsync(&w[1], &s->ctrl->finished, 4, cudaMemcpyDeviceToHost, s->copy_stream);
  cudaMemcpyAsync(&w[2], &s->ctrl->status, 4, cudaMemcpyDeviceToHost, s->copy_stream);
  cudaMemcpyAsync(&ex, &s->ctrl->executed, 8, cudaMemcpyDeviceToHost, s->copy_stream);
  if (cudaStreamSynchronize(s->copy_stream) != cudaSuccess) return sfail(RT_ERR_CUDA, "stats copy");
  int64_t v[9];
  v[0] = s->mail->posted;
  v[1] = w[0];
  v[2] = w[1];
  v[3] = w[2];
  v[4] = (int64_t)ex;
  int by_state[5] = {0, 0, 0, 0, 0};
  {
    std::lock_guard<std::mutex> lk(s->mu);
    for (auto& kv : s->reqs) by_state[std::min(std::max(kv.second->state, 0), 4)]++;
  }
  v[5] = by_state[0];
  v[6] = by_state[1];
  v[7] = by_state[2];
  v[8] = cudaStreamQuery(s->exec_stream) == cudaErrorNotReady ? 1 : 0;
  for (int k = 0; k < n && k < 9; ++k) out[k] = v[k];
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
