// static_exec.cu -- executor entry point that allocates nothing.
//
// Some callers cannot allocate device memory at the point where they want to
// run a graph: code running inside a memory-pool or arena manager that forbids
// stray cudaMalloc calls, real-time loops where an allocation (and the
// device-wide synchronisation cudaFree implies) is not acceptable, or plugins
// embedded in a host process that owns all device memory. For them,
// rt_execute_csr_static runs the persistent executor over a CSR the caller
// already holds, with the executor's scratch (countdown counters, ready ring,
// trigger records, control block, graph table) in one file-scope device array
// instead of library-allocated buffers.
//
// With a caller-owned tickets buffer the executor also records each task's
// start and finish ticket (one global counter), so that a caller can check
// that every edge was respected.
//
// Limits and sharing: the array holds kStaticMaxTasks tasks worth of scratch
// (about 11 MB) and stays resident on every device that loads the library until
// the process exits. All calls share it and it keeps the previous call's
// contents, so each call first clears what must start from a known state;
// calls whose GPU work overlaps (different streams, or host threads racing)
// corrupt each other and must be serialised by the caller.
#include <mutex>

#include "grt_internal.cuh"

namespace grt {

namespace {

constexpr int32_t kStaticMaxTasks = 1 << 18;
constexpr size_t kOffCtrl = 0;                        // ExecCtrl (640 bytes)
constexpr size_t kOffDone = 1024;                     // one uint32 per graph (1 graph)
constexpr size_t kOffTable = 1280;                    // one ExecGraph
constexpr size_t kOffCount = 2048;                    // int32 [kStaticMaxTasks]
constexpr size_t kOffRing = kOffCount + (size_t)kStaticMaxTasks * 4;  // uint64 [max + 64]
constexpr size_t kOffAdj = kOffRing + ((size_t)kStaticMaxTasks + 64) * 8;  // int4 [2 * max]
constexpr size_t kStaticBytes = kOffAdj + (size_t)kStaticMaxTasks * 32;

static __device__ __align__(256) unsigned char g_static_scratch[kStaticBytes];

static_assert(sizeof(ExecCtrl) <= kOffDone - kOffCtrl, "control block does not fit");
static_assert(sizeof(ExecGraph) <= kOffCount - kOffTable, "graph table does not fit");

std::mutex g_setup_mu;
void* g_static_ptr[64] = {};  // device address of g_static_scratch, per device ordinal

// Resets the scratch for one run: counters from in-degrees, an empty ring,
// fresh control words, the one-entry graph table; then seeds the roots.
__global__ void k_static_reset(const int32_t* indeg, int32_t n, int32_t spin_iters, int32_t* out) {
  unsigned char* base = g_static_scratch;
  int32_t* count = reinterpret_cast<int32_t*>(base + kOffCount);
  uint64_t* ring = reinterpret_cast<uint64_t*>(base + kOffRing);
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t v = i; v < n + 64; v += stride) {
    if (v < n) count[v] = indeg[v];
    ring[v] = kEmpty64;
  }
  if (i == 0) {
    ExecCtrl* c = reinterpret_cast<ExecCtrl*>(base + kOffCtrl);
    c->head = 0;
    c->tail = 0;
    c->graphs_done = 0;
    c->status = 0;
    c->executed = 0;
    c->ticket = 0;
    c->err_where = 0;
    c->err_info = 0;
    for (int k = 0; k < kCntCount; ++k) c->counters[k] = 0;
    *reinterpret_cast<uint32_t*>(base + kOffDone) = 0u;
    ExecGraph G{};
    G.task_base = 0;
    G.n_tasks = n;
    G.body = RT_BODY_SPIN;
    G.spin_iters = spin_iters;
    G.ndim = 1;
    G.out = out;
    G.ext[0] = 1;
    G.ext[1] = 1;
    *reinterpret_cast<ExecGraph*>(base + kOffTable) = G;
  }
}

__global__ void k_static_seed(const int32_t* indeg, int32_t n) {
  unsigned char* base = g_static_scratch;
  uint64_t* ring = reinterpret_cast<uint64_t*>(base + kOffRing);
  ExecCtrl* c = reinterpret_cast<ExecCtrl*>(base + kOffCtrl);
  const int32_t v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v < n && indeg[v] == 0) ring[atomicAdd(&c->tail, 1u)] = (uint64_t)(uint32_t)v;
}

// Validation, in two launches so that `col` is read only through row offsets
// already known to be sane: (1) row_ptr[0] == 0, non-decreasing, row_ptr[n] ==
// n_edges; (2) every column is a later task (the graph is then acyclic) and the
// in-degrees match the columns. Problems set bits in the control block.
__global__ void k_static_check_rows(const int32_t* row_ptr, int32_t n, int64_t n_edges) {
  unsigned char* base = g_static_scratch;
  ExecCtrl* c = reinterpret_cast<ExecCtrl*>(base + kOffCtrl);
  int32_t* count = reinterpret_cast<int32_t*>(base + kOffCount);
  const int32_t v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v > n) return;
  if (v < n) count[v] = 0;
  uint32_t bad = 0;
  if (v == 0 && row_ptr[0] != 0) bad = 1u;
  if (v == n && (int64_t)row_ptr[n] != n_edges) bad = 1u;
  if (v < n && row_ptr[v + 1] < row_ptr[v]) bad = 1u;
  if (bad) atomicOr(&c->err_info, bad);
}

__global__ void k_static_check_cols(const int32_t* row_ptr, const int32_t* col, int32_t n) {
  unsigned char* base = g_static_scratch;
  ExecCtrl* c = reinterpret_cast<ExecCtrl*>(base + kOffCtrl);
  int32_t* count = reinterpret_cast<int32_t*>(base + kOffCount);
  const int32_t v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= n) return;
  for (int32_t e = row_ptr[v]; e < row_ptr[v + 1]; ++e) {
    const int32_t s = col[e];
    if (s <= v || s >= n) {
      atomicOr(&c->err_info, 2u);
      return;
    }
    atomicAdd(&count[s], 1);
  }
}

__global__ void k_static_check_indeg(const int32_t* indeg, int32_t n) {
  unsigned char* base = g_static_scratch;
  ExecCtrl* c = reinterpret_cast<ExecCtrl*>(base + kOffCtrl);
  const int32_t* count = reinterpret_cast<const int32_t*>(base + kOffCount);
  const int32_t v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v < n && count[v] != indeg[v]) atomicOr(&c->err_info, 4u);
}

__global__ void k_static_clear_err() {
  reinterpret_cast<ExecCtrl*>(g_static_scratch + kOffCtrl)->err_info = 0u;
}

// device address of the array on the current device (looked up once per device)
cudaError_t static_scratch(void** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lk(g_setup_mu);
  if (!g_static_ptr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_static_scratch);
    if (e != cudaSuccess) return e;
    g_static_ptr[dev] = p;
  }
  *out = g_static_ptr[dev];
  return cudaSuccess;
}

}  // namespace

int32_t static_max_tasks() { return kStaticMaxTasks; }

rt_status static_execute(const int32_t* row_ptr, const int32_t* col, const int32_t* indeg, int32_t n,
                         int64_t n_edges, int32_t spin_iters, int32_t* out, int32_t* tickets, cudaStream_t s,
                         int64_t timeout_ns, const char** why) {
  // an error left pending by earlier, unrelated work is reported as such (and
  // left pending), not taken for a failure of the launches below
  cudaError_t e = cudaPeekAtLastError();
  if (e != cudaSuccess) {
    *why = "a CUDA error was already pending before the call";
    return RT_ERR_CUDA;
  }
  // the call reads back validation flags and the status with synchronous
  // copies into host memory, which a stream capture cannot hold
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  e = cudaStreamIsCapturing(s, &cap);
  if (e != cudaSuccess) {
    *why = cudaGetErrorString(e);
    return RT_ERR_CUDA;
  }
  if (cap != cudaStreamCaptureStatusNone) {
    *why = "the stream is being captured; this call is synchronous and cannot be captured";
    return RT_ERR_STATE;
  }
  void* scratch = nullptr;
  e = static_scratch(&scratch);
  if (e != cudaSuccess) {
    *why = cudaGetErrorString(e);
    return RT_ERR_CUDA;
  }
  unsigned char* base = static_cast<unsigned char*>(scratch);
  const unsigned nb = (unsigned)((n + 1 + 255) / 256);
  uint32_t flags = 0;
  const uint32_t* err = &reinterpret_cast<ExecCtrl*>(base + kOffCtrl)->err_info;
  count_launch(2);
  k_static_clear_err<<<1, 1, 0, s>>>();
  k_static_check_rows<<<nb, 256, 0, s>>>(row_ptr, n, n_edges);
  e = cudaGetLastError();  // the flags word is trusted only if both kernels launched
  if (e == cudaSuccess) e = cudaMemcpyAsync(&flags, err, 4, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) {
    *why = cudaGetErrorString(e);
    return RT_ERR_CUDA;
  }
  if (flags) {
    *why = "row_ptr must start at 0, not decrease and end at n_edges";
    return RT_ERR_INVALID;
  }
  count_launch(2);
  k_static_check_cols<<<nb, 256, 0, s>>>(row_ptr, col, n);
  k_static_check_indeg<<<nb, 256, 0, s>>>(indeg, n);
  e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaMemcpyAsync(&flags, err, 4, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) {
    *why = cudaGetErrorString(e);
    return RT_ERR_CUDA;
  }
  if (flags & 2u) {
    *why = "every column must be a later task id below n_tasks";
    return RT_ERR_INVALID;
  }
  if (flags) {
    *why = "indeg does not match the column counts";
    return RT_ERR_INVALID;
  }
  count_launch(2);
  k_static_reset<<<256, 256, 0, s>>>(indeg, n, spin_iters, out);
  k_static_seed<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(indeg, n);
  launch_pack_adj(row_ptr, col, indeg, n, reinterpret_cast<int4*>(base + kOffAdj), nullptr, s);
  e = cudaGetLastError();
  if (e != cudaSuccess) {
    *why = cudaGetErrorString(e);
    return RT_ERR_CUDA;
  }
  ExecParams p{};
  p.adj = reinterpret_cast<const int4*>(base + kOffAdj);
  p.row_ptr = row_ptr;
  p.col = col;
  p.indeg = indeg;
  p.count = reinterpret_cast<int32_t*>(base + kOffCount);
  p.ring = reinterpret_cast<uint64_t*>(base + kOffRing);
  p.ring_cap = (uint32_t)n + 64u;
  p.n_graphs = 1;
  p.root_items = nullptr;  // one run: the roots are seeded above, never re-pushed
  p.graphs = reinterpret_cast<const ExecGraph*>(base + kOffTable);
  p.done_g = reinterpret_cast<uint32_t*>(base + kOffDone);
  p.ctrl = reinterpret_cast<ExecCtrl*>(base + kOffCtrl);
  p.replays = 1;
  p.graphs_target = 1;
  p.timeout_ns = timeout_ns;
  p.claim = 32;
  p.keep = 32;
  p.tickets = tickets;  // caller-owned int32[2n], or null
  p.total_roots = 0;
  p.need_fence = 0;
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  launch_exec(p, sms > 0 ? sms : 1, 2, s);
  uint32_t status = 0;
  e = cudaMemcpyAsync(&status, &p.ctrl->status, 4, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e == cudaSuccess) e = cudaGetLastError();
  if (e != cudaSuccess) {
    *why = cudaGetErrorString(e);
    return RT_ERR_CUDA;
  }
  if (status == (uint32_t)RT_ERR_TIMEOUT) {
    *why = "executor made no progress before the timeout";
    return RT_ERR_TIMEOUT;
  }
  if (status != 0u) {
    *why = "executor ring overflow";
    return RT_ERR_OOM;
  }
  return RT_OK;
}

void preload_static() {
  cudaFuncAttributes a;
  cudaFuncGetAttributes(&a, k_static_reset);
  cudaFuncGetAttributes(&a, k_static_seed);
  cudaFuncGetAttributes(&a, k_static_check_rows);
  cudaFuncGetAttributes(&a, k_static_check_cols);
  cudaFuncGetAttributes(&a, k_static_check_indeg);
  cudaFuncGetAttributes(&a, k_static_clear_err);
}

}  // namespace grt
