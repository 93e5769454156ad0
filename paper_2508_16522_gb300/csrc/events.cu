// events.cu -- the standard, event-based executor, for comparison with the
// compiled one (exec.cu).
//
// The paper models today's task runtimes as a scheduler that builds the DAG
// dynamically as tasks are launched (its Fig. task-to-rt-actor reduction):
// every launch makes a fresh completion event and registers the task as
// pending on the events of its preconditions; a finished task triggers its
// event, which notifies the tasks waiting on it; a task whose events have all
// triggered becomes ready. Compiling the graph (Section 4.2) replaces this
// generic machinery by per-task countdowns and precomputed trigger lists.
//
// This kernel is that standard runtime on the GPU, run on the same DAG as the
// compiled executor: each run starts with fresh events and rebuilds the
// waiter lists. Warps first register the launches in program order, 32 at a
// time: for each precondition the task either finds the event triggered
// already or pushes a waiter node onto the event's list (an atomic push that
// fails once the event has triggered). A task's pending count starts at 1 (a
// guard released when its registration ends), so it cannot fire before it is
// fully registered. Then warps take ready tasks from a ring (each lane claims
// one of the warp's `claim` tickets and waits for its slot), run the body,
// trigger the event (an atomic exchange that returns the waiter list) and
// walk the list, decrementing each waiter's pending count. Per edge that is
// a node allocation, a pending increment, a list push and a pending decrement
// reached through a dependent walk, where the compiled executor does one
// decrement. Every wait is bounded: a run without progress for timeout_ns ends
// with RT_ERR_TIMEOUT.
#include "bodies.cuh"
#include "grt_internal.cuh"

namespace grt {

namespace {

constexpr uint32_t kNil = 0xFFFFFFFFu;   // an event nobody waits on yet
constexpr uint32_t kTrig = 0xFFFFFFFEu;  // a triggered event
constexpr uint32_t kFree = 0xFFFFFFFFu;  // an unfilled ring slot
constexpr uint32_t kNoTk = 0xFFFFFFFFu;

__device__ __forceinline__ uint32_t ld_acquire_u32_gpu(const uint32_t* p) {
  uint32_t v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release_u32_gpu(uint32_t* p, uint32_t v) {
  asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// in-edges from the CSR by source: pred[pred_off[d] + k] are d's predecessors
__global__ void k_ev_transpose(const int32_t* row_ptr, const int32_t* col, int32_t n, const int32_t* pred_off,
                               int32_t* cursor, int32_t* pred) {
  const int32_t v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= n) return;
  for (int32_t e = row_ptr[v]; e < row_ptr[v + 1]; ++e) {
    const int32_t d = col[e];
    pred[pred_off[d] + atomicAdd(&cursor[d], 1)] = v;
  }
}

// fresh events and an empty ring for a run
__global__ void k_ev_reset(uint32_t* head, int32_t n, uint32_t* ring, uint32_t ring_cap) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t k = i; k < n; k += stride) head[k] = kNil;
  for (int64_t k = i; k < ring_cap; k += stride) ring[k] = kFree;
}

__device__ __forceinline__ void ev_push(const EvParams& p, uint32_t t) {
  const uint32_t slot = atomicAdd(&p.ctrl->rtail, 1u);
  if (slot < p.ring_cap) {
    st_release_u32_gpu(p.ring + slot, t);
  } else {
    atomicCAS(&p.ctrl->status, 0u, (uint32_t)RT_ERR_OOM);
  }
}

// LAUNCH: register task t as pending on its preconditions' events
__device__ void ev_register(const EvParams& p, int t) {
  p.pending[t] = 1;  // the guard: released below
  __threadfence();
  for (int32_t k = p.pred_off[t]; k < p.pred_off[t + 1]; ++k) {
    const int32_t e = p.pred[k];
    uint32_t h = __ldcg(p.head + e);
    if (h == kTrig) continue;  // triggered already: nothing to wait for
    atomicAdd(&p.pending[t], 1);
    const uint32_t node = atomicAdd(&p.ctrl->pool, 1u);
    p.node_task[node] = (uint32_t)t;
    for (;;) {
      if (h == kTrig) {  // triggered meanwhile: undo (the guard keeps the count positive)
        atomicSub(&p.pending[t], 1);
        break;
      }
      p.node_next[node] = h;
      __threadfence();  // the node before its publication
      const uint32_t old = atomicCAS(p.head + e, h, node);
      if (old == h) break;
      h = old;
    }
  }
  if (atomicSub(&p.pending[t], 1) == 1) ev_push(p, (uint32_t)t);
}

__global__ void __launch_bounds__(256) k_events(EvParams p) {
  const int lane = threadIdx.x & 31;
  uint32_t my = kNoTk;  // this lane's claimed ring ticket
  uint64_t idle_since = 0;
  uint32_t seen = 0, backoff = 32;
  for (;;) {
    // 1. launches still to register, in program order, 32 per claim
    uint32_t c = kNoTk;
    if (lane == 0 && ld_relaxed_u32(&p.ctrl->reg) < (uint32_t)p.n) c = atomicAdd(&p.ctrl->reg, 32u);
    c = __shfl_sync(0xffffffffu, c, 0);
    if (c < (uint32_t)p.n) {
      const int t = (int)c + lane;
      if (t < p.n) ev_register(p, t);
      continue;
    }
    // 2. EXEC: this lane's ticket, once published
    uint32_t item = kFree;
    if (my != kNoTk && my < p.ring_cap) {
      const uint32_t v = ld_acquire_u32_gpu(p.ring + my);
      if (v != kFree) {
        item = v;
        my = kNoTk;
      }
    }
    if (!__any_sync(0xffffffffu, item != kFree)) {
      if (!__any_sync(0xffffffffu, my != kNoTk)) {
        uint32_t h = 0;
        if (lane == 0) h = atomicAdd(&p.ctrl->rhead, (uint32_t)p.claim);
        h = __shfl_sync(0xffffffffu, h, 0);
        if (lane < p.claim) my = h + (uint32_t)lane;
        continue;
      }
      int stop = 0;
      if (lane == 0) {
        const uint32_t d = ld_relaxed_u32(&p.ctrl->done);
        if (d >= (uint32_t)p.n || ld_relaxed_u32(&p.ctrl->status) != 0u) {
          stop = 1;
        } else {
          const uint64_t now = globaltimer_ns();
          if (idle_since == 0 || d != seen) {
            idle_since = now;
            seen = d;
          } else if (now - idle_since > (uint64_t)p.timeout_ns) {
            atomicCAS(&p.ctrl->status, 0u, (uint32_t)RT_ERR_TIMEOUT);
            stop = 1;
          }
        }
      }
      if (__shfl_sync(0xffffffffu, stop, 0)) break;
      __nanosleep(backoff);
      if (backoff < 512) backoff <<= 1;
      continue;
    }
    backoff = 32;
    idle_since = 0;
    if (item != kFree) {
      fence_acq_rel_gpu();  // the predecessors' effects before the body
      if (p.G.body == RT_BODY_SPIN) {
        p.G.out[item] = (int32_t)spin_body(item, p.G.spin_iters);
      } else {
        run_body<true>(p.G, (int)item);
      }
      fence_acq_rel_gpu();  // the body's effects before the trigger
      // TASK_DONE: trigger the event and notify its waiters
      uint32_t x = atomicExch(p.head + item, kTrig);
      __threadfence();  // the nodes published before the exchange
      while (x != kNil && x != kTrig) {
        const uint32_t w = __ldcg(p.node_task + x);
        const uint32_t nx = __ldcg(p.node_next + x);
        if (atomicSub(&p.pending[w], 1) == 1) ev_push(p, w);
        x = nx;
      }
    }
    const unsigned ran = __ballot_sync(0xffffffffu, item != kFree);
    if (lane == 0) atomicAdd(&p.ctrl->done, (uint32_t)__popc(ran));
  }
}

}  // namespace

void launch_ev_transpose(const int32_t* row_ptr, const int32_t* col, int32_t n, const int32_t* pred_off,
                         int32_t* cursor, int32_t* pred, cudaStream_t s) {
  if (n > 0) {
    count_launch();
    k_ev_transpose<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(row_ptr, col, n, pred_off, cursor, pred);
  }
}

void launch_events(const EvParams& p, int blocks, cudaStream_t s) {
  count_launch(2);
  k_ev_reset<<<1024, 256, 0, s>>>(p.head, p.n, p.ring, p.ring_cap);
  k_events<<<blocks, 256, 0, s>>>(p);
}

void preload_events() {
  cudaFuncAttributes a;
  cudaFuncGetAttributes(&a, k_ev_transpose);
  cudaFuncGetAttributes(&a, k_ev_reset);
  cudaFuncGetAttributes(&a, k_events);
}

}  // namespace grt
