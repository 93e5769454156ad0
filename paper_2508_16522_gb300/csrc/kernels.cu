// kernels.cu -- tasks whose bodies are whole GPU kernels (the paper's
// optimisation for accelerators, Section 4.3).
//
// When a task launches accelerator work, the paper splits it into the host
// side that launches and an async node for the device work: an edge between
// two async nodes is enforced by the device itself (a kernel predicated on an
// event), so the host runs ahead; only edges into host-side work wait for a
// completion message. The alternative it improves on lifts device events into
// the runtime's own events and polls them from the host. rt_execute_kernels
// runs an analysed DAG with one kernel per task in three ways: lifted (the host
// launches a task when polling shows its predecessors' events have completed),
// async edges (every kernel enqueued up front on a pool of streams, predicated
// on its predecessors' events), and a CUDA graph of kernel nodes whose edges
// are the DAG's (instantiated once, then relaunched).
//
// The task kernel: one block of `threads` threads, each running `iters`
// dependent FMAs (the task's work); thread 0 then writes the task's depth, one
// more than the largest depth of its predecessors. The depths come out right
// only if every predecessor finished first, which the tests check.
#include "grt_internal.cuh"

namespace grt {

namespace {

__global__ void k_task(int32_t v, const int32_t* pred_off, const int32_t* pred, int32_t* depth, float* sink,
                       int32_t iters) {
  float x = (float)threadIdx.x;
  for (int32_t k = 0; k < iters; ++k) x = fmaf(x, 1.0000001f, 0.5f);
  if (threadIdx.x == 0) {
    int32_t d = 0;
    for (int32_t k = pred_off[v]; k < pred_off[v + 1]; ++k) {
      const int32_t pd = __ldcg(depth + pred[k]);
      d = pd > d ? pd : d;
    }
    __stcg(depth + v, d + 1);
  }
  if (x == -1.0f) sink[threadIdx.x] = x;  // keeps the loop; never true
}

}  // namespace

void* task_kernel_fn() { return reinterpret_cast<void*>(&k_task); }

void launch_task_kernel(int32_t v, const int32_t* pred_off, const int32_t* pred, int32_t* depth, float* sink,
                        int32_t iters, int threads, cudaStream_t s) {
  count_launch();
  k_task<<<1, threads, 0, s>>>(v, pred_off, pred, depth, sink, iters);
}

void preload_task_kernel() {
  cudaFuncAttributes a;
  cudaFuncGetAttributes(&a, k_task);
}

}  // namespace grt
