// microbench.cu -- the atomic and latency rooflines the executor is held to.
//
// The executor's work is one atomic decrement per edge and its critical path
// is a chain of dependent decrements (one per wavefront step), so its
// rooflines are not HBM bandwidth but:
//   [0] dependent atomic latency: one thread, each atomicAdd's address taken
//       from the previous one's result (ns per operation)
//   [1] dependent L2 load latency: pointer chasing through an L2-resident
//       array (ns per load)
//   [2] distinct-address atomicSub throughput, result used (G ops/s): every
//       thread decrements scattered counters of a 64 MB array, as the executor
//       does
//   [3] the same without using the result (fire-and-forget reductions)
//   [4] contended atomicAdd on one address by every thread (G ops/s)
//   [5] the same, warp-aggregated (one atomic per warp; G thread-ops/s)
//   [6] the FMA task body alone: ns per dependent iteration on one warp (one
//       task per lane), the body's peak rate that Task Bench's efficiency is
//       measured against
#include "bodies.cuh"
#include "grt_internal.cuh"

namespace grt {

namespace {

constexpr int64_t kMbWords = 16 << 20;  // 64 MB of uint32 counters (fits the 129 MB L2)

__global__ void k_mb_init(uint32_t* a, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    a[i] = (uint32_t)((i * 2654435761ull + 12345ull) & (uint64_t)(n - 1));  // a permutation-ish chase
}

__global__ void k_mb_dep_atomic(uint32_t* a, int64_t n, int ops, uint32_t* sink) {
  uint32_t idx = 7;
  for (int k = 0; k < ops; ++k) idx = (atomicAdd(&a[idx], 0u) + (uint32_t)k) & (uint32_t)(n - 1);
  *sink = idx;
}

__global__ void k_mb_dep_load(const uint32_t* a, int64_t n, int ops, uint32_t* sink) {
  uint32_t idx = 7;
  for (int k = 0; k < ops; ++k) idx = (__ldcg(a + idx) + (uint32_t)k) & (uint32_t)(n - 1);
  *sink = idx;
}

template <bool USE>
__global__ void k_mb_distinct(uint32_t* a, int64_t n, int iters, uint32_t* sink) {
  const uint64_t t = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  uint32_t acc = 0;
  for (int k = 0; k < iters; ++k) {
    const uint32_t idx = (uint32_t)(((t * 64 + (uint64_t)k) * 2654435761ull) & (uint64_t)(n - 1));
    if (USE) {
      acc += atomicSub(&a[idx], 1u) == 1u;
    } else {
      atomicSub(&a[idx], 1u);
    }
  }
  if (USE && acc == 0xFFFFFFFFu) *sink = acc;
}

__global__ void k_mb_fma(int iters, int32_t* sink) {
  const int32_t x = fma_body(threadIdx.x, iters);
  if (x == 0x7fffffff) *sink = x;  // keeps the chain live
}

template <bool AGG>
__global__ void k_mb_contended(uint32_t* a, int iters) {
  for (int k = 0; k < iters; ++k) {
    if (AGG) {
      if ((threadIdx.x & 31) == 0) atomicAdd(a, 32u);
    } else {
      atomicAdd(a, 1u);
    }
  }
}

}  // namespace

rt_status microbench(double* out, int n_out, cudaStream_t s, const char** why) {
  uint32_t* a = nullptr;
  uint32_t* sink = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t e = cudaMalloc(&a, kMbWords * 4);
  if (e == cudaSuccess) e = cudaMalloc(&sink, 256);
  if (e == cudaSuccess) e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  int dev = 0, sms = 0;
  if (e == cudaSuccess) e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  double r[7] = {0, 0, 0, 0, 0, 0, 0};
  auto timed = [&](auto launch) -> double {
    launch();  // warm-up
    cudaEventRecord(e0, s);
    launch();
    cudaEventRecord(e1, s);
    cudaEventSynchronize(e1);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    return (double)ms;
  };
  if (e == cudaSuccess) {
    count_launch(1);
    k_mb_init<<<sms * 8, 256, 0, s>>>(a, kMbWords);
    const int dep_ops = 20000;
    count_launch(2);
    r[0] = timed([&] { k_mb_dep_atomic<<<1, 1, 0, s>>>(a, kMbWords, dep_ops, sink); }) * 1e6 / dep_ops;
    count_launch(2);
    r[1] = timed([&] { k_mb_dep_load<<<1, 1, 0, s>>>(a, kMbWords, dep_ops, sink); }) * 1e6 / dep_ops;
    const int blocks = sms * 8, threads = 256, iters = 64;
    const double total = (double)blocks * threads * iters;
    count_launch(6);
    r[2] = total / (timed([&] { k_mb_distinct<true><<<blocks, threads, 0, s>>>(a, kMbWords, iters, sink); }) * 1e6);
    r[3] = total / (timed([&] { k_mb_distinct<false><<<blocks, threads, 0, s>>>(a, kMbWords, iters, sink); }) * 1e6);
    r[4] = total / (timed([&] { k_mb_contended<false><<<blocks, threads, 0, s>>>(sink, iters); }) * 1e6);
    r[5] = total / (timed([&] { k_mb_contended<true><<<blocks, threads, 0, s>>>(sink, iters); }) * 1e6);
    const int fma_iters = 1 << 20;
    count_launch(2);
    r[6] = timed([&] { k_mb_fma<<<1, 32, 0, s>>>(fma_iters, reinterpret_cast<int32_t*>(sink)); }) * 1e6 / fma_iters;
    e = cudaGetLastError();
  }
  if (a) cudaFree(a);
  if (sink) cudaFree(sink);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (e != cudaSuccess) {
    *why = cudaGetErrorString(e);
    return RT_ERR_CUDA;
  }
  for (int k = 0; k < n_out && k < 7; ++k) out[k] = r[k];
  return RT_OK;
}

void preload_microbench() {
  cudaFuncAttributes a;
  cudaFuncGetAttributes(&a, k_mb_init);
  cudaFuncGetAttributes(&a, k_mb_dep_atomic);
  cudaFuncGetAttributes(&a, k_mb_dep_load);
  cudaFuncGetAttributes(&a, k_mb_distinct<true>);
  cudaFuncGetAttributes(&a, k_mb_distinct<false>);
  cudaFuncGetAttributes(&a, k_mb_fma);
  cudaFuncGetAttributes(&a, k_mb_contended<true>);
  cudaFuncGetAttributes(&a, k_mb_contended<false>);
}

}  // namespace grt
