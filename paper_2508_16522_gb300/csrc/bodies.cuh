// bodies.cuh -- the task bodies, shared by the compiled executor (exec.cu),
// the event-based one (events.cu), the serving kernel (serve.cu) and stitched
// replay (stitch.cu).
#pragma once
#include "grt_internal.cuh"

namespace grt {
namespace {

// The SPIN body: `iters` steps of the 32-bit LCG x <- a x + c (a = 1664525,
// c = 1013904223) from x = the task's id: a chain of `iters` dependent integer
// multiply-adds. Each step is one hand-written mad.lo.u32, so that the
// compiler cannot fold the recurrence (it would in some kernels and not in
// others): the body costs the same `iters` dependent operations in every
// executor, which is what its granularity stands for.
__device__ __forceinline__ uint32_t spin_body(uint32_t x, int iters) {
  for (int k = 0; k < iters; ++k) asm volatile("mad.lo.u32 %0, %0, 1664525, 1013904223;" : "+r"(x));
  return x;
}

// The FMA body: `iters` dependent single-precision fused multiply-adds
// x <- x * 0.999f + 0.25f from x = the task's id (rounded to float), each one
// hand-written fma.rn.f32 (IEEE, round to nearest even): the floating-point
// loop of a compute-bound Task Bench kernel, on one lane. Its result's bits go
// to out[task].
__device__ __forceinline__ int32_t fma_body(uint32_t task, int iters) {
  float x = (float)task;
  for (int k = 0; k < iters; ++k) asm volatile("fma.rn.f32 %0, %0, %1, %2;" : "+f"(x) : "f"(0.999f), "f"(0.25f));
  return __float_as_int(x);
}

__device__ __forceinline__ uint32_t cell_index(const ExecGraph& G, int64_t x, int64_t y) {
  return (uint32_t)((y - G.dom_lo[1]) * G.ext[0] + (x - G.dom_lo[0]));
}

// CHECK body (order-sensitive): see grt.h. Lane-serial; meant for test sizes.
// Applies task j's accesses to the state and returns its output word; `id` is
// the task id the body mixes in (j itself, or j's id within its own request).
__device__ uint32_t check_apply(const ExecGraph& G, int j, uint32_t id) {
  const int r0 = G.req_off[j], r1 = G.req_off[j + 1];
  const int D = G.ndim;
  uint32_t acc = 0;
  for (int pass = 0; pass < 2; ++pass) {
    uint32_t sum = 0;
    for (int e = r0; e < r1; ++e) {
      const int64_t x0 = G.lo[(int64_t)e * D], x1 = G.hi[(int64_t)e * D];
      const int64_t y0 = D == 2 ? G.lo[(int64_t)e * 2 + 1] : G.dom_lo[1];
      const int64_t y1 = D == 2 ? G.hi[(int64_t)e * 2 + 1] : G.dom_lo[1];
      for (int64_t y = y0; y <= y1; ++y) {
        for (int64_t x = x0; x <= x1; ++x) {
          bool seen = false;
          for (int f = r0; f < e && !seen; ++f) {
            const int64_t fx0 = G.lo[(int64_t)f * D], fx1 = G.hi[(int64_t)f * D];
            const int64_t fy0 = D == 2 ? G.lo[(int64_t)f * 2 + 1] : y, fy1 = D == 2 ? G.hi[(int64_t)f * 2 + 1] : y;
            seen = fx0 <= x && x <= fx1 && fy0 <= y && y <= fy1;
          }
          if (seen) continue;  // the first rectangle covering the cell handles it
          uint32_t comb = G.priv[e];
          for (int f = e + 1; f < r1; ++f) {
            const int64_t fx0 = G.lo[(int64_t)f * D], fx1 = G.hi[(int64_t)f * D];
            const int64_t fy0 = D == 2 ? G.lo[(int64_t)f * 2 + 1] : y, fy1 = D == 2 ? G.hi[(int64_t)f * 2 + 1] : y;
            if (fx0 <= x && x <= fx1 && fy0 <= y && y <= fy1) comb = combine_priv(comb, G.priv[f]);
          }
          const uint32_t c = cell_index(G, x, y);
          if (pass == 0) {
            if (comb == (uint32_t)kKindRead) sum += (uint32_t)__ldcg(G.state + c);
          } else if (comb == (uint32_t)kKindWrite) {
            __stcg(G.state + c, (int32_t)mix32(acc, c));
          } else if (comb == (uint32_t)kKindReduce) {
            atomicAdd(reinterpret_cast<unsigned*>(G.state) + c, mix32(id, c));
          }
        }
      }
    }
    if (pass == 0) acc = mix32(id, sum);
  }
  return acc;
}

__device__ __forceinline__ void check_body(const ExecGraph& G, int j) { G.out[j] = (int32_t)check_apply(G, j, (uint32_t)j); }

// FENCE = false: the launch only has bodies that read nothing written by
// other tasks (EMPTY, SPIN, FMA), so the order-sensitive bodies are compiled out.
template <bool FENCE>
__device__ __forceinline__ void run_body(const ExecGraph& G, int j) {
  if (!FENCE) {
    if (G.body == RT_BODY_SPIN) {
      G.out[j] = (int32_t)spin_body((uint32_t)j, G.spin_iters);
    } else if (G.body == RT_BODY_FMA) {
      G.out[j] = fma_body((uint32_t)j, G.spin_iters);
    }
    return;
  }
  switch (G.body) {
    case RT_BODY_SPIN: {
      G.out[j] = (int32_t)spin_body((uint32_t)j, G.spin_iters);
      break;
    }
    case RT_BODY_FMA:
      G.out[j] = fma_body((uint32_t)j, G.spin_iters);
      break;
    case RT_BODY_COUNTER: {
      const int k = G.body_arg[j];
      const int32_t v = __ldcg(G.state + k);
      __stcg(G.state + k, (int32_t)((uint32_t)v + 1u));
      break;
    }
    case RT_BODY_CHECK:
      check_body(G, j);
      break;
    default:
      break;
  }
}

}  // namespace
}  // namespace grt
