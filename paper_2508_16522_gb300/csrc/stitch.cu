// stitch.cu -- stitched replay: R replays of one trace in one persistent
// launch, joined by external conditions instead of a barrier.
//
// A compiled graph meets the rest of the program through external pre- and
// post-condition vertices (Section 4.1): a precondition holds back the tasks
// that depend on work outside the graph, a postcondition tells the outside
// that the tasks it follows are done. Section 5 uses them to join the graphs
// of a sharded trace. Consecutive replays of one trace are the simplest such
// program: replay r + 1 needs replay r only where its tasks touch data that
// replay r's tasks still use. rt_replay puts a barrier between replays (the
// next one starts when the last task of the previous one has run); here every
// replay is a copy of the compiled graph whose preconditions are the edges
// from the previous replay, so a task of replay r + 1 starts as soon as its
// own predecessors in replays r and r + 1 are done and replays overlap.
//
// The edges come from one analysis of the trace issued twice: edges inside
// the first copy are the graph's own (the same as the second copy's, which
// k_st_check verifies along with the rectangles), edges from the first copy to
// the second are the conditions. Under the per-cell run rule they leave
// replay r only for replay r + 1 and are the same for every r, so one
// trigger list per task serves every replay: a successor below n is in the
// same replay, a successor n + t is task t of the next one. Counter (replay r,
// task t) lives at count[r * n + t], so both kinds decrement count[r * n + c]
// for successor c; replay 0 starts at the in-copy in-degrees, the others at
// the full ones. Replays need not finish in order (a trace whose dependences
// are all explicit has no edges between replays), so every replay keeps its
// own counters.
//
// The executor is the compiled one's design (exec.cu): a persistent grid of
// warps, per-lane ring tickets, successors kept per warp, trigger records read
// speculatively beside each decrement; ready items carry (replay << 32 |
// task). Every wait is bounded by timeout_ns without progress.
#include "bodies.cuh"
#include "grt_internal.cuh"

namespace grt {

namespace {

constexpr unsigned kFullT = 0xffffffffu;
constexpr uint32_t kNoTk = 0xFFFFFFFFu;
constexpr int kStKeepMax = 64;
constexpr int kStRound = 4;  // 32-edge groups whose decrements are in flight together

// the second copy repeats the first: same rectangles, same in-copy edges
__global__ void k_st_check(const int32_t* req_off, const int64_t* lo, const int64_t* hi, const uint8_t* priv,
                           int D, const int32_t* row_ptr, const int32_t* col, int32_t n, uint32_t* err) {
  const int32_t v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= n) return;
  const int32_t a0 = req_off[v], a1 = req_off[v + 1], b0 = req_off[n + v], b1 = req_off[n + v + 1];
  bool bad = (a1 - a0) != (b1 - b0);
  for (int32_t k = 0; !bad && k < a1 - a0; ++k) {
    bad = priv[a0 + k] != priv[b0 + k];
    for (int d = 0; d < D && !bad; ++d) {
      const int64_t ia = (int64_t)(a0 + k) * D + d, ib = (int64_t)(b0 + k) * D + d;
      bad = lo[ia] != lo[ib] || hi[ia] != hi[ib];
    }
  }
  if (bad) {
    atomicOr(err, 1u);
    return;
  }
  // row v's targets below n, shifted by n, are row n + v (rows are sorted)
  const int32_t r0 = row_ptr[v], r1 = row_ptr[v + 1], s0 = row_ptr[n + v], s1 = row_ptr[n + v + 1];
  int32_t k = 0;
  for (; r0 + k < r1 && col[r0 + k] < n; ++k) {
    if (s0 + k >= s1 || col[s0 + k] != col[r0 + k] + n) {
      atomicOr(err, 2u);
      return;
    }
  }
  if (s0 + k != s1) atomicOr(err, 2u);
}

// counters of every (replay, task), the first ready items and the control
// block; the ring was cleared to kEmpty64 before this kernel
__global__ void k_st_init(StitchParams p, const int32_t* indeg, const uint64_t* root_items,
                          const uint32_t* rootpos) {
  const int64_t i0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const int64_t n = p.n;
  for (int64_t i = i0; i < p.total; i += stride) {
    const int64_t r = i / n, v = i - r * n;
    p.count[i] = r == 0 ? indeg[v] : indeg[n + v];
  }
  // roots of the two-copy graph: first copy's (no in-copy predecessor) come
  // first, then the second copy's (no predecessor at all)
  const int64_t a = rootpos[n], b = (int64_t)rootpos[2 * n] - a;
  for (int64_t k = i0; k < a; k += stride) p.ring[k] = (uint32_t)root_items[k];
  for (int64_t k = i0; k < (int64_t)(p.R - 1) * b; k += stride) {
    const int64_t r = 1 + k / b, j = k - (r - 1) * b;
    const uint32_t v = (uint32_t)root_items[a + j] - (uint32_t)n;
    p.ring[a + k] = ((uint64_t)r << 32) | v;
  }
  if (i0 == 0) {
    ExecCtrl* c = p.ctrl;
    c->head = 0;
    c->tail = (uint32_t)(a + (int64_t)(p.R - 1) * b);
    c->status = 0;
    c->executed = 0;
    c->ticket = 0;
  }
}

struct StWarp {
  int4 adj[kStKeepMax][2];   // trigger records of the kept ready items
  int4 bat[32][2];           // trigger records of the current batch
  uint64_t item[kStKeepMax];  // kept ready items
};

template <bool TICKETS, bool FENCE>
__global__ void __launch_bounds__(256, 1) k_stitch(StitchParams p) {
  extern __shared__ int4 st_smem[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  StWarp& q = reinterpret_cast<StWarp*>(st_smem)[warp];
  ExecCtrl* ctrl = p.ctrl;
  const unsigned lt = lanemask_lt();
  const uint32_t n = (uint32_t)p.n;
  int nl = 0;          // kept ready items (warp-uniform)
  uint32_t pend = 0;   // executed, not yet counted (warp-uniform)
  uint64_t idle_since = 0, last_check = 0;
  unsigned long long seen = 0;
  uint32_t backoff = 32;
  uint32_t my_t = kNoTk;  // this lane's claimed ring ticket

  for (;;) {
    uint64_t item = kEmpty64;
    int4 a0 = make_int4(0, 0, 0, -1), a1 = make_int4(-1, -1, -1, -1);
    bool have_rec = false;
    // 1. this lane's ticket, once published
    bool waiting = my_t != kNoTk;
    if (waiting && my_t < p.ring_cap) {
      const uint64_t vv = ld_acquire_u64(p.ring + my_t);
      if (vv != kEmpty64) {
        item = vv;
        my_t = kNoTk;
        waiting = false;
      }
    }
    // 2. lanes without an item take this warp's kept ones
    if (nl > 0) {
      const unsigned need = __ballot_sync(kFullT, item == kEmpty64);
      const int m = nl < __popc(need) ? nl : __popc(need);
      const int r = __popc(need & lt);
      if (item == kEmpty64 && r < m) {
        item = q.item[nl - m + r];
        a0 = q.adj[nl - m + r][0];
        a1 = q.adj[nl - m + r][1];
        have_rec = true;
      }
      nl -= m;
      __syncwarp();
    }
    if (!__any_sync(kFullT, item != kEmpty64)) {
      if (!__any_sync(kFullT, waiting)) {
        uint32_t h = 0;
        if (lane == 0) h = atomicAdd(&ctrl->head, (uint32_t)p.claim);
        h = __shfl_sync(kFullT, h, 0);
        if (lane < p.claim) my_t = h + (uint32_t)lane;
        continue;
      }
      if (pend) {
        if (FENCE) fence_acq_rel_gpu();
        if (lane == 0) atomicAdd(&ctrl->executed, (unsigned long long)pend);
        pend = 0;
        continue;
      }
      int stop = 0;
      if (lane == 0) {
        const unsigned long long ex = ld_relaxed_u64(&ctrl->executed);
        if (ld_relaxed_u32(&ctrl->status) != 0u || ex >= (unsigned long long)p.total) {
          stop = 1;
        } else {
          const uint64_t now = globaltimer_ns();
          if (idle_since == 0) {
            idle_since = last_check = now;
            seen = ex;
          } else if (now - last_check > 20000u) {
            last_check = now;
            if (ex != seen) {
              seen = ex;
              idle_since = now;
            } else if (now - idle_since > (uint64_t)p.timeout_ns) {
              atomicCAS(&ctrl->status, 0u, (uint32_t)RT_ERR_TIMEOUT);
              stop = 1;
            }
          }
        }
      }
      if (__shfl_sync(kFullT, stop, 0)) break;
      __nanosleep(backoff);
      if (backoff < 512) backoff <<= 1;
      continue;
    }
    backoff = 32;
    idle_since = 0;

    if (FENCE) fence_acq_rel_gpu();  // acquire: predecessors' effects before the bodies
    const bool has = item != kEmpty64;
    const uint32_t rep = (uint32_t)(item >> 32);
    const int v = (int)(uint32_t)item;
    if (has && !have_rec) {
      a0 = __ldg(p.adj + 2 * (int64_t)v);
      a1 = __ldg(p.adj + 2 * (int64_t)v + 1);
    }
    const int rbeg = has ? a0.x : 0;
    const int deg = has ? a0.y : 0;
    q.bat[lane][0] = a0;
    q.bat[lane][1] = a1;
    if (has) {
      const int64_t slot = (int64_t)rep * n + v;
      if (TICKETS) p.tickets[2 * slot] = (int32_t)atomicAdd(&ctrl->ticket, 1u);
      const ExecGraph& G = p.G;
      if (G.body == RT_BODY_SPIN) {
        G.out[slot] = (int32_t)spin_body((uint32_t)v, G.spin_iters);
      } else if (G.body == RT_BODY_FMA) {
        G.out[slot] = fma_body((uint32_t)v, G.spin_iters);
      } else if (FENCE) {
        if (G.body == RT_BODY_CHECK) {
          G.out[slot] = (int32_t)check_apply(G, v, (uint32_t)v);
        } else if (G.body == RT_BODY_COUNTER) {
          run_body<true>(G, v);
        }
      }
      if (TICKETS) p.tickets[2 * slot + 1] = (int32_t)atomicAdd(&ctrl->ticket, 1u);
    }
    if (FENCE || TICKETS) fence_acq_rel_gpu();  // release: bodies before the decrements
    __syncwarp();

    // COMPLETED_EDGE for the batch's out-edges; successor c of (rep, v) is
    // counter rep * n + c, in this replay (c < n) or the next (c >= n)
    int incl = deg;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(kFullT, incl, o);
      if (lane >= o) incl += y;
    }
    const int excl = incl - deg;
    const int D = __shfl_sync(kFullT, incl, 31);
    for (int e0 = 0; e0 < D; e0 += kStRound * 32) {
      int32_t tsk[kStRound];  // successor task, -1 if none
      uint32_t srep[kStRound];  // its replay
      int old[kStRound];
      int4 r0[kStRound], r1[kStRound];
#pragma unroll
      for (int k = 0; k < kStRound; ++k) {
        tsk[k] = -1;
        srep[k] = 0;
        if (e0 + k * 32 < D) {  // warp-uniform
          const int e = e0 + k * 32 + lane;
          int owner = 0;
#pragma unroll
          for (int step = 16; step >= 1; step >>= 1) {
            const int cand = owner + step;
            const int ex = __shfl_sync(kFullT, excl, cand);
            if (ex <= e) owner = cand;
          }
          const int orb = __shfl_sync(kFullT, rbeg, owner);
          const int oex = __shfl_sync(kFullT, excl, owner);
          const uint32_t orep = (uint32_t)(__shfl_sync(kFullT, item, owner) >> 32);
          if (e < D) {
            const int j = e - oex;
            const int c = j < kAdjInline ? reinterpret_cast<const int*>(&q.bat[owner][0])[3 + j] : p.col[orb + j];
            const bool next = (uint32_t)c >= n;
            srep[k] = orep + (next ? 1u : 0u);
            if (srep[k] < (uint32_t)p.R) tsk[k] = next ? c - (int)n : c;  // replay R's conditions are dropped
          }
        }
      }
#pragma unroll
      for (int k = 0; k < kStRound; ++k) {
        old[k] = 0;
        if (tsk[k] >= 0) {
          old[k] = atomicSub(&p.count[(int64_t)srep[k] * n + tsk[k]], 1);
          r0[k] = __ldg(p.adj + 2 * (int64_t)tsk[k]);
          r1[k] = __ldg(p.adj + 2 * (int64_t)tsk[k] + 1);
        }
      }
#pragma unroll
      for (int k = 0; k < kStRound; ++k) {
        if (e0 + k * 32 >= D) break;  // warp-uniform
        const bool ready = tsk[k] >= 0 && old[k] == 1;
        const unsigned rm = __ballot_sync(kFullT, ready);
        if (!rm) continue;
        const uint64_t nit = ((uint64_t)srep[k] << 32) | (uint32_t)tsk[k];
        const int rcount = __popc(rm);
        const int rank = __popc(rm & lt);
        int room = p.keep - nl;
        if (room < 0) room = 0;
        if (ready && rank < room) {
          q.item[nl + rank] = nit;
          q.adj[nl + rank][0] = r0[k];
          q.adj[nl + rank][1] = r1[k];
        }
        const int nover = rcount > room ? rcount - room : 0;
        if (nover > 0) {
          uint32_t base = 0;
          if (lane == 0) base = atomicAdd(&ctrl->tail, (uint32_t)nover);
          base = __shfl_sync(kFullT, base, 0);
          if ((uint64_t)base + (uint64_t)nover > (uint64_t)p.ring_cap) {
            if (lane == 0) atomicCAS(&ctrl->status, 0u, (uint32_t)RT_ERR_OOM);
          } else if (ready && rank >= room) {
            st_release_u64(p.ring + base + (rank - room), nit);
          }
        }
        nl += rcount < room ? rcount : room;
        __syncwarp();
      }
    }
    pend += (uint32_t)__popc(__ballot_sync(kFullT, has));
    if (pend >= 256u) {
      if (FENCE) fence_acq_rel_gpu();
      if (lane == 0) atomicAdd(&ctrl->executed, (unsigned long long)pend);
      pend = 0;
    }
  }
}

// at most 8 warps of 3.5 KB: under the 48 KB of dynamic shared memory a
// launch gets without opting in
template <bool TICKETS, bool FENCE>
void launch_one(const StitchParams& p, int blocks, int warps, cudaStream_t s) {
  k_stitch<TICKETS, FENCE><<<blocks, warps * 32, (size_t)warps * sizeof(StWarp), s>>>(p);
}

}  // namespace

void launch_stitch_check(const int32_t* req_off, const int64_t* lo, const int64_t* hi, const uint8_t* priv, int D,
                         const int32_t* row_ptr, const int32_t* col, int32_t n, uint32_t* err, cudaStream_t s) {
  if (n <= 0) return;
  count_launch();
  k_st_check<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(req_off, lo, hi, priv, D, row_ptr, col, n, err);
}

void launch_stitch(const StitchParams& p, const int32_t* indeg, const uint64_t* root_items, const uint32_t* rootpos,
                   int blocks, int warps, bool tickets, bool fence, cudaStream_t s) {
  count_launch(2);
  k_st_init<<<1024, 256, 0, s>>>(p, indeg, root_items, rootpos);
  if (tickets) {
    if (fence) launch_one<true, true>(p, blocks, warps, s);
    else launch_one<true, false>(p, blocks, warps, s);
  } else {
    if (fence) launch_one<false, true>(p, blocks, warps, s);
    else launch_one<false, false>(p, blocks, warps, s);
  }
}

void preload_stitch() {
  cudaFuncAttributes a;
  cudaFuncGetAttributes(&a, k_st_check);
  cudaFuncGetAttributes(&a, k_st_init);
  cudaFuncGetAttributes(&a, k_stitch<false, false>);
  cudaFuncGetAttributes(&a, k_stitch<false, true>);
  cudaFuncGetAttributes(&a, k_stitch<true, false>);
  cudaFuncGetAttributes(&a, k_stitch<true, true>);
}

}  // namespace grt
