// exec.cu -- persistent actor-style executor of compiled task graphs.
//
// Section 4.2 / Algorithm 1 on one GPU. Each task has a countdown of pending
// incoming edges and its CSR row of out-edges (the trigger list). A persistent
// grid of warps plays the workers:
//  * INIT: every task without incoming edges is seeded into a global ready
//    ring (k_seed);
//  * EXECUTE_OP: a warp takes up to 32 ready tasks (its own kept successors
//    first, else a claim of published ring slots), re-arms each task's own
//    counter for the next run, runs the bodies in place, then walks the
//    batch's out-edges warp-cooperatively;
//  * COMPLETED_EDGE: one atomic decrement per edge; the decrement that finds
//    1 makes the successor ready. The warp keeps up to `keep` of them for its
//    next batch and publishes the rest to the ring (reserve by one atomic on
//    the tail, publish by store-release per slot).
// Replays: a per-graph completion counter; the warp whose increment completes
// graph g's run r seeds g's roots again for run r+1 (graphs in a batch advance
// independently), until `replays` runs are done. A single graph's counters
// count down and each task re-arms its own; a batch's counters start at 0 and
// count up across the replays, a task being ready in run r when its counter
// reaches (r + 1) times its in-degree (each ready item carries its run, so the
// test is one multiply). Run r+1's increments of a counter cannot
// overtake run r's (the task ran in run r only after all of them), so a batch
// needs no re-arm and no release of it before the completion count.
// Every wait is bounded: a warp that sees no progress of the global executed
// counter for timeout_ns sets status TIMEOUT and returns.
#include <algorithm>
#include <mutex>
#include <vector>

#include "bodies.cuh"
#include "grt_internal.cuh"

namespace grt {

namespace {
constexpr int kKeepMax = 64;
constexpr uint32_t kNoTicket = 0xFFFFFFFFu;
constexpr int kEdgeRound = 4;  // 32-edge groups whose decrements are in flight together
// a batch's ready item: run << 52 | graph << 32 | task (graphs < 2^20, runs < 2^12)
constexpr uint64_t kGraphMask = 0xFFFFFull;
constexpr unsigned kFull = 0xffffffffu;

__global__ void k_reset_counts(int32_t* count, const int32_t* indeg, int64_t n, int32_t hold_task,
                               int32_t hold_extra) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) count[i] = indeg[i] + (i == hold_task ? hold_extra : 0);
}

__global__ void k_seed(ExecParams p, int64_t ring_clear) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t k = i; k < ring_clear; k += stride) p.ring[k] = kEmpty64;
  for (int64_t k = i; k < p.total_roots; k += stride) p.ring[k] = p.root_items[k];
  for (int64_t k = i; k < p.n_graphs; k += stride) p.done_g[k] = 0;
  if (i == 0) {
    ExecCtrl* c = p.ctrl;
    c->head = 0;
    c->tail = (uint32_t)p.total_roots;
    c->graphs_done = 0;
    c->status = 0;
    c->executed = 0;
    c->ticket = 0;
    c->err_where = 0;
    c->err_info = 0;
    for (int k = 0; k < kCntCount; ++k) c->counters[k] = 0;
  }
}


// pushes graph g's roots into the ring for its next run (warp-cooperative)
__device__ void push_roots(const ExecParams& p, int g, int lane, uint64_t tag) {
  const ExecGraph& G = p.graphs[g];
  uint32_t base = 0;
  if (lane == 0) base = atomicAdd(&p.ctrl->tail, (uint32_t)G.n_roots);
  base = __shfl_sync(kFull, base, 0);
  if ((uint64_t)base + (uint64_t)G.n_roots > (uint64_t)p.ring_cap) {
    if (lane == 0) atomicCAS(&p.ctrl->status, 0u, (uint32_t)RT_ERR_OOM);
    return;
  }
  for (int k = lane; k < G.n_roots; k += 32) st_release_u64(p.ring + base + k, p.root_items[G.root_base + k] | tag);
}

// the warp whose count completed a run of graph g: next run or graph finished
// (tag: the bits a batch's items carry for the run they belong to)
__device__ void on_run_complete(const ExecParams& p, int g, uint32_t runs_done, int lane, uint64_t tag) {
  fence_acq_rel_gpu();  // acquire every re-armed counter of the finished run
  if ((int)runs_done < p.replays)
    push_roots(p, g, lane, tag);
  else if (lane == 0)
    atomicAdd(&p.ctrl->graphs_done, 1u);
}

// per-warp shared memory of the executor
struct WarpQ {
  int4 adj[kKeepMax][2];  // trigger records of the kept ready tasks
  int4 bat[32][2];        // trigger records of the current batch, one per lane
  uint64_t item[kKeepMax];  // kept ready tasks (task | graph << 32; a batch's also run << 52)
};

template <bool TICKETS, bool FENCE, bool SINGLE>
__global__ void __launch_bounds__(256, 1) k_exec(ExecParams p) {
  extern __shared__ int4 exec_smem[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  WarpQ& q = reinterpret_cast<WarpQ*>(exec_smem)[warp];
  ExecCtrl* ctrl = p.ctrl;
  const unsigned lt = lanemask_lt();
  const uint32_t n0 = SINGLE ? (uint32_t)p.graphs[0].n_tasks : 0u;
  const int body0 = SINGLE ? p.graphs[0].body : 0;
  const int spin0 = SINGLE ? p.graphs[0].spin_iters : 0;
  int32_t* const out0 = SINGLE ? p.graphs[0].out : nullptr;  // task_base is 0 for a single graph
  int nl = 0;                    // kept ready tasks (warp-uniform)
  uint32_t pend = 0;             // executed but not yet counted (warp-uniform)
  uint64_t idle_since = 0, last_check = 0, last_status = 0;  // lane 0
  unsigned long long seen = 0;
  uint32_t backoff = 32;
  uint32_t my_t = kNoTicket;     // this lane's claimed ring ticket
  uint32_t cnt[kCntCount];  // diagnostics, per warp (lane 0's copy is added to the totals at exit)
#pragma unroll
  for (int k = 0; k < kCntCount; ++k) cnt[k] = 0;

  // adds this warp's executed tasks to the shared counters (convergent)
  auto flush = [&]() {
    if (pend == 0) return;
    fence_acq_rel_gpu();  // release: bodies and re-armed counters before the count
    if (SINGLE) {
      uint32_t now = 0;
      if (lane == 0) now = atomicAdd(&p.done_g[0], pend) + pend;
      now = __shfl_sync(kFull, now, 0);
      if (now % n0 == 0u) on_run_complete(p, 0, now / n0, lane, 0ull);
    } else if (lane == 0) {
      atomicAdd(&ctrl->executed, (unsigned long long)pend);
    }
    pend = 0;
  };

  for (;;) {
    uint64_t item = kEmpty64;
    int4 a0 = make_int4(0, 0, 0, -1), a1 = make_int4(-1, -1, -1, -1);  // trigger record
    bool have_rec = false;
    // 1. this lane's claimed ring ticket, if it has been published
    bool waiting = my_t != kNoTicket;
    if (waiting) {
      if (my_t >= p.ring_cap) {
        // past the ring: never filled; dropped when the run ends
      } else {
        const uint64_t vv = ld_acquire_u64(p.ring + my_t);
        if (vv != kEmpty64) {
          item = vv;
          st_relaxed_u64(p.ring + my_t, kEmpty64);  // leave the ring clean for the next launch
          my_t = kNoTicket;
          waiting = false;
        }
      }
    }
    // 2. lanes without an item take this warp's kept ready tasks
    if (nl > 0) {
      const unsigned need = __ballot_sync(kFull, item == kEmpty64);
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
    if (!__any_sync(kFull, item != kEmpty64)) {
      if (!__any_sync(kFull, waiting)) {
        // 3. claim the next `claim` tickets: one atomic, never fails; each
        // lane then watches its own slot, so no shared word is polled
        uint32_t h = 0;
        if (lane == 0) {
          h = atomicAdd(&ctrl->head, (uint32_t)p.claim);
          ++cnt[kCntClaims];
        }
        h = __shfl_sync(kFull, h, 0);
        if (lane < p.claim) my_t = h + (uint32_t)lane;
        continue;
      }
      if (pend) {
        flush();  // may seed the next run: look for work again first
        continue;
      }
      ++cnt[kCntIdle];
      int stop = 0;
      if (lane == 0) {
        // the shared status words, read at most every microsecond per idle
        // warp (all of them reading at every pass would pile onto one L2 line)
        const uint64_t now = globaltimer_ns();
        uint32_t st = 0u, gd = 0u;
        if (now - last_status >= 1000u) {
          last_status = now;
          st = ld_relaxed_u32(&ctrl->status);
          gd = ld_relaxed_u32(&ctrl->graphs_done);
        }
        if (st != 0u || (int)gd >= p.graphs_target) {
          stop = 1;
        } else {
          if (idle_since == 0) {
            idle_since = last_check = now;
            seen = SINGLE ? ld_relaxed_u32(&p.done_g[0]) : ld_relaxed_u64(&ctrl->executed);
          } else if (now - last_check > 20000u) {
            last_check = now;
            const unsigned long long pr = SINGLE ? ld_relaxed_u32(&p.done_g[0]) : ld_relaxed_u64(&ctrl->executed);
            if (pr != seen) {
              seen = pr;
              idle_since = now;
            } else if (now - idle_since > (uint64_t)p.timeout_ns) {
              atomicCAS(&ctrl->status, 0u, (uint32_t)RT_ERR_TIMEOUT);
              stop = 1;
            }
          }
        }
      }
      if (__shfl_sync(kFull, stop, 0)) break;
      __nanosleep(backoff);
      if (backoff < 512) backoff <<= 1;
      continue;
    }
    backoff = 32;
    idle_since = 0;

    if (FENCE) fence_acq_rel_gpu();  // acquire: predecessors' effects visible to the bodies
    const bool has = item != kEmpty64;
    const int v = (int)(uint32_t)item;
    const int g = SINGLE ? 0 : (has ? (int)((item >> 32) & kGraphMask) : -1);
    if (has && !have_rec) {
      a0 = __ldg(p.adj + 2 * (int64_t)v);
      a1 = __ldg(p.adj + 2 * (int64_t)v + 1);
    }
    const int rbeg = has ? a0.x : 0;
    const int deg = has ? a0.y : 0;
    q.bat[lane][0] = a0;
    q.bat[lane][1] = a1;
    if (has) {
      if (SINGLE) p.count[v] = a0.z;  // INIT's reset, done by the task itself for the next run
      if (TICKETS) p.tickets[2 * (int64_t)v] = (int32_t)atomicAdd(&ctrl->ticket, 1u);
      if (SINGLE && !FENCE) {
        if (body0 == RT_BODY_SPIN) {  // the one graph's fields live in registers
          out0[v] = (int32_t)spin_body((uint32_t)v, spin0);
        } else if (body0 == RT_BODY_FMA) {
          out0[v] = fma_body((uint32_t)v, spin0);
        }
      } else {
        const ExecGraph& G = p.graphs[g];
        run_body<FENCE>(G, v - G.task_base);
      }
      if (TICKETS) p.tickets[2 * (int64_t)v + 1] = (int32_t)atomicAdd(&ctrl->ticket, 1u);
    }
    if (FENCE || TICKETS) fence_acq_rel_gpu();  // release: bodies before the decrements
    __syncwarp();

    // COMPLETED_EDGE for every out-edge of the batch, kEdgeRound x 32 edges per
    // round. The first kAdjInline successors of a task come from its trigger
    // record (no load); all decrements of a round are in flight together, and
    // each successor's own record is read speculatively with its decrement, so
    // a successor kept by this warp starts its next batch with no dependent
    // load: about one memory round trip per wavefront step.
    int incl = deg;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(kFull, incl, o);
      if (lane >= o) incl += y;
    }
    const int excl = incl - deg;
    const int D = __shfl_sync(kFull, incl, 31);
    cnt[kCntEdges] += (unsigned)D;
    for (int e0 = 0; e0 < D; e0 += kEdgeRound * 32) {
      int succ[kEdgeRound];
      uint32_t gsel[kEdgeRound];
      int old[kEdgeRound];
      int4 r0[kEdgeRound], r1[kEdgeRound];
#pragma unroll
      for (int k = 0; k < kEdgeRound; ++k) {
        succ[k] = -1;
        gsel[k] = 0;
        if (e0 + k * 32 < D) {  // warp-uniform
          const int e = e0 + k * 32 + lane;
          int owner = 0;
#pragma unroll
          for (int step = 16; step >= 1; step >>= 1) {
            const int cand = owner + step;
            const int ex = __shfl_sync(kFull, excl, cand);
            if (ex <= e) owner = cand;
          }
          const int orb = __shfl_sync(kFull, rbeg, owner);
          const int oex = __shfl_sync(kFull, excl, owner);
          gsel[k] = (uint32_t)(__shfl_sync(kFull, item, owner) >> 32);
          if (e < D) {
            const int j = e - oex;
            succ[k] = j < kAdjInline ? reinterpret_cast<const int*>(&q.bat[owner][0])[3 + j] : p.col[orb + j];
          }
        }
      }
#pragma unroll
      for (int k = 0; k < kEdgeRound; ++k) {
        old[k] = 0;
        if (succ[k] >= 0) {
          old[k] = SINGLE ? atomicSub(&p.count[succ[k]], 1)
                          : (int)atomicAdd(reinterpret_cast<unsigned*>(p.count) + succ[k], 1u);
          r0[k] = __ldg(p.adj + 2 * (int64_t)succ[k]);
          r1[k] = __ldg(p.adj + 2 * (int64_t)succ[k] + 1);
        }
      }
#pragma unroll
      for (int k = 0; k < kEdgeRound; ++k) {
        if (e0 + k * 32 >= D) break;  // warp-uniform
        // one graph counts down and re-arms; a batch's counters count up across
        // its replays (the successor's in-degree is in its speculative record,
        // the run in the item's high bits)
        const bool ready = succ[k] >= 0 && (SINGLE ? old[k] == 1
                                                   : (uint32_t)old[k] + 1u == ((gsel[k] >> 20) + 1u) * (uint32_t)r0[k].z);
        const unsigned rm = __ballot_sync(kFull, ready);
        if (!rm) continue;
        const uint64_t nit = ((uint64_t)gsel[k] << 32) | (uint32_t)succ[k];
        const int r = __popc(rm);
        const int rank = __popc(rm & lt);
        int room = p.keep - nl;
        if (room < 0) room = 0;
        if (ready && rank < room) {
          q.item[nl + rank] = nit;
          q.adj[nl + rank][0] = r0[k];
          q.adj[nl + rank][1] = r1[k];
        }
        const int nover = r > room ? r - room : 0;
        if (nover > 0) {
          uint32_t base = 0;
          if (lane == 0) base = atomicAdd(&ctrl->tail, (uint32_t)nover);
          base = __shfl_sync(kFull, base, 0);
          if ((uint64_t)base + (uint64_t)nover > (uint64_t)p.ring_cap) {
            if (lane == 0) atomicCAS(&ctrl->status, 0u, (uint32_t)RT_ERR_OOM);
          } else if (ready && rank >= room) {
            st_release_u64(p.ring + base + (rank - room), nit);
          }
          cnt[kCntPushed] += (unsigned)nover;
        }
        const int kept = r < room ? r : room;
        cnt[kCntKept] += (unsigned)kept;
        nl += kept;
        __syncwarp();
      }
    }

    // completion accounting
    const unsigned hm = __ballot_sync(kFull, has);
    cnt[kCntBatches] += 1;
    cnt[kCntTasks] += (unsigned)__popc(hm);
    if (SINGLE) {
      pend += (uint32_t)__popc(hm);
      if (pend >= 4096u) flush();
    } else {
      // per graph, immediately: a finished run re-seeds that graph at once
      const int gkey = has ? g : -1;
      const unsigned peers = __match_any_sync(kFull, gkey);
      bool cross = false;
      uint32_t runs_done = 0;
      // release: the bodies' effects before the count (a finished run starts the
      // next one); the counters need none, as they are never re-armed here
      if ((FENCE || TICKETS) && hm) fence_acq_rel_gpu();
      if (has && (peers & lt) == 0) {
        const uint32_t c = (uint32_t)__popc(peers);
        const uint32_t ng = (uint32_t)p.graphs[g].n_tasks;
        const uint32_t now = atomicAdd(&p.done_g[g], c) + c;
        if (now % ng == 0u) {
          cross = true;
          runs_done = now / ng;
        }
      }
      pend += (uint32_t)__popc(hm);
      if (pend >= 256u && lane == 0) atomicAdd(&ctrl->executed, (unsigned long long)pend);
      if (pend >= 256u) pend = 0;
      unsigned cm = __ballot_sync(kFull, cross);
      while (cm) {
        const int L = __ffs((int)cm) - 1;
        cm &= cm - 1;
        const uint32_t rd = __shfl_sync(kFull, runs_done, L);
        on_run_complete(p, __shfl_sync(kFull, g, L), rd, lane, (uint64_t)rd << 52);
      }
    }
  }
  if (lane == 0) {
#pragma unroll
    for (int k = 0; k < kCntCount; ++k)
      if (cnt[k]) atomicAdd(&ctrl->counters[k], (unsigned long long)cnt[k]);
  }
}

// The owned-chunk executor (RT_EXEC_OWNED, one graph). Algorithm 1 compiles
// every operation to one worker; here warp w owns chunks c = w, w + W, w + 2W
// ... of C consecutive tasks (W = warps of the grid) and runs them in that
// order. Each task of a chunk is held by a group of L consecutive lanes
// (C = 32 / L). Every lane of a group polls the task's countdown (one
// coalesced load per chunk and poll; the group reads one word in one load, so
// its lanes agree on readiness), and once it reads 0 the group runs the task:
// its head lane re-arms the countdown (INIT for the next run) and runs the
// body in place, and every lane decrements the successors held in its part
// of the task's trigger record with fire-and-forget reductions
// (COMPLETED_EDGE needs no answer: the successor's owner sees the zero when
// it polls). A record is R = 2 int4 per task (kAdjInline successors inline)
// or, when some task has more, R = 4 (the extension record adds successors
// up to kAdjWide); lane h of a group holds record int4s [h R / L,
// (h + 1) R / L). A warp alone on its SM hides no instruction latency, and a
// predicated reduction slot costs about the same whether or not its lanes
// are active, so spreading a record over L lanes cuts the slots one wave
// issues from 4R to 4R / L. Successors past the record take the warp-shared
// path through the CSR's columns. No ring, no reservation, no record load on
// the critical path: a wavefront step costs a reduction reaching L2 and the
// owner's next poll (issued before the wave's bodies run, and read after).
// Every warp takes its chunks in increasing task order and holds its oldest
// unfinished one, and every edge points to a later task, so the smallest
// unfinished task is always in a chunk its owner holds, with all its
// predecessors done: no warp waits forever. Replays: a warp starts run r+1
// once every task of run r has run (a counter of finished tasks), so a run's
// decrements never reach a counter of the run before. Waits are bounded by
// timeout_ns without global progress.
constexpr uint32_t kOwnedBackoffMax = 256;  // ns between polls of a warp whose tasks are all waiting

template <bool TICKETS, bool FENCE, int L, bool BATCHED>
__global__ void __launch_bounds__(256, 1) k_exec_owned(ExecParams p) {
  constexpr int C = 32 / L;   // tasks per chunk
  constexpr int QM = 4 / L;   // record int4s one lane holds at most
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int grp = lane / L, h = lane % L;  // the lane's task in the chunk, its part of the record
  const int W = (int)(gridDim.x * (blockDim.x >> 5));
  const int gw = (int)blockIdx.x * (int)(blockDim.x >> 5) + warp;
  ExecCtrl* ctrl = p.ctrl;
  const ExecGraph& G = p.graphs[0];
  const int n = BATCHED ? p.owned_n : G.n_tasks;
  const int body = G.body, spin = G.spin_iters;
  int32_t* const out = G.out;
  const int nchunks = (n + C - 1) / C;
  constexpr bool batched = BATCHED;  // a batch: bodies run with their own graph's table entry
  const int R = p.adjx != nullptr ? 4 : 2;              // int4s per trigger record
  const int inl = 4 * R - 3;                            // successors a record holds
  const int g0 = h * R / L, nq = (h + 1) * R / L - g0;  // this lane's record int4s [g0, g0 + nq)
  const int head = (L + R - 1) / R - 1;                 // the group's lane holding int4 0
  const bool is_head = h == head;
  const int head_lane = grp * L + head;
  const unsigned heads = __ballot_sync(kFull, is_head);
  uint32_t edges = 0;  // out-edges of the tasks this lane ran as head (diagnostics)
  uint32_t cnt[kCntCount];
#pragma unroll
  for (int k = 0; k < kCntCount; ++k) cnt[k] = 0;
  uint64_t idle_since = 0, last_check = 0;  // lane 0
  unsigned long long seen = 0;
  bool stop = false;

  // lane 0 of a warp that has nothing to do: is the launch over (status), or
  // has no task anywhere run for timeout_ns? (the shared status and progress
  // words are read at most every 2 us per warp: every waiting warp reading
  // them at every poll would pile onto one L2 line)
  auto idle_check = [&]() -> bool {
    int st = 0;
    if (lane == 0) {
      const uint64_t now = globaltimer_ns();
      if (idle_since == 0) {
        idle_since = last_check = now;
        seen = ld_relaxed_u64(&ctrl->executed);
      } else if (now - last_check > 2000u) {
        last_check = now;
        const unsigned long long pr = ld_relaxed_u64(&ctrl->executed);
        if (ld_relaxed_u32(&ctrl->status) != 0u) {
          st = 1;
        } else if (pr != seen) {
          seen = pr;
          idle_since = now;
        } else if (now - idle_since > (uint64_t)p.timeout_ns) {
          atomicCAS(&ctrl->status, 0u, (uint32_t)RT_ERR_TIMEOUT);
          st = 1;
        }
      }
    }
    return __shfl_sync(kFull, st, 0) != 0;
  };

  for (int r = 0; r < p.replays && !stop; ++r) {
    if (r > 0) {
      // run r starts once every task of run r - 1 has run and re-armed itself
      const uint32_t target = (uint32_t)r * (uint32_t)n;
      for (;;) {
        uint32_t d = 0;
        if (lane == 0) d = ld_relaxed_u32(&p.done_g[0]);
        d = __shfl_sync(kFull, d, 0);
        if (d >= target) break;
        if (idle_check()) {
          stop = true;
          break;
        }
        __nanosleep(64);
      }
      if (stop) break;
      idle_since = 0;
      fence_acq_rel_gpu();  // acquire: the counters re-armed by run r - 1
    }
    uint32_t ran = 0;  // tasks this warp ran in run r (warp-uniform)
    int next_c = gw;   // the next chunk this warp takes
    int ck = -1, v = 0, ctasks = 0, deg = 0, dmax = 0, gi = 0;
    int4 q[QM];        // this lane's part of its task's trigger record
    int32_t polled = 1;  // the lane's countdown, polled one round ahead
    unsigned pending = 0u;
    auto take = [&]() {
      ck = -1;
      ctasks = 0;
      pending = 0u;
      polled = 1;
      deg = 0;
      dmax = 0;
      if (next_c >= nchunks) return;
      ck = next_c;
      next_c += W;
      v = ck * C + grp;
      const bool has = v < n;
#pragma unroll
      for (int k = 0; k < QM; ++k) {
        const int g = g0 + k;
        q[k] = make_int4(-1, -1, -1, -1);
        if (k < nq && has) q[k] = __ldg(g < 2 ? p.adj + 2 * (int64_t)v + g : p.adjx + 2 * (int64_t)v + (g - 2));
      }
      if (has) polled = ld_relaxed_s32(p.count + v);
      if (batched && has) gi = __ldg(p.task_graph + v);
      pending = __ballot_sync(kFull, has);
      ctasks = __popc(pending & heads);
      deg = __shfl_sync(kFull, q[0].y, head_lane);  // the head's int4 0: {row start, degree, in-degree, s0}
      if (!has) deg = 0;
      dmax = (int)__reduce_max_sync(kFull, (unsigned)deg);  // record slots past it stay unissued
    };
    take();
    uint32_t backoff = 0;
    for (;;) {
      if (pending == 0u || stop) break;
      const bool ready = ((pending >> lane) & 1u) && polled == 0;
      const unsigned rm = __ballot_sync(kFull, ready);
      if (!rm) {
        ++cnt[kCntIdle];
        // the first empty polls retry at once (a stale prefetch); the launch's
        // status and progress are watched once polls keep failing
        if (backoff >= 64 && idle_check()) {
          stop = true;
          break;
        }
        if (backoff) __nanosleep(backoff);
        backoff = backoff ? (backoff < kOwnedBackoffMax ? backoff * 2 : kOwnedBackoffMax) : 16;
        if ((pending >> lane) & 1u) polled = ld_relaxed_s32(p.count + v);
        continue;
      }
      backoff = 0;
      idle_since = 0;
      pending &= ~rm;
      // the next poll is in flight during the work below; a value read before
      // this warp's own decrements can only be late (counters only go down to
      // 0), never early
      if (!FENCE && !TICKETS) polled = ((pending >> lane) & 1u) ? ld_relaxed_s32(p.count + v) : 1;
      if (FENCE) fence_acq_rel_gpu();  // acquire: the predecessors' effects before the bodies
      if (ready && is_head) {
        p.count[v] = q[0].z;  // INIT's reset for the next run, done by the task itself
        if (TICKETS) p.tickets[2 * (int64_t)v] = (int32_t)atomicAdd(&ctrl->ticket, 1u);
        if (batched) {
          const ExecGraph& Gv = p.graphs[gi];  // a batched body sees its graph's own task ids
          run_body<FENCE>(Gv, v - Gv.task_base);
        } else if (!FENCE) {
          if (body == RT_BODY_SPIN) out[v] = (int32_t)spin_body((uint32_t)v, spin);
          else if (body == RT_BODY_FMA) out[v] = fma_body((uint32_t)v, spin);
        } else {
          run_body<true>(G, v);
        }
        if (TICKETS) p.tickets[2 * (int64_t)v + 1] = (int32_t)atomicAdd(&ctrl->ticket, 1u);
      }
      if (FENCE || TICKETS) {
        // release: bodies before the decrements. A task's body ran in its head
        // lane and its decrements come from every lane of its group, so the
        // warp synchronizes first: the head's writes then precede each lane's
        // fence, which releases them with that lane's reductions
        if (L > 1) __syncwarp();
        fence_acq_rel_gpu();
      }
      // COMPLETED_EDGE for every out-edge of the tasks that just ran: each
      // lane the successors in its part of the record (int4 g holds successors
      // 4g - 3 .. 4g; int4 0 only successor 0), as reductions; the warp shares
      // the edges past the record
      if (ready) {
#pragma unroll
        for (int k = 0; k < QM; ++k) {
          if (k < nq && 4 * (g0 + k) - 3 < dmax) {  // uniform when L = 1: the chunk's largest degree
            const int j = 4 * (g0 + k) - 3;  // successor index of q[k].x
            if (j >= 0 && j < deg) red_dec_s32(p.count + q[k].x);
            if (j + 1 >= 0 && j + 1 < deg) red_dec_s32(p.count + q[k].y);
            if (j + 2 >= 0 && j + 2 < deg) red_dec_s32(p.count + q[k].z);
            if (j + 3 < deg) red_dec_s32(p.count + q[k].w);
          }
        }
      }
      const bool ran_head = ready && is_head;
      if (ran_head) edges += (uint32_t)deg;
      const int extra = ran_head && deg > inl ? deg - inl : 0;
      if (__any_sync(kFull, extra > 0)) {
        int incl = extra;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
          const int y = __shfl_up_sync(kFull, incl, o);
          if (lane >= o) incl += y;
        }
        const int excl = incl - extra;
        const int D = __shfl_sync(kFull, incl, 31);
        const int rbeg = is_head ? q[0].x + inl : 0;
        for (int e0 = 0; e0 < D; e0 += 32) {
          const int e = e0 + lane;
          int owner = 0;
#pragma unroll
          for (int step = 16; step >= 1; step >>= 1) {
            const int cand = owner + step;
            if (__shfl_sync(kFull, excl, cand) <= e) owner = cand;
          }
          const int oex = __shfl_sync(kFull, excl, owner);
          const int orb = __shfl_sync(kFull, rbeg, owner);
          if (e < D) red_dec_s32(p.count + p.col[orb + (e - oex)]);
        }
      }
      if (FENCE || TICKETS) polled = ((pending >> lane) & 1u) ? ld_relaxed_s32(p.count + v) : 1;
      const int k_ran = __popc(rm & heads);
      cnt[kCntBatches] += 1;
      cnt[kCntTasks] += (unsigned)k_ran;
      ran += (uint32_t)k_ran;
      // a finished chunk: progress for the other warps' bounded waits, and the
      // warp takes its next chunk
      if (ck >= 0 && pending == 0u) {
        if (lane == 0) red_add_u64(&ctrl->executed, (unsigned long long)ctasks);
        take();
      }
    }
    if (stop) break;
    // release: this warp's bodies and re-armed counters before its count
    fence_acq_rel_gpu();
    __syncwarp();
    if (lane == 0 && ran) red_add_u32(&p.done_g[0], ran);
  }
  cnt[kCntEdges] = __reduce_add_sync(kFull, edges);
  if (lane == 0) {
#pragma unroll
    for (int k = 0; k < kCntCount; ++k)
      if (cnt[k]) atomicAdd(&ctrl->counters[k], (unsigned long long)cnt[k]);
  }
}

// trigger record of each task: {row start, out-degree, in-degree, first
// kAdjInline successors (-1 padded)}, two int4 per task; optionally the
// largest out-degree (atomicMax into *maxdeg)
__global__ void k_pack_adj(const int32_t* row_ptr, const int32_t* col, const int32_t* indeg, int64_t n,
                           int4* adj, uint32_t* maxdeg) {
  const int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (maxdeg) {  // uniform over the grid: every lane of a warp reaches the reduction
    const uint32_t m = __reduce_max_sync(0xffffffffu, v < n ? (uint32_t)(row_ptr[v + 1] - row_ptr[v]) : 0u);
    if ((threadIdx.x & 31) == 0 && m) atomicMax(maxdeg, m);
  }
  if (v >= n) return;
  const int b = row_ptr[v], d = row_ptr[v + 1] - b;
  int c[kAdjInline];
#pragma unroll
  for (int j = 0; j < kAdjInline; ++j) c[j] = j < d ? col[b + j] : -1;
  adj[2 * v] = make_int4(b, d, indeg[v], c[0]);
  adj[2 * v + 1] = make_int4(c[1], c[2], c[3], c[4]);
}

// extension record of each task for the owned-chunk executor: successors
// kAdjInline .. kAdjWide - 1 (-1 padded), two int4 per task
__global__ void k_pack_adjx(const int32_t* row_ptr, const int32_t* col, int64_t n, int4* adjx) {
  const int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= n) return;
  const int b = row_ptr[v], d = row_ptr[v + 1] - b;
  int c[kAdjWide - kAdjInline];
#pragma unroll
  for (int j = 0; j < kAdjWide - kAdjInline; ++j) c[j] = kAdjInline + j < d ? col[b + kAdjInline + j] : -1;
  adjx[2 * v] = make_int4(c[0], c[1], c[2], c[3]);
  adjx[2 * v + 1] = make_int4(c[4], c[5], c[6], c[7]);
}

// each task's graph in a batch: block k fills graph k's task range
__global__ void k_fill_task_graph(const ExecGraph* graphs, int32_t G, int32_t* out) {
  for (int32_t k = blockIdx.x; k < G; k += gridDim.x) {
    const int32_t b = graphs[k].task_base, m = graphs[k].n_tasks;
    for (int32_t i = threadIdx.x; i < m; i += blockDim.x) out[b + i] = k;
  }
}

// the largest out-degree (atomicMax into *out, zeroed by the caller)
__global__ void k_max_outdeg(const int32_t* row_ptr, int64_t n, uint32_t* out) {
  uint32_t m = 0;
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x)
    m = max(m, (uint32_t)(row_ptr[v + 1] - row_ptr[v]));
  m = __reduce_max_sync(0xffffffffu, m);
  if ((threadIdx.x & 31) == 0 && m) atomicMax(out, m);
}

__global__ void k_rebase_roots(const uint64_t* src, uint64_t* dst, int32_t n, int32_t graph,
                               int32_t task_base) {
  int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) dst[i] = ((uint64_t)(uint32_t)graph << 32) | (uint32_t)(task_base + (int32_t)(uint32_t)src[i]);
}
// the last k with first[k] <= x (first[0] = 0 <= x; first is nondecreasing)
__device__ __forceinline__ int32_t last_le(const uint32_t* first, int32_t n, uint32_t x) {
  int32_t lo = 0, hi = n - 1;
  while (lo < hi) {
    const int32_t mid = (lo + hi + 1) >> 1;
    if (first[mid] <= x) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// roots of a stacked batch: tags each with its graph (its root range's index)
__global__ void k_tag_roots(const uint64_t* src, uint64_t* dst, int64_t n, const uint32_t* root_first, int32_t G) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int32_t k = last_le(root_first, G, (uint32_t)i);
  dst[i] = ((uint64_t)(uint32_t)k << 32) | (uint32_t)src[i];
}

// every edge of a stacked batch stays inside its source task's graph
__global__ void k_check_stacked(const int32_t* row_ptr, const int32_t* col, int64_t T, const uint32_t* task_first,
                                int32_t G, uint32_t* bad) {
  const int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= T) return;
  const int32_t k = last_le(task_first, G, (uint32_t)v);
  const int32_t lo = (int32_t)task_first[k], hi = (int32_t)task_first[k + 1];
  for (int32_t e = row_ptr[v]; e < row_ptr[v + 1]; ++e) {
    const int32_t c = col[e];
    if (c < lo || c >= hi) {
      atomicOr(bad, 1u);
      return;
    }
  }
}
}  // namespace

void launch_tag_roots(const uint64_t* src, uint64_t* dst, int64_t n, const uint32_t* root_first, int32_t G,
                      cudaStream_t s) {
  if (n > 0) {
    count_launch();
    k_tag_roots<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(src, dst, n, root_first, G);
  }
}

void launch_check_stacked(const int32_t* row_ptr, const int32_t* col, int64_t T, const uint32_t* task_first,
                          int32_t G, uint32_t* bad, cudaStream_t s) {
  if (T > 0) {
    count_launch();
    k_check_stacked<<<(unsigned)((T + 255) / 256), 256, 0, s>>>(row_ptr, col, T, task_first, G, bad);
  }
}

void launch_pack_adj(const int32_t* row_ptr, const int32_t* col, const int32_t* indeg, int64_t n, int4* adj,
                     uint32_t* maxdeg, cudaStream_t s) {
  if (n > 0) {
    count_launch();
    k_pack_adj<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(row_ptr, col, indeg, n, adj, maxdeg);
  }
}

void launch_pack_adjx(const int32_t* row_ptr, const int32_t* col, int64_t n, int4* adjx, cudaStream_t s) {
  if (n > 0) {
    count_launch();
    k_pack_adjx<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(row_ptr, col, n, adjx);
  }
}

void launch_fill_task_graph(const ExecGraph* graphs, int32_t G, int32_t* out, cudaStream_t s) {
  if (G > 0) {
    count_launch();
    k_fill_task_graph<<<(unsigned)std::min<int32_t>(G, 65535), 256, 0, s>>>(graphs, G, out);
  }
}

void launch_max_outdeg(const int32_t* row_ptr, int64_t n, uint32_t* out, cudaStream_t s) {
  if (n > 0) {
    count_launch();
    const unsigned blocks = (unsigned)std::min<int64_t>((n + 255) / 256, 4096);
    k_max_outdeg<<<blocks, 256, 0, s>>>(row_ptr, n, out);
  }
}

void launch_rebase_roots(const uint64_t* src, uint64_t* dst, int32_t n, int32_t graph, int32_t task_base,
                         cudaStream_t s) {
  if (n > 0) {
    count_launch();
    k_rebase_roots<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(src, dst, n, graph, task_base);
  }
}

void launch_reset_counts(int32_t* count, const int32_t* indeg, int64_t n, int32_t hold_task,
                         int32_t hold_extra, cudaStream_t s) {
  if (n > 0) {
    count_launch();
    k_reset_counts<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(count, indeg, n, hold_task, hold_extra);
  }
}

void launch_seed(ExecParams p, int64_t ring_clear, cudaStream_t s) {
  int64_t work = ring_clear > p.total_roots ? ring_clear : p.total_roots;
  if (work < p.n_graphs) work = p.n_graphs;
  unsigned blocks = (unsigned)((work + 255) / 256);
  if (blocks < 1) blocks = 1;
  if (blocks > 4096) blocks = 4096;
  count_launch();
  k_seed<<<blocks, 256, 0, s>>>(p, ring_clear);
}

int exec_max_blocks_per_sm(int warps) {
  int nb = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_exec<false, false, true>, warps * 32,
                                                (size_t)warps * sizeof(WarpQ));
  return nb;
}

// every instantiation of the owned-chunk executor
std::vector<void (*)(ExecParams)> owned_kernels() {
  return {k_exec_owned<false, false, 1, false>, k_exec_owned<false, false, 2, false>,
          k_exec_owned<false, false, 4, false>, k_exec_owned<false, true, 1, false>,
          k_exec_owned<false, true, 2, false>,  k_exec_owned<false, true, 4, false>,
          k_exec_owned<true, false, 1, false>,  k_exec_owned<true, false, 2, false>,
          k_exec_owned<true, false, 4, false>,  k_exec_owned<true, true, 1, false>,
          k_exec_owned<true, true, 2, false>,   k_exec_owned<true, true, 4, false>,
          k_exec_owned<false, false, 1, true>,  k_exec_owned<false, false, 2, true>,
          k_exec_owned<false, false, 4, true>,  k_exec_owned<false, true, 1, true>,
          k_exec_owned<false, true, 2, true>,   k_exec_owned<false, true, 4, true>};
}

template <bool T, bool F, bool S>
void prefer_shared() {
  cudaFuncSetAttribute(k_exec<T, F, S>, cudaFuncAttributePreferredSharedMemoryCarveout,
                       cudaSharedmemCarveoutMaxShared);
}

void launch_exec(ExecParams p, int blocks, int warps, cudaStream_t s) {
  // An SM's shared-memory/L1 split is fixed while a block is resident. The
  // executor is persistent and uses little shared memory; it asks for the
  // largest carveout so that analysis kernels of other graphs (a sweep block
  // takes tens of KB) can run beside it on other streams.
  static std::once_flag carveout;
  std::call_once(carveout, [] {
    prefer_shared<false, false, true>();
    prefer_shared<false, true, true>();
    prefer_shared<true, false, true>();
    prefer_shared<true, true, true>();
    prefer_shared<false, false, false>();
    prefer_shared<false, true, false>();
    prefer_shared<true, false, false>();
    prefer_shared<true, true, false>();
    for (auto f : owned_kernels())
      cudaFuncSetAttribute(f, cudaFuncAttributePreferredSharedMemoryCarveout, cudaSharedmemCarveoutMaxShared);
  });
  const size_t smem = (size_t)warps * sizeof(WarpQ);
  if (p.keep > kKeepMax) p.keep = kKeepMax;
  if (p.keep < 0) p.keep = 0;
  if (p.claim > 32) p.claim = 32;
  if (p.claim < 1) p.claim = 1;
  const bool single = p.n_graphs == 1;
  const bool fence = p.need_fence != 0;
  count_launch();
  if (p.policy == RT_EXEC_OWNED && (single || p.task_graph)) {  // keeps nothing in shared memory
    // the claim width is the group size: lanes per task (1, 2 or 4)
    const int Lg = p.claim >= 4 ? 4 : (p.claim >= 2 ? 2 : 1);
#define GRT_OWNED(T, F, B)                                                         \
  do {                                                                            \
    if (Lg == 4) k_exec_owned<T, F, 4, B><<<blocks, warps * 32, 0, s>>>(p);        \
    else if (Lg == 2) k_exec_owned<T, F, 2, B><<<blocks, warps * 32, 0, s>>>(p);   \
    else k_exec_owned<T, F, 1, B><<<blocks, warps * 32, 0, s>>>(p);               \
  } while (0)
    if (p.task_graph) {  // a batch (it records no tickets)
      if (fence) GRT_OWNED(false, true, true); else GRT_OWNED(false, false, true);
    } else if (p.tickets) {
      if (fence) GRT_OWNED(true, true, false); else GRT_OWNED(true, false, false);
    } else {
      if (fence) GRT_OWNED(false, true, false); else GRT_OWNED(false, false, false);
    }
#undef GRT_OWNED
    return;
  }
#define GRT_EXEC(T, F, S) k_exec<T, F, S><<<blocks, warps * 32, smem, s>>>(p)
  if (p.tickets) {
    if (single) { if (fence) GRT_EXEC(true, true, true); else GRT_EXEC(true, false, true); }
    else { if (fence) GRT_EXEC(true, true, false); else GRT_EXEC(true, false, false); }
  } else {
    if (single) { if (fence) GRT_EXEC(false, true, true); else GRT_EXEC(false, false, true); }
    else { if (fence) GRT_EXEC(false, true, false); else GRT_EXEC(false, false, false); }
  }
#undef GRT_EXEC
}

void preload_exec() {
  cudaFuncAttributes a;
  cudaFuncGetAttributes(&a, k_reset_counts);
  cudaFuncGetAttributes(&a, k_seed);
  cudaFuncGetAttributes(&a, k_pack_adj);
  cudaFuncGetAttributes(&a, k_pack_adjx);
  cudaFuncGetAttributes(&a, k_fill_task_graph);
  cudaFuncGetAttributes(&a, k_max_outdeg);
  cudaFuncGetAttributes(&a, k_rebase_roots);
  cudaFuncGetAttributes(&a, k_tag_roots);
  cudaFuncGetAttributes(&a, k_check_stacked);
  cudaFuncGetAttributes(&a, k_exec<false, false, true>);
  cudaFuncGetAttributes(&a, k_exec<false, true, true>);
  cudaFuncGetAttributes(&a, k_exec<true, false, true>);
  cudaFuncGetAttributes(&a, k_exec<true, true, true>);
  cudaFuncGetAttributes(&a, k_exec<false, false, false>);
  cudaFuncGetAttributes(&a, k_exec<false, true, false>);
  cudaFuncGetAttributes(&a, k_exec<true, false, false>);
  cudaFuncGetAttributes(&a, k_exec<true, true, false>);
  for (auto f : owned_kernels()) cudaFuncGetAttributes(&a, f);
}

}  // namespace grt
