// serve.cu -- the device-resident serving executor.
//
// A persistent kernel that runs for the whole life of a server (rt_server_*).
// Host worker threads analyse arriving requests in batches on their own
// streams (server.cu); each request gets a slot of a device table, pointing
// into its batch's graph, and is *posted* through a host-mapped mailbox. Idle
// warps of this kernel take posted activations, seed the request's roots, and
// from then on its tasks are executed exactly as in
// the batch executor (countdown counters, one atomic decrement per edge, kept
// successors, a ring for the rest), interleaved with every other admitted
// graph: new requests join while others are running (continuous batching).
// When a graph's last task finishes, the kernel writes the slot's activation
// number to host-mapped memory, where the host's completion thread sees it.
//
// The ready ring is circular (the server runs indefinitely): every ring slot
// carries a 64-bit sequence number; a producer of ticket t waits until the
// slot's sequence is t, writes, then releases t+1; the consumer of ticket t
// waits for t+1, reads, then releases t+cap. The ring holds at least as many
// slots as the admitted graphs have tasks, so producers do not wait on
// consumers. All waits are bounded; a stall longer than the timeout while
// graphs are admitted ends the kernel with status TIMEOUT.
#include "bodies.cuh"
#include "grt_internal.cuh"

namespace grt {

namespace {

constexpr int kKeepS = 64;
constexpr unsigned kFullS = 0xffffffffu;
constexpr unsigned long long kNoTk = ~0ull;
constexpr int kRoundS = 4;

struct WarpQS {
  int4 adj[kKeepS][2];
  int4 bat[32][2];
  uint64_t item[kKeepS];
};

__device__ __forceinline__ unsigned long long ld_acquire_ull(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release_ull(unsigned long long* p, unsigned long long v) {
  asm volatile("st.release.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

__global__ void k_serve_init(ServeParams p) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t k = i; k < (int64_t)p.cap; k += stride) p.seq[k] = (unsigned long long)k;
  for (int64_t k = i; k < p.max_slots; k += stride) p.done_s[k] = 0;
  if (i == 0) {
    ServeCtrl* c = p.ctrl;
    c->head = 0;
    c->tail = 0;
    c->taken = 0;
    c->finished = 0;
    c->status = 0;
    c->executed = 0;
    for (int k = 0; k < 16; ++k) c->counters[k] = 0;
  }
}

// Publishes one item per lane that has one (warp-convergent): one atomic
// reserves the warp's tickets, then each lane waits (bounded) for its slot to
// be free, writes, and releases the slot's sequence.
__device__ void ring_publish(const ServeParams& p, bool has, uint64_t it, int lane, unsigned lt) {
  const unsigned m = __ballot_sync(kFullS, has);
  if (!m) return;
  unsigned long long base = 0;
  if (lane == 0) base = atomicAdd(&p.ctrl->tail, (unsigned long long)__popc(m));
  base = __shfl_sync(kFullS, base, 0);
  if (!has) return;
  const unsigned long long t = base + (unsigned long long)__popc(m & lt);
  unsigned long long* sq = p.seq + (t & (p.cap - 1));
  if (ld_acquire_ull(sq) != t) {
    const uint64_t t0 = globaltimer_ns();
    while (ld_acquire_ull(sq) != t) {
      if (globaltimer_ns() - t0 > (uint64_t)p.timeout_ns) {
        atomicCAS(&p.ctrl->status, 0u, (uint32_t)RT_ERR_TIMEOUT);
        return;
      }
      __nanosleep(64);
    }
  }
  p.items[t & (p.cap - 1)] = it;
  st_release_ull(sq, t + 1);
}

// Takes one posted activation, if any (lane 0 decides; warp-convergent):
// resets the slot's completion count and publishes its roots.
__device__ bool take_activation(const ServeParams& p, int lane, unsigned lt) {
  int slot = -1;
  if (lane == 0) {
    const uint32_t posted = p.mail->posted;
    uint32_t taken = ld_relaxed_u32(&p.ctrl->taken);
    while (taken < posted) {
      const uint32_t old = atomicCAS(&p.ctrl->taken, taken, taken + 1);
      if (old == taken) {
        slot = (int)p.mail->queue[taken % 1024u];
        break;
      }
      taken = old;
    }
  }
  slot = __shfl_sync(kFullS, slot, 0);
  if (slot < 0) return false;
  fence_acq_rel_gpu();  // the slot's table entry was written before it was posted
  const ServeSlot* S = p.slots + slot;
  const int nr = __ldcg(&S->n_roots);
  const unsigned long long* roots =
      reinterpret_cast<const unsigned long long*>(__ldcg(reinterpret_cast<const unsigned long long*>(&S->roots)));
  if (lane == 0) p.done_s[slot] = 0;
  __syncwarp();
  fence_acq_rel_gpu();
  for (int k0 = 0; k0 < nr; k0 += 32) {
    const int k = k0 + lane;
    const bool has = k < nr;
    const uint64_t it = has ? (((uint64_t)(uint32_t)slot << 32) | (uint32_t)__ldcg(roots + k)) : 0ull;
    ring_publish(p, has, it, lane, lt);
  }
  return true;
}

// a slot's table fields, read through L2 (a slot is rewritten between activations)
struct SlotView {
  const int4* adj;
  const int32_t* col;
  int32_t* count;
  int32_t* out;
  int32_t n_tasks, body, spin_iters, base;
  uint32_t gen;
};

// the CHECK body's view of a request: the batch graph's launches, and the
// request's own state and band origin, so that cell indices and task ids are
// those of the request alone
__device__ ExecGraph check_view(const ServeParams& p, int slot) {
  const ServeSlot* S = p.slots + slot;
  ExecGraph G{};
  G.req_off = reinterpret_cast<const int32_t*>(__ldcg(reinterpret_cast<const unsigned long long*>(&S->req_off)));
  G.lo = reinterpret_cast<const int64_t*>(__ldcg(reinterpret_cast<const unsigned long long*>(&S->lo)));
  G.hi = reinterpret_cast<const int64_t*>(__ldcg(reinterpret_cast<const unsigned long long*>(&S->hi)));
  G.priv = reinterpret_cast<const uint8_t*>(__ldcg(reinterpret_cast<const unsigned long long*>(&S->priv)));
  G.state = reinterpret_cast<int32_t*>(__ldcg(reinterpret_cast<const unsigned long long*>(&S->state)));
  G.dom_lo[0] = __ldcg(reinterpret_cast<const long long*>(&S->band_lo[0]));
  G.dom_lo[1] = __ldcg(reinterpret_cast<const long long*>(&S->band_lo[1]));
  G.ext[0] = __ldcg(reinterpret_cast<const long long*>(&S->ext0));
  G.ext[1] = 1;
  G.ndim = __ldcg(&S->ndim);
  return G;
}

__device__ __forceinline__ SlotView slot_view(const ServeParams& p, int slot) {
  const ServeSlot* S = p.slots + slot;
  const unsigned long long* w = reinterpret_cast<const unsigned long long*>(S);
  SlotView v;
  v.adj = reinterpret_cast<const int4*>(__ldcg(w + 0));
  v.col = reinterpret_cast<const int32_t*>(__ldcg(w + 1));
  v.count = reinterpret_cast<int32_t*>(__ldcg(w + 2));
  v.out = reinterpret_cast<int32_t*>(__ldcg(w + 4));
  v.n_tasks = __ldcg(&S->n_tasks);
  v.body = __ldcg(&S->body);
  v.spin_iters = __ldcg(&S->spin_iters);
  v.gen = __ldcg(&S->gen);
  v.base = __ldcg(&S->base);
  return v;
}

__global__ void __launch_bounds__(256, 1) k_serve(ServeParams p) {
  extern __shared__ int4 serve_smem[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  WarpQS& q = reinterpret_cast<WarpQS*>(serve_smem)[warp];
  ServeCtrl* ctrl = p.ctrl;
  const unsigned lt = lanemask_lt();
  int nl = 0;
  unsigned long long my_t = kNoTk;
  uint64_t idle_since = 0, last_check = 0;
  unsigned long long seen = 0;
  uint32_t backoff = 32;
  uint32_t pend = 0;
  uint64_t last_mail = 0;
  uint32_t iter = 0;

  for (;;) {
    // force-stop (mailbox stop == 2): leave at once, even with graphs admitted
    if ((++iter & 63u) == 0u) {
      int fs = 0;
      if (lane == 0) fs = p.mail->stop == 2u;
      if (__shfl_sync(kFullS, fs, 0)) break;
    }
    uint64_t item = kEmpty64;
    int4 a0 = make_int4(0, 0, 0, -1), a1 = make_int4(-1, -1, -1, -1);
    bool have_rec = false;
    bool waiting = my_t != kNoTk;
    if (waiting) {
      unsigned long long* sq = p.seq + (my_t & (p.cap - 1));
      if (ld_acquire_ull(sq) == my_t + 1) {
        item = p.items[my_t & (p.cap - 1)];
        st_release_ull(sq, my_t + p.cap);  // the slot is free for ticket my_t + cap
        my_t = kNoTk;
        waiting = false;
      }
    }
    if (nl > 0) {
      const unsigned need = __ballot_sync(kFullS, item == kEmpty64);
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
    if (!__any_sync(kFullS, item != kEmpty64)) {
      if (pend && lane == 0) atomicAdd(&ctrl->executed, (unsigned long long)pend);
      pend = 0;
      // the mailbox lives in host memory: one warp per block looks, at most
      // every 2 us, instead of every idle warp on every idle pass
      if (warp == 0) {
        uint64_t now = 0;
        if (lane == 0) now = globaltimer_ns();
        now = __shfl_sync(kFullS, now, 0);
        if (now - last_mail >= 2000u) {
          last_mail = now;
          if (take_activation(p, lane, lt)) continue;
        }
      }
      if (!__any_sync(kFullS, waiting)) {
        unsigned long long h = 0;
        if (lane == 0) h = atomicAdd(&ctrl->head, (unsigned long long)p.claim);
        h = __shfl_sync(kFullS, h, 0);
        if (lane < p.claim) my_t = h + (unsigned long long)lane;
        continue;
      }
      int stop = 0;
      if (lane == 0) {
        const uint32_t st = ld_relaxed_u32(&ctrl->status);
        const uint32_t taken = ld_relaxed_u32(&ctrl->taken);
        const uint32_t fin = ld_relaxed_u32(&ctrl->finished);
        if (st != 0u || p.mail->stop == 2u) {
          stop = 1;
        } else if (taken == fin) {
          idle_since = 0;  // nothing admitted: idling is not a stall
          if (p.mail->stop && p.mail->posted == taken) stop = 1;
        } else {
          const uint64_t now = globaltimer_ns();
          if (idle_since == 0) {
            idle_since = last_check = now;
            seen = ld_relaxed_u64(&ctrl->executed) + fin;
          } else if (now - last_check > 20000u) {
            last_check = now;
            const unsigned long long pr = ld_relaxed_u64(&ctrl->executed) + fin;
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
      if (__shfl_sync(kFullS, stop, 0)) break;
      __nanosleep(backoff);
      if (backoff < 1024) backoff <<= 1;
      continue;
    }
    backoff = 32;
    idle_since = 0;

    // one batch: up to 32 tasks, possibly of different graphs
    const bool has = item != kEmpty64;
    const int v = (int)(uint32_t)item;
    const int slot = has ? (int)(item >> 32) : 0;
    SlotView S{};
    if (has) S = slot_view(p, slot);
    if (has && !have_rec) {
      a0 = __ldcg(S.adj + 2 * (int64_t)v);
      a1 = __ldcg(S.adj + 2 * (int64_t)v + 1);
    }
    const int rbeg = has ? a0.x : 0;
    const int deg = has ? a0.y : 0;
    q.bat[lane][0] = a0;
    q.bat[lane][1] = a1;
    // an order-sensitive body reads what its predecessors wrote: acquire their
    // effects before it runs and release its own before the decrements
    const bool chk = __any_sync(kFullS, has && S.body == RT_BODY_CHECK);
    if (chk) fence_acq_rel_gpu();
    if (has) {
      // (no counter re-arm: every served request is analysed afresh)
      if (S.body == RT_BODY_SPIN && S.out) {
        S.out[v] = (int32_t)spin_body((uint32_t)(v - S.base), S.spin_iters);  // id within its request
      } else if (S.body == RT_BODY_CHECK) {
        const ExecGraph G = check_view(p, slot);
        S.out[v] = (int32_t)check_apply(G, v, (uint32_t)(v - S.base));
      }
    }
    if (chk) fence_acq_rel_gpu();
    __syncwarp();

    int incl = deg;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(kFullS, incl, o);
      if (lane >= o) incl += y;
    }
    const int excl = incl - deg;
    const int D = __shfl_sync(kFullS, incl, 31);
    for (int e0 = 0; e0 < D; e0 += kRoundS * 32) {
      int succ[kRoundS], old[kRoundS], sl[kRoundS];
      int32_t* cnt_ptr[kRoundS];
      const int4* adj_ptr[kRoundS];
      int4 r0[kRoundS], r1[kRoundS];
#pragma unroll
      for (int k = 0; k < kRoundS; ++k) {
        succ[k] = -1;
        sl[k] = 0;
        cnt_ptr[k] = nullptr;
        adj_ptr[k] = nullptr;
        if (e0 + k * 32 < D) {
          const int e = e0 + k * 32 + lane;
          int owner = 0;
#pragma unroll
          for (int step = 16; step >= 1; step >>= 1) {
            const int cand = owner + step;
            if (__shfl_sync(kFullS, excl, cand) <= e) owner = cand;
          }
          const int orb = __shfl_sync(kFullS, rbeg, owner);
          const int oex = __shfl_sync(kFullS, excl, owner);
          sl[k] = __shfl_sync(kFullS, slot, owner);
          cnt_ptr[k] = reinterpret_cast<int32_t*>(
              __shfl_sync(kFullS, reinterpret_cast<unsigned long long>(S.count), owner));
          adj_ptr[k] = reinterpret_cast<const int4*>(
              __shfl_sync(kFullS, reinterpret_cast<unsigned long long>(S.adj), owner));
          const int32_t* ocol = reinterpret_cast<const int32_t*>(
              __shfl_sync(kFullS, reinterpret_cast<unsigned long long>(S.col), owner));
          if (e < D) {
            const int j = e - oex;
            succ[k] = j < kAdjInline ? reinterpret_cast<const int*>(&q.bat[owner][0])[3 + j] : __ldcg(ocol + orb + j);
          }
        }
      }
#pragma unroll
      for (int k = 0; k < kRoundS; ++k) {
        old[k] = 0;
        if (succ[k] >= 0) {
          old[k] = atomicSub(cnt_ptr[k] + succ[k], 1);
          r0[k] = __ldcg(adj_ptr[k] + 2 * (int64_t)succ[k]);
          r1[k] = __ldcg(adj_ptr[k] + 2 * (int64_t)succ[k] + 1);
        }
      }
#pragma unroll
      for (int k = 0; k < kRoundS; ++k) {
        if (e0 + k * 32 >= D) break;
        const bool ready = succ[k] >= 0 && old[k] == 1;
        const unsigned rm = __ballot_sync(kFullS, ready);
        if (!rm) continue;
        const uint64_t nit = ((uint64_t)(uint32_t)sl[k] << 32) | (uint32_t)succ[k];
        const int r = __popc(rm);
        const int rank = __popc(rm & lt);
        int room = p.keep - nl;
        if (room < 0) room = 0;
        if (ready && rank < room) {
          q.item[nl + rank] = nit;
          q.adj[nl + rank][0] = r0[k];
          q.adj[nl + rank][1] = r1[k];
        }
        ring_publish(p, ready && rank >= room, nit, lane, lt);
        nl += r < room ? r : room;
        __syncwarp();
      }
    }

    // completion accounting per graph: outputs and decrements are released
    // before the count, so a completed graph's buffers are final when the host
    // sees its completion
    fence_acq_rel_gpu();
    const int gkey = has ? slot : -1;
    const unsigned peers = __match_any_sync(kFullS, gkey);
    if (has && (peers & lt) == 0) {
      const uint32_t c = (uint32_t)__popc(peers);
      const uint32_t now = atomicAdd(&p.done_s[slot], c) + c;
      if (now == (uint32_t)S.n_tasks) {
        // the graph finished: publish it to the host, then count it
        __threadfence_system();
        p.done_gen[slot] = S.gen;
        __threadfence_system();
        atomicAdd(&ctrl->finished, 1u);
      }
    }
    pend += (uint32_t)__popc(__ballot_sync(kFullS, has));
    if (pend >= 256u) {
      if (lane == 0) atomicAdd(&ctrl->executed, (unsigned long long)pend);
      pend = 0;
    }
  }
}

__global__ void k_serve_gather(const uint32_t* rootpos, const int32_t* row_ptr, const int32_t* idx, int k,
                               uint32_t* out) {
  const int i = (int)(blockIdx.x * blockDim.x + threadIdx.x);
  if (i < k) {
    const int t = idx[i];
    out[2 * i] = rootpos[t];
    out[2 * i + 1] = (uint32_t)row_ptr[t];
  }
}

}  // namespace

void launch_serve_gather(const uint32_t* rootpos, const int32_t* row_ptr, const int32_t* idx, int k, uint32_t* out,
                         cudaStream_t s) {
  count_launch();
  k_serve_gather<<<(k + 127) / 128, 128, 0, s>>>(rootpos, row_ptr, idx, k, out);
}

void launch_serve_init(ServeParams p, cudaStream_t s) {
  unsigned long long work = p.cap > (unsigned long long)p.max_slots ? p.cap : (unsigned long long)p.max_slots;
  unsigned blocks = (unsigned)((work + 255) / 256);
  if (blocks > 4096) blocks = 4096;
  count_launch();
  k_serve_init<<<blocks, 256, 0, s>>>(p);
}

void launch_serve(ServeParams p, int blocks, int warps, cudaStream_t s) {
  const size_t smem = (size_t)warps * sizeof(WarpQS);
  if (p.keep > kKeepS) p.keep = kKeepS;
  if (p.claim > 32) p.claim = 32;
  if (p.claim < 1) p.claim = 1;
  // An SM's shared-memory/L1 split is fixed while a block is resident. This
  // kernel stays resident on every SM for the server's life, so it asks for
  // the largest shared-memory carveout: analysis kernels launched by the
  // workers (the tile sweep needs tens of KB per block) must fit beside it.
  cudaFuncSetAttribute(k_serve, cudaFuncAttributePreferredSharedMemoryCarveout, cudaSharedmemCarveoutMaxShared);
  count_launch();
  k_serve<<<blocks, warps * 32, smem, s>>>(p);
}

void preload_serve() {
  cudaFuncAttributes a;
  cudaFuncGetAttributes(&a, k_serve_init);
  cudaFuncGetAttributes(&a, k_serve);
  cudaFuncGetAttributes(&a, k_serve_gather);
}

}  // namespace grt
