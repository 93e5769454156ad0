// analysis.cu -- implicit dependence analysis on the GPU.
//
// Pipeline (one graph, all launches so far):
//  1. bin count:  each rectangle -> number of tiles it overlaps
//  2. scan + expand: one (tile, packed entry) per overlap, written in
//     rectangle order with coalesced int4 loads of the rectangle arrays
//  3. stable radix sort by tile -> per tile, its candidates in program order
//  4. sweep (sweep.cu): one warp per tile walks the candidates in program
//     order, keeps per-cell run state in shared memory and emits (src, dst)
//     pairs deduplicated per task within the tile
//     (tiles whose pairs overflowed the buffer are swept again, alone, into a
//     larger one)
//  5. radix sort of the 64-bit pair keys, unique, CSR by source: row counts
//     and in-degrees by warp-aggregated atomics, row_ptr by a device scan
//  6. countdown counters (the in-degrees) and the compacted root list; the
//     executor's trigger records are packed from the CSR (exec.cu)
//
// The edge rule is the per-cell run reading of "infer the DAG from the data
// usage of tasks" (Section 2.2, Section 5): a task's rectangles combine into
// one privilege per cell, and each access gets edges from every member of the
// run preceding its own run at that cell.
#include "grt_internal.cuh"

namespace grt {

namespace {

// error bits of the device-side validation
constexpr uint32_t kErrReqOff = 1u, kErrRect = 2u, kErrPriv = 4u, kErrPred = 8u, kErrBodyArg = 16u, kErrBand = 32u;

// the last k in [0, n) with first[k] <= x (first[0] <= x, first nondecreasing)
__device__ __forceinline__ int32_t last_at_most(const int32_t* first, int32_t n, int64_t x) {
  int32_t lo = 0, hi = n - 1;
  while (lo < hi) {
    const int32_t mid = (lo + hi + 1) >> 1;
    if ((int64_t)first[mid] <= x) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// Band placement of a captured batch (rt_batch_capture): rectangle r belongs
// to the task whose rectangle range holds it, which belongs to graph k; it must
// lie in graph k's own domain (kErrBand otherwise) and moves by graph k's shift
// into its band of the stacked domain. box[k] = {lo[D], hi[D], shift[D]}.
__global__ void k_band_place(const int32_t* req_off, int32_t n, const int32_t* task_first, int32_t G,
                             const int64_t* box, int D, int64_t* lo, int64_t* hi, int64_t R, uint32_t* err) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < R; r += stride) {
    const int32_t t = last_at_most(req_off, n, r);
    const int32_t k = last_at_most(task_first, G, t);
    const int64_t* b = box + (int64_t)k * 3 * D;
    bool outside = false;
    for (int d = 0; d < D; ++d) {
      const int64_t a = lo[r * D + d], c = hi[r * D + d];
      if (a < b[d] || c > b[D + d]) outside = true;
      lo[r * D + d] = a + b[2 * D + d];
      hi[r * D + d] = c + b[2 * D + d];
    }
    if (outside) atomicOr(err, kErrBand);
  }
}

// Checks one appended batch whose offsets were already shifted to graph-wide
// positions: req_off[0..n] must run from r_first to r_end without decreasing;
// pred_off likewise from p_first to p_end, every pred in [0, own id).
__global__ void k_validate_tasks(const int32_t* req_off, int32_t n, int64_t r_first, int64_t r_end,
                                 const int32_t* pred_off, const int32_t* pred, int64_t p_first,
                                 int64_t p_end, int32_t task_base, const int32_t* body_arg,
                                 int64_t body_limit, uint32_t* err) {
  int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i > n) return;
  uint32_t e = 0;
  if (i == 0 && (int64_t)req_off[0] != r_first) e |= kErrReqOff;
  if (i == n && (int64_t)req_off[n] != r_end) e |= kErrReqOff;
  if (pred_off && i == 0 && (int64_t)pred_off[0] != p_first) e |= kErrPred;
  if (pred_off && i == n && (int64_t)pred_off[n] != p_end) e |= kErrPred;
  if (i < n) {
    if (req_off[i + 1] < req_off[i]) e |= kErrReqOff;
    if (pred_off) {
      int32_t a = pred_off[i], b = pred_off[i + 1];
      if (b < a || (int64_t)a < p_first || (int64_t)b > p_end) {
        e |= kErrPred;
      } else {
        for (int32_t k = a; k < b; ++k) {
          int32_t p = pred[k];
          if (p < 0 || p >= task_base + i) {
            e |= kErrPred;
            break;
          }
        }
      }
    }
    if (body_arg && body_limit >= 0) {
      int32_t v = body_arg[i];
      if (v < 0 || (int64_t)v >= body_limit) e |= kErrBodyArg;
    }
  }
  if (e) atomicOr(err, e);
}

__global__ void k_validate_rects(const int64_t* lo, const int64_t* hi, const uint8_t* priv, int64_t R,
                                 AnalysisDims d, uint32_t* err) {
  int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= R) return;
  uint32_t e = 0;
  for (int k = 0; k < d.ndim; ++k) {
    int64_t a = lo[r * d.ndim + k], b = hi[r * d.ndim + k];
    if (a > b || a < d.dom_lo[k] || b > d.dom_lo[k] + d.ext[k] - 1) e |= kErrRect;
  }
  if (priv[r] > 2) e |= kErrPriv;
  if (e) atomicOr(err, e);
}

__global__ void k_add_offset(int32_t* a, int64_t n, int32_t add) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) a[i] += add;
}

// int32 rectangle bounds (both arrays, m values each) widened to int64 in the
// graph's own arrays
__global__ void k_widen_bounds(const int32_t* lo32, const int32_t* hi32, int64_t m, int64_t* lo, int64_t* hi) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += stride) {
    lo[i] = lo32[i];
    hi[i] = hi32[i];
  }
}

// tile range of one rectangle (coordinates relative to the domain origin)
struct TileRange {
  int64_t lx, hx, ly, hy;  // relative inclusive bounds
  int32_t tx0, ty0, ntx, nty;
};

__device__ __forceinline__ TileRange tile_range(const int64_t* lo, const int64_t* hi, int64_t r,
                                                const AnalysisDims& d) {
  TileRange t;
  if (d.ndim == 2) {
    // one 16-byte load per corner: the rectangle arrays are int64[R][2]
    longlong2 a = *reinterpret_cast<const longlong2*>(lo + 2 * r);
    longlong2 b = *reinterpret_cast<const longlong2*>(hi + 2 * r);
    t.lx = a.x - d.dom_lo[0];
    t.hx = b.x - d.dom_lo[0];
    t.ly = a.y - d.dom_lo[1];
    t.hy = b.y - d.dom_lo[1];
  } else {
    t.lx = lo[r] - d.dom_lo[0];
    t.hx = hi[r] - d.dom_lo[0];
    t.ly = 0;
    t.hy = 0;
  }
  t.tx0 = (int32_t)(t.lx / d.tw);
  t.ty0 = (int32_t)(t.ly / d.th);
  t.ntx = (int32_t)(t.hx / d.tw) - t.tx0 + 1;
  t.nty = (int32_t)(t.hy / d.th) - t.ty0 + 1;
  return t;
}

__global__ void k_bin_count(const int32_t* req_off, int32_t n, const int64_t* lo, const int64_t* hi,
                            AnalysisDims d, int32_t* rect_task, uint64_t* cnt) {
  int32_t t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n) return;
  for (int32_t r = req_off[t]; r < req_off[t + 1]; ++r) {
    rect_task[r] = t;
    TileRange tr = tile_range(lo, hi, r, d);
    cnt[r] = (uint64_t)tr.ntx * (uint64_t)tr.nty;
  }
}

// One thread per rectangle: a rectangle over a few tiles writes its own
// entries; the entries of a larger one are written by its whole warp
// (lane-strided), so that large rectangles do not serialise on one lane.
constexpr uint64_t kOwnTiles = 4;

__global__ void k_bin_expand(const int32_t* rect_task, const int64_t* lo, const int64_t* hi,
                             const uint8_t* priv, int64_t R, const uint64_t* off, AnalysisDims d,
                             uint32_t* keys, uint64_t* payload) {
  const int lane = threadIdx.x & 31;
  int64_t r = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x);
  bool valid = r < R;
  TileRange tr{};
  uint64_t base = 0, cnt = 0;
  uint32_t task = 0, pv = 0;
  if (valid) {
    tr = tile_range(lo, hi, r, d);
    base = off[r];
    cnt = off[r + 1] - base;
    task = (uint32_t)rect_task[r];
    pv = priv[r];
  }
  // A rectangle over at most kOwnTiles tiles (the usual case: one) is written
  // by its own lane; consecutive rectangles then write consecutive entries, so
  // the stores coalesce. Larger ones are written by the whole warp below.
  const bool own = valid && cnt <= (uint64_t)kOwnTiles;
  if (own) {
    for (uint64_t k = 0; k < cnt; ++k) {
      const int32_t tx = tr.tx0 + (int32_t)(k % (uint64_t)tr.ntx);
      const int32_t ty = tr.ty0 + (int32_t)(k / (uint64_t)tr.ntx);
      const int64_t ox = (int64_t)tx * d.tw, oy = (int64_t)ty * d.th;
      const int64_t x0 = (tr.lx > ox ? tr.lx : ox) - ox, x1 = (tr.hx < ox + d.tw - 1 ? tr.hx : ox + d.tw - 1) - ox;
      const int64_t y0 = (tr.ly > oy ? tr.ly : oy) - oy, y1 = (tr.hy < oy + d.th - 1 ? tr.hy : oy + d.th - 1) - oy;
      keys[base + k] = (uint32_t)ty * (uint32_t)d.ntx + (uint32_t)tx;
      payload[base + k] = pack_entry(task, pv, d.ndim, (uint32_t)x0, (uint32_t)x1, (uint32_t)y0, (uint32_t)y1);
    }
  }
  unsigned shared = __ballot_sync(0xffffffffu, valid && !own && cnt > 0);
  while (shared) {
    const int i = __ffs((int)shared) - 1;
    shared &= shared - 1;
    uint64_t c = __shfl_sync(0xffffffffu, cnt, i);
    uint64_t b = __shfl_sync(0xffffffffu, base, i);
    int64_t lx = __shfl_sync(0xffffffffu, tr.lx, i), hx = __shfl_sync(0xffffffffu, tr.hx, i);
    int64_t ly = __shfl_sync(0xffffffffu, tr.ly, i), hy = __shfl_sync(0xffffffffu, tr.hy, i);
    int32_t tx0 = __shfl_sync(0xffffffffu, tr.tx0, i), ty0 = __shfl_sync(0xffffffffu, tr.ty0, i);
    int32_t ntx = __shfl_sync(0xffffffffu, tr.ntx, i);
    uint32_t tk = __shfl_sync(0xffffffffu, task, i), p = __shfl_sync(0xffffffffu, pv, i);
    for (uint64_t k = lane; k < c; k += 32) {
      int32_t tx = tx0 + (int32_t)(k % (uint64_t)ntx);
      int32_t ty = ty0 + (int32_t)(k / (uint64_t)ntx);
      int64_t ox = (int64_t)tx * d.tw, oy = (int64_t)ty * d.th;
      int64_t x0 = (lx > ox ? lx : ox) - ox, x1 = (hx < ox + d.tw - 1 ? hx : ox + d.tw - 1) - ox;
      int64_t y0 = (ly > oy ? ly : oy) - oy, y1 = (hy < oy + d.th - 1 ? hy : oy + d.th - 1) - oy;
      keys[b + k] = (uint32_t)ty * (uint32_t)d.ntx + (uint32_t)tx;
      payload[b + k] = pack_entry(tk, p, d.ndim, (uint32_t)x0, (uint32_t)x1, (uint32_t)y0, (uint32_t)y1);
    }
  }
}

__global__ void k_segments(const uint32_t* keys, int64_t M, uint32_t* seg_begin, uint32_t* seg_end) {
  int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= M) return;
  uint32_t k = keys[e];
  if (e == 0 || keys[e - 1] != k) seg_begin[k] = (uint32_t)e;
  if (e == M - 1 || keys[e + 1] != k) seg_end[k] = (uint32_t)(e + 1);
}

__global__ void k_explicit_pairs(const int32_t* pred_off, const int32_t* pred, int32_t n, int key_bits,
                                 uint64_t* pairs) {
  int32_t t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n) return;
  for (int32_t k = pred_off[t]; k < pred_off[t + 1]; ++k)
    pairs[k] = ((uint64_t)(uint32_t)pred[k] << key_bits) | (uint32_t)t;
}

__global__ void k_unique_flags(const uint64_t* keys, int64_t P, uint32_t* flags) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= P) return;
  uint64_t k = keys[i];
  flags[i] = (k != kEmpty64 && (i == 0 || keys[i - 1] != k)) ? 1u : 0u;
}

// warp-aggregated increment: lanes adding to the same counter elect one leader
__device__ __forceinline__ void warp_agg_inc(int32_t* base, int32_t idx, bool active) {
  int32_t key = active ? idx : -1;
  unsigned peers = __match_any_sync(0xffffffffu, key);
  if (active && (peers & lanemask_lt()) == 0) red_add_s32(base + idx, (int32_t)__popc(peers));
}

__global__ void k_emit_csr(const uint64_t* keys, const uint32_t* flags, const uint32_t* upos, int64_t P,
                           int key_bits, int32_t* col, int32_t* rowcnt, int32_t* indeg) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  bool act = i < P && flags[i] != 0;
  int32_t src = 0, dst = 0;
  if (act) {
    uint64_t k = keys[i];
    src = (int32_t)(k >> key_bits);
    dst = (int32_t)(k & ((1ull << key_bits) - 1ull));
    col[upos[i]] = dst;
  }
  warp_agg_inc(rowcnt, src, act);
  warp_agg_inc(indeg, dst, act);
}

__global__ void k_root_flags(const int32_t* indeg, int32_t n, uint32_t* flags) {
  int32_t v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v < n) flags[v] = indeg[v] == 0 ? 1u : 0u;
}

__global__ void k_roots_emit(const int32_t* indeg, const uint32_t* pos, int32_t n, int32_t task_base,
                             int32_t graph, uint64_t* root_items, int32_t* count) {
  int32_t v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= n) return;
  int32_t dg = indeg[v];
  count[v] = dg;  // Algorithm 1: one pending-edge counter per node
  if (dg == 0) root_items[pos[v]] = ((uint64_t)(uint32_t)graph << 32) | (uint32_t)(task_base + v);
}

// ---------------------------------------------------------------------------
// CSR by buckets (graphs whose rows hold at most kBucketMaxRow candidate
// pairs): the pairs are counted per source, each pair's target is scattered
// into its source's bucket, every bucket is sorted and deduplicated in place,
// and the unique targets are compacted into the CSR. One pass over the pairs
// and a few over the targets, where an LSD radix sort of (source, target) keys
// makes five.
// ---------------------------------------------------------------------------
constexpr int kBucketSmallRow = 32;  // rows sorted by one thread
constexpr int kBucketLanes = 32;

// pairs counted per source; the pair count is read on the device (the sweep's
// cursor, capped at the buffer) so that no host sync is needed before it
__global__ void k_bucket_count(const uint64_t* pairs, const unsigned long long* cursor, unsigned long long cap,
                               int key_bits, uint32_t* cnt) {
  const unsigned long long P = *cursor < cap ? *cursor : cap;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i0 = (int64_t)blockIdx.x * blockDim.x; i0 < (int64_t)P; i0 += stride) {
    const int64_t i = i0 + threadIdx.x;
    const uint64_t k = i < (int64_t)P ? pairs[i] : kEmpty64;
    const int src = k != kEmpty64 ? (int)(k >> key_bits) : -1;
    const unsigned peers = __match_any_sync(0xffffffffu, src);
    if (src >= 0 && (peers & lanemask_lt()) == 0) red_add_u32(cnt + src, (uint32_t)__popc(peers));
  }
}

// the longest row (atomicMax into *out)
__global__ void k_bucket_maxrow(const uint32_t* cnt, int32_t n, uint32_t* out) {
  uint32_t m = 0;
  for (int32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) m = max(m, cnt[v]);
#pragma unroll
  for (int o = 16; o >= 1; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0 && m) atomicMax(out, m);
}

// each pair's target into its source's bucket: positions off[src] .. off[src]
// + cnt[src] - 1, handed out by counting cnt down (it ends at 0)
__global__ void k_bucket_scatter(const uint64_t* pairs, int64_t P, int key_bits, const uint32_t* off, uint32_t* cnt,
                                 uint32_t* bucket) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const uint64_t k = i < P ? pairs[i] : kEmpty64;
  const int src = k != kEmpty64 ? (int)(k >> key_bits) : -1;
  const unsigned peers = __match_any_sync(0xffffffffu, src);
  const int leader = __ffs((int)peers) - 1;
  uint32_t old = 0;
  if (src >= 0 && (peers & lanemask_lt()) == 0) old = atomicSub(cnt + src, (uint32_t)__popc(peers));
  old = __shfl_sync(0xffffffffu, old, leader);
  if (src >= 0) {
    const uint32_t rank = (uint32_t)__popc(peers & lanemask_lt());
    bucket[off[src] + old - 1u - rank] = (uint32_t)(k & ((1ull << key_bits) - 1ull));
  }
}

// rows of at most kBucketSmallRow pairs: one thread sorts its row in place
// (insertion sort) and keeps the distinct targets at its front; longer rows are
// listed for k_bucket_sort_large
__global__ void k_bucket_sort_small(const uint32_t* off, int32_t n, uint32_t* bucket, uint32_t* ucnt, uint32_t* big,
                                    uint32_t* nbig) {
  const int32_t v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= n) return;
  const uint32_t a = off[v], len = off[v + 1] - a;
  if (len > (uint32_t)kBucketSmallRow) {
    big[atomicAdd(nbig, 1u)] = (uint32_t)v;
    return;
  }
  uint32_t* b = bucket + a;
  for (uint32_t i = 1; i < len; ++i) {
    const uint32_t x = b[i];
    int j = (int)i - 1;
    while (j >= 0 && b[j] > x) {
      b[j + 1] = b[j];
      --j;
    }
    b[j + 1] = x;
  }
  uint32_t u = 0;
  for (uint32_t i = 0; i < len; ++i)
    if (u == 0 || b[i] != b[u - 1]) b[u++] = b[i];
  ucnt[v] = u;
}

// the listed long rows (at most kBucketMaxRow pairs): one warp each, a bitonic
// sort in shared memory padded with ~0, then the distinct targets written back
// to the row's front
__global__ void __launch_bounds__(128) k_bucket_sort_large(const uint32_t* off, uint32_t* bucket, uint32_t* ucnt,
                                                           const uint32_t* big, const uint32_t* nbig) {
  __shared__ uint32_t buf[4][kBucketMaxRow];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  uint32_t* s = buf[warp];
  const uint32_t nb = *nbig;
  for (uint32_t r = blockIdx.x * 4 + warp; r < nb; r += gridDim.x * 4) {
    const uint32_t v = big[r];
    const uint32_t a = off[v], len = off[v + 1] - a;
    uint32_t N = 64;
    while (N < len) N <<= 1;
    for (uint32_t i = lane; i < N; i += 32) s[i] = i < len ? bucket[a + i] : 0xFFFFFFFFu;
    __syncwarp();
    for (uint32_t k = 2; k <= N; k <<= 1) {
      for (uint32_t j = k >> 1; j > 0; j >>= 1) {
        for (uint32_t i = lane; i < N; i += 32) {
          const uint32_t p = i ^ j;
          if (p > i) {
            const uint32_t x = s[i], y = s[p];
            const bool up = (i & k) == 0;
            if ((x > y) == up) {
              s[i] = y;
              s[p] = x;
            }
          }
        }
        __syncwarp();
      }
    }
    uint32_t u = 0;
    for (uint32_t i0 = 0; i0 < len; i0 += 32) {
      const uint32_t i = i0 + lane;
      const bool keep = i < len && (i == 0 || s[i] != s[i - 1]);
      const unsigned m = __ballot_sync(0xffffffffu, keep);
      if (keep) bucket[a + u + (uint32_t)__popc(m & lanemask_lt())] = s[i];
      u += (uint32_t)__popc(m);
    }
    if (lane == 0) ucnt[v] = u;
    __syncwarp();
  }
}

// the distinct targets of every row into the CSR's columns, and in-degrees
__global__ void k_bucket_compact(const uint32_t* off, const uint32_t* row_ptr, int32_t n, const uint32_t* bucket,
                                 int32_t* col, int32_t* indeg) {
  const int32_t v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= n) return;
  const uint32_t a = off[v], o = row_ptr[v], u = row_ptr[v + 1] - o;
  for (uint32_t i = 0; i < u; ++i) {
    const uint32_t t = bucket[a + i];
    col[o + i] = (int32_t)t;
    red_add_s32(indeg + t, 1);
  }
}

inline unsigned nblk(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

}  // namespace

void launch_validate(const int32_t* req_off, int32_t n, int64_t r_first, const int64_t* lo,
                     const int64_t* hi, const uint8_t* priv, int64_t R, const int32_t* pred_off,
                     const int32_t* pred, int64_t p_first, int64_t p_end, int32_t task_base,
                     const int32_t* body_arg, int64_t body_limit, AnalysisDims d, uint32_t* err,
                     cudaStream_t s) {
  count_launch();
  k_validate_tasks<<<nblk((int64_t)n + 1, 256), 256, 0, s>>>(req_off, n, r_first, r_first + R, pred_off,
                                                           pred, p_first, p_end, task_base, body_arg,
                                                           body_limit, err);
  if (R > 0) {
    count_launch();
    k_validate_rects<<<nblk(R, 256), 256, 0, s>>>(lo, hi, priv, R, d, err);
  }
}

void launch_band_place(const int32_t* req_off, int32_t n, const int32_t* task_first, int32_t G, const int64_t* box,
                       int D, int64_t* lo, int64_t* hi, int64_t R, uint32_t* err, cudaStream_t s) {
  if (R <= 0) return;
  unsigned blocks = nblk(R, 256);
  if (blocks > 4096) blocks = 4096;
  count_launch();
  k_band_place<<<blocks, 256, 0, s>>>(req_off, n, task_first, G, box, D, lo, hi, R, err);
}

void launch_widen_bounds(const int32_t* lo32, const int32_t* hi32, int64_t m, int64_t* lo, int64_t* hi,
                         cudaStream_t s) {
  if (m <= 0) return;
  unsigned blocks = nblk(m, 256);
  if (blocks > 8192) blocks = 8192;
  count_launch();
  k_widen_bounds<<<blocks, 256, 0, s>>>(lo32, hi32, m, lo, hi);
}

void launch_add_offset(int32_t* a, int64_t n, int32_t add, cudaStream_t s) {
  if (n > 0 && add != 0) {
    count_launch();
    k_add_offset<<<nblk(n, 256), 256, 0, s>>>(a, n, add);
  }
}

void launch_bin_count(const int32_t* req_off, int32_t n, const int64_t* lo, const int64_t* hi,
                      int64_t R, AnalysisDims d, int32_t* rect_task, uint64_t* cnt, cudaStream_t s) {
  (void)R;
  if (n > 0) {
    count_launch();
    k_bin_count<<<nblk(n, 256), 256, 0, s>>>(req_off, n, lo, hi, d, rect_task, cnt);
  }
}

void launch_bin_expand(const int32_t* rect_task, const int64_t* lo, const int64_t* hi,
                       const uint8_t* priv, int64_t R, const uint64_t* off, AnalysisDims d,
                       uint32_t* keys, uint64_t* payload, cudaStream_t s) {
  if (R > 0) {
    count_launch();
    k_bin_expand<<<nblk(R, 256), 256, 0, s>>>(rect_task, lo, hi, priv, R, off, d, keys, payload);
  }
}

void launch_segments(const uint32_t* keys, int64_t M, uint32_t* seg_begin, uint32_t* seg_end,
                     cudaStream_t s) {
  if (M > 0) {
    count_launch();
    k_segments<<<nblk(M, 256), 256, 0, s>>>(keys, M, seg_begin, seg_end);
  }
}

void launch_explicit_pairs(const int32_t* pred_off, const int32_t* pred, int32_t n, int key_bits,
                           uint64_t* pairs, cudaStream_t s) {
  if (n > 0) {
    count_launch();
    k_explicit_pairs<<<nblk(n, 256), 256, 0, s>>>(pred_off, pred, n, key_bits, pairs);
  }
}

void launch_unique_flags(const uint64_t* keys, int64_t P, uint32_t* flags, cudaStream_t s) {
  if (P > 0) {
    count_launch();
    k_unique_flags<<<nblk(P, 256), 256, 0, s>>>(keys, P, flags);
  }
}

void launch_bucket_count(const uint64_t* pairs, const unsigned long long* cursor, unsigned long long cap,
                         int key_bits, uint32_t* cnt, int32_t n, uint32_t* maxrow, cudaStream_t s) {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  count_launch(2);
  k_bucket_count<<<(unsigned)(sms > 0 ? sms * 8 : 1024), 256, 0, s>>>(pairs, cursor, cap, key_bits, cnt);
  unsigned mb = nblk(n, 256);
  if (mb > 1024) mb = 1024;
  if (mb < 1) mb = 1;
  k_bucket_maxrow<<<mb, 256, 0, s>>>(cnt, n, maxrow);
}

void launch_bucket_build(const uint64_t* pairs, int64_t P, int key_bits, int32_t n, uint32_t* cnt, uint32_t* off,
                         uint32_t* ucnt, uint32_t* big, uint32_t* nbig, uint32_t* bucket, uint32_t* row_ptr,
                         uint32_t* scan_ws, int32_t* col, int32_t* indeg, cudaStream_t s) {
  scan_exclusive<uint32_t>(cnt, off, n, scan_ws, s);
  if (P > 0) {
    count_launch();
    k_bucket_scatter<<<nblk(P, 256), 256, 0, s>>>(pairs, P, key_bits, off, cnt, bucket);
  }
  cudaMemsetAsync(nbig, 0, 4, s);
  count_launch(2);
  k_bucket_sort_small<<<nblk(n, 256), 256, 0, s>>>(off, n, bucket, ucnt, big, nbig);
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  k_bucket_sort_large<<<(unsigned)(sms > 0 ? sms * 4 : 512), 128, 0, s>>>(off, bucket, ucnt, big, nbig);
  scan_exclusive<uint32_t>(ucnt, row_ptr, n, scan_ws, s);
  cudaMemsetAsync(indeg, 0, (size_t)n * 4, s);
  count_launch();
  k_bucket_compact<<<nblk(n, 256), 256, 0, s>>>(off, row_ptr, n, bucket, col, indeg);
}

void launch_emit_csr(const uint64_t* keys, const uint32_t* flags, const uint32_t* upos, int64_t P,
                     int key_bits, int32_t* col, int32_t* rowcnt, int32_t* indeg, cudaStream_t s) {
  if (P > 0) {
    count_launch();
    k_emit_csr<<<nblk(P, 256), 256, 0, s>>>(keys, flags, upos, P, key_bits, col, rowcnt, indeg);
  }
}

void launch_roots(const int32_t* indeg, int32_t n, uint32_t* flags, cudaStream_t s) {
  if (n > 0) {
    count_launch();
    k_root_flags<<<nblk(n, 256), 256, 0, s>>>(indeg, n, flags);
  }
}

void launch_roots_emit(const int32_t* indeg, const uint32_t* pos, int32_t n, int32_t task_base,
                       int32_t graph, uint64_t* root_items, int32_t* count, cudaStream_t s) {
  if (n > 0) {
    count_launch();
    k_roots_emit<<<nblk(n, 256), 256, 0, s>>>(indeg, pos, n, task_base, graph, root_items, count);
  }
}

void preload_analysis() {
  cudaFuncAttributes a;
  cudaFuncGetAttributes(&a, k_validate_tasks);
  cudaFuncGetAttributes(&a, k_validate_rects);
  cudaFuncGetAttributes(&a, k_add_offset);
  cudaFuncGetAttributes(&a, k_bin_count);
  cudaFuncGetAttributes(&a, k_bin_expand);
  cudaFuncGetAttributes(&a, k_segments);
  cudaFuncGetAttributes(&a, k_explicit_pairs);
  cudaFuncGetAttributes(&a, k_unique_flags);
  cudaFuncGetAttributes(&a, k_emit_csr);
  cudaFuncGetAttributes(&a, k_root_flags);
  cudaFuncGetAttributes(&a, k_roots_emit);
  cudaFuncGetAttributes(&a, k_band_place);
  cudaFuncGetAttributes(&a, k_widen_bounds);
  cudaFuncGetAttributes(&a, k_bucket_count);
  cudaFuncGetAttributes(&a, k_bucket_maxrow);
  cudaFuncGetAttributes(&a, k_bucket_scatter);
  cudaFuncGetAttributes(&a, k_bucket_sort_small);
  cudaFuncGetAttributes(&a, k_bucket_sort_large);
  cudaFuncGetAttributes(&a, k_bucket_compact);
}

}  // namespace grt
