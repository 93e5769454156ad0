// sweep.cu -- per-tile interference sweep (the analysis hot loop).
//
// One warp owns one tile at a time (tiles handed out by an atomic counter).
// The tile's candidates -- every (task, rectangle) overlapping it, in program
// order, each packed as task | privilege | rectangle clipped to the tile --
// are staged 32 at a time in shared memory with one coalesced 8-byte load per
// lane. Each cell of the tile keeps its run state in shared memory (16 bytes):
//
//   x = start position of the current run | kind << 30
//   y = position of its last member      | member count (1, 2, >=3) << 30
//   z = start position of the previous run | its member count << 30
//   w = position of the previous run's last member
//
// (positions index the tile's candidate list; a task's candidates are
// consecutive there, and its first one stands for the task). A task touching a
// cell either joins the current run (read after reads, reduce after reduces)
// and takes edges from the previous run, or starts a new run and takes edges
// from the current one. Runs of one or two members name them directly; longer
// runs are enumerated by re-reading the candidates between their first and
// last member (the ones covering the cell are exactly the members).
//
// Before sweeping a tile, its columns and rows are split into classes at the
// rectangle boundaries that fall inside it (a column class is a maximal run of
// columns no candidate's edge separates). Every cell of a class is covered by
// the same candidates, so the sweep runs on the class grid instead of the
// cells: a rectangle covering the whole tile costs one class, not tw x th
// cells, and the predecessor sets are the same.
//
// A class grid larger than the 1024 cells a warp keeps is swept in strips of
// class rows. Three ways to apply candidates (segment mode is chosen per tile,
// the other two per window of candidates):
//   * lane-parallel: small boxes whose overlaps chain at most 16 deep, one
//     candidate per lane, overlapping ones ordered by conflict levels;
//   * cell-parallel: the warp's lanes split the cells of one candidate's box;
//   * segment mode (tiles whose candidates cover 8+ class cells each on
//     average): each class row is kept as segments of equal run state, so a
//     candidate costs its rows' segments, not its cells. In 2-D tiles (row
//     mode) each lane takes whole class rows and runs a staged window's
//     candidates over them without waiting for the other lanes, and the
//     predecessors inside the window are bits of the window, OR-ed per task;
//     a task with more than 32 candidates in the tile (and 1-D tiles) takes
//     the rows of one candidate's box at a time, one lane per row.
// Predecessors found by several lanes are merged with match_any, and the
// survivors go through a per-warp shared-memory hash set, so each (src, dst)
// pair leaves the tile once per task. Pairs are appended to per-warp chunks of
// a global buffer (one atomic per chunk; a flush that does not fit continues
// in fresh chunks, so only a warp's last chunk keeps holes, filled with a
// sentinel key that the later sort moves to the end). A tile that drops pairs
// past the buffer's end is flagged with its pair count, for a rerun of just the
// flagged tiles.
// On dense inputs a pair is found again in every tile where the two tasks'
// rectangles meet; there the first sweep passes each flushed key through a
// direct-mapped table in global memory (one atomic exchange per key) and does
// not write a key the table already held. The table is lossy only towards
// keeping duplicates, which the CSR stage removes anyway; the rerun of flagged
// tiles sweeps without it.
#include <map>
#include <mutex>

#include "grt_internal.cuh"

namespace grt {

namespace {
constexpr int kHashSlots = 128;
constexpr int kListCap = 64;
constexpr int kLaneBuf = 16;     // predecessors one lane buffers in the lane-parallel path
constexpr int kSmallCells = 16;  // largest box the lane-parallel path takes
constexpr int kMaxRounds = 16;   // deeper conflict chains go to the warp-wide path
constexpr int kLongSpan = 64;    // run spans the whole warp scans together
constexpr int kSegMinArea = 8;   // mean class cells per candidate from which rows go segmented
constexpr int kExtSlots = 256;   // row mode: hash set of (predecessor, task) pairs from before the window
constexpr int kExtMax = 192;     // ... entries it takes before further pairs are written at once
constexpr int kExtProbes = 32;
constexpr unsigned kFull = 0xffffffffu;

// cells of the class grid one warp sweeps at once (taller grids go in strips)
__host__ __device__ inline int class_cap(int tw, int th) { return tw * th < kMaxClassCells ? tw * th : kMaxClassCells; }

// class maps: tw + th uint16 entries
__host__ __device__ inline size_t class_map_bytes(int tw, int th) { return (size_t)((2 * (tw + th) + 15) & ~15); }

// segment starts: one bit per class column, one row of words per class row
// swept at once (rows x words never exceed the class cells of a strip)
__host__ __device__ inline size_t seg_bytes(int tw, int th) {
  const int C = class_cap(tw, th), words = th * ((tw + 31) >> 5);
  return (size_t)((4 * (words < C ? words : C) + 15) & ~15);
}

// row mode's window tables (2-D tiles): class boxes and predecessor masks of
// the 32 staged candidates, and two column masks per class column
__host__ __device__ inline size_t row_table_bytes(int tw) {
  return tw <= kMaxTileSide2D ? (size_t)((32 * 4 * 2 + 8 * tw + 15) & ~15) : 0;
}

__host__ __device__ inline size_t per_warp_bytes(int tw, int th) {
  const int C = class_cap(tw, th);
  return (size_t)16 * C + (size_t)((C + 15) & ~15) + 32 * 8 + kHashSlots * 4 + kListCap * 8 + 16 +
         32 * kLaneBuf * 4 + class_map_bytes(tw, th) + seg_bytes(tw, th) + row_table_bytes(tw);  // 16-byte
                                                                       // multiple: warps' uint4 cells stay aligned
}

struct WarpSmem {
  uint4* cell;
  uint8_t* scr;
  uint64_t* stage;
  int* htab;
  int* hlist;
  int* hslot;
  int* hcount;
  int* lbuf;  // [32][kLaneBuf]
  uint16_t* cmx;  // column -> column class of the current tile
  uint16_t* cmy;  // row -> row class
  int* dropped;   // a pair of the current tile fell past the buffer's end
  int* npairs;    // pairs the current tile emitted
  uint32_t* seg;  // segment mode: per class row, bit x set where a segment starts
  // row mode (segment tiles in 2-D), per staged window:
  uint32_t* rbox;   // [32] candidate k's class box, x0 | x1 << 8 | y0 << 16 | y1 << 24
  uint32_t* rpred;  // [32] per task (its first candidate's index): window candidates it follows
  uint32_t* rlo;    // [class column x] bit k: candidate k's box starts at or left of x
  uint32_t* rhi;    // [class column x] bit k: candidate k's box ends at or right of x
  unsigned long long* xtab;  // [kExtSlots] (predecessor << 5 | task index) pairs from before the window
                            // (in the lane-parallel path's buffer)
  int* xcount;              // its entries
};

// in place: a[i] <- a[0] + ... + a[i] over a[0..L) (one warp, convergent)
__device__ void scan_flags(uint16_t* a, int L, int lane) {
  const int per = (L + 31) >> 5;
  const int b0 = min(lane * per, L), b1 = min(b0 + per, L);
  int sum = 0;
  for (int i = b0; i < b1; ++i) sum += a[i];
  int incl = sum;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int y = __shfl_up_sync(kFull, incl, o);
    if (lane >= o) incl += y;
  }
  int run = incl - sum;
  for (int i = b0; i < b1; ++i) {
    run += a[i];
    a[i] = (uint16_t)run;
  }
  __syncwarp();
}

struct Ctx {
  const uint64_t* L;  // the tile's candidates
  int n;              // number of candidates
  int pos;            // position of the staged window
  int cnt;            // entries in the window
  int tw, ndim;
  int ylo, yhi;       // the strip of class rows being swept
  bool segmode;       // rows kept as segments of equal state (large boxes)
  unsigned long long chunk_base;
  uint32_t chunk_left;
  int lane;
};

// A candidate's box in class coordinates. Within a tile, the columns (rows)
// are split into classes at every rectangle boundary that falls inside it;
// cells of one class are covered by exactly the same candidates, so their
// run states evolve identically and one cell per class stands for all.
// Rows are further clipped to the strip of class rows being swept, and
// renumbered from its first; a candidate outside the strip gets an empty box
// (x0 > x1, y0 > y1) that covers no cell. The overlap tests that order
// candidates may still pair an empty box with another; that only orders it
// more than needed.
__device__ __forceinline__ Box unpack_c(const Ctx& x, const WarpSmem& w, uint64_t p) {
  Box b = unpack_entry(p, x.ndim);
  b.x0 = w.cmx[b.x0];
  b.x1 = w.cmx[b.x1];
  int y0 = w.cmy[b.y0], y1 = w.cmy[b.y1];
  y0 = y0 > x.ylo ? y0 : x.ylo;
  y1 = y1 < x.yhi ? y1 : x.yhi;
  if (y0 > y1) {
    b.x0 = b.y0 = 1;
    b.x1 = b.y1 = 0;
  } else {
    b.y0 = y0 - x.ylo;
    b.y1 = y1 - x.ylo;
  }
  return b;
}

__device__ __forceinline__ void put_pair(const WarpSmem& w, const SweepOut& o, unsigned long long idx,
                                         uint64_t key) {
  if (idx < o.cap) {
    o.pairs[idx] = key;
  } else if (key != kEmpty64) {
    *w.dropped = 1;
  }
}

__device__ __forceinline__ uint64_t pair_key(int src, int dst, int key_bits) {
  return ((uint64_t)(uint32_t)src << key_bits) | (uint32_t)dst;
}

// the pair-key filter of dense inputs: the key takes its slot (multiplicative
// hashing by the 64-bit golden ratio); false when the slot already held it,
// i.e. some tile emitted this pair before (its write stands, or its tile was
// flagged for the rerun, which sweeps without the filter)
__device__ __forceinline__ bool filt_fresh(const SweepOut& o, uint64_t key) {
  const uint64_t h = (key * 0x9E3779B97F4A7C15ull) >> (64 - o.filt_bits);
  return atomicExch(o.filt + h, (unsigned long long)key) != (unsigned long long)key;
}

__device__ __forceinline__ uint64_t entry_at(const Ctx& x, const WarpSmem& w, int p) {
  int q = p - x.pos;
  return (q >= 0 && q < x.cnt) ? w.stage[q] : __ldg(x.L + p);
}

// lane-level insert (may run divergently)
__device__ void hash_insert(const WarpSmem& w, const SweepOut& o, int src, int dst) {
  if (*(volatile int*)w.hcount >= kListCap) {
    // the list is full: written at once, unfiltered (an exchange's round trip
    // per insert here cost more than the duplicates it saves)
    put_pair(w, o, atomicAdd(o.cursor, 1ull), pair_key(src, dst, o.key_bits));
    atomicAdd(w.npairs, 1);
    return;
  }
  uint32_t h = ((uint32_t)src * 2654435761u) >> 25;  // 7 bits -> 128 slots
  for (;;) {
    int old = atomicCAS(&w.htab[h], -1, src);
    if (old == -1) {
      int idx = atomicAdd(w.hcount, 1);
      if (idx < kListCap) {
        w.hlist[idx] = src;
        w.hslot[idx] = (int)h;
      } else {
        put_pair(w, o, atomicAdd(o.cursor, 1ull), pair_key(src, dst, o.key_bits));
        atomicAdd(w.npairs, 1);
      }
      return;
    }
    if (old == src) return;
    h = (h + 1) & (kHashSlots - 1);
  }
}

// warp-convergent insert: lanes holding the same predecessor elect one
__device__ __forceinline__ void warp_insert(const WarpSmem& w, const SweepOut& o, int src, int dst) {
  unsigned peers = __match_any_sync(kFull, src);
  if (src >= 0 && (peers & lanemask_lt()) == 0) hash_insert(w, o, src, dst);
}

// Where `need` pairs of one flush go: the first `split` fill the rest of the
// warp's current chunk (from `a`), the others start a fresh contiguous run of
// chunks (at `b`). Only a warp's last, partly used chunk is ever left with
// holes, so the cursor exceeds the pairs written by less than one chunk per
// warp (convergent).
struct PairDst {
  unsigned long long a, b;
  uint32_t split;
};

__device__ PairDst reserve_pairs(Ctx& x, const SweepOut& o, uint32_t need) {
  PairDst d{x.chunk_base, 0ull, need};
  if (x.chunk_left >= need) {
    x.chunk_base += need;
    x.chunk_left -= need;
    return d;
  }
  d.split = x.chunk_left;
  const uint32_t rest = need - x.chunk_left;
  const uint32_t k = (rest + o.chunk - 1) / o.chunk;
  unsigned long long nb = 0;
  if (x.lane == 0) nb = atomicAdd(o.cursor, (unsigned long long)k * o.chunk);
  d.b = __shfl_sync(kFull, nb, 0);
  x.chunk_base = d.b + rest;
  x.chunk_left = k * o.chunk - rest;
  return d;
}

__device__ __forceinline__ unsigned long long pair_pos(const PairDst& d, uint32_t i) {
  return i < d.split ? d.a + i : d.b + (i - d.split);
}

// writes the task's distinct predecessors found in this tile (convergent)
__device__ void flush(Ctx& x, const WarpSmem& w, const SweepOut& o, int dst) {
  __syncwarp();
  const int cnt = *(volatile int*)w.hcount;
  const int m = cnt < kListCap ? cnt : kListCap;
  if (m > 0 && o.filt) {
    // two list entries per lane (kListCap = 64); the keys the filter has seen
    // are dropped before the reservation, so the buffer only takes fresh ones
    static_assert(kListCap == 64, "two list entries per lane");
    const int i0 = x.lane, i1 = x.lane + 32;
    const uint64_t k0 = i0 < m ? pair_key(w.hlist[i0], dst, o.key_bits) : kEmpty64;
    const uint64_t k1 = i1 < m ? pair_key(w.hlist[i1], dst, o.key_bits) : kEmpty64;
    const bool f0 = i0 < m && filt_fresh(o, k0);
    const bool f1 = i1 < m && filt_fresh(o, k1);
    const unsigned b0 = __ballot_sync(kFull, f0), b1 = __ballot_sync(kFull, f1);
    const uint32_t n0 = (uint32_t)__popc(b0), total = n0 + (uint32_t)__popc(b1);
    // the tile's count bounds a rerun, which writes every pair: count them all
    if (x.lane == 0) atomicAdd(w.npairs, m);
    if (total > 0) {
      const PairDst pd = reserve_pairs(x, o, total);
      const unsigned lt = lanemask_lt();
      if (f0) put_pair(w, o, pair_pos(pd, (uint32_t)__popc(b0 & lt)), k0);
      if (f1) put_pair(w, o, pair_pos(pd, n0 + (uint32_t)__popc(b1 & lt)), k1);
    }
    if (cnt <= kListCap) {
      if (i0 < m) w.htab[w.hslot[i0]] = -1;
      if (i1 < m) w.htab[w.hslot[i1]] = -1;
    }
  } else if (m > 0) {
    const PairDst pd = reserve_pairs(x, o, (uint32_t)m);
    if (x.lane == 0) atomicAdd(w.npairs, m);
    for (int i = x.lane; i < m; i += 32) {
      put_pair(w, o, pair_pos(pd, (uint32_t)i), pair_key(w.hlist[i], dst, o.key_bits));
      if (cnt <= kListCap) w.htab[w.hslot[i]] = -1;
    }
  }
  if (cnt > kListCap)
    for (int i = x.lane; i < kHashSlots; i += 32) w.htab[i] = -1;
  __syncwarp();
  if (x.lane == 0) *w.hcount = 0;
  __syncwarp();
}

// One access at cell c by the task whose first candidate sits at `gpos`, with
// privilege pc: updates the cell's run state and returns the run whose members
// precede the access (first position rs, last position rl, member count rc:
// 0 none, 1, 2, 3 = three or more).
__device__ __forceinline__ void apply_cell(const WarpSmem& w, int c, int gpos, int pc, uint32_t& rs, uint32_t& rl,
                                           uint32_t& rc) {
  uint4 s = w.cell[c];
  const uint32_t ck = s.x >> 30;
  rs = rl = rc = 0;
  if (ck == (uint32_t)pc && pc != kKindWrite) {
    // join the current run: predecessors are the previous run
    rs = s.z & kPosMask;
    rl = s.w;
    rc = s.z >> 30;
    uint32_t cc = (s.y >> 30) + 1u;
    if (cc > 3u) cc = 3u;
    s.y = (uint32_t)gpos | (cc << 30);
  } else {
    // start a new run: predecessors are the current run
    if (ck != (uint32_t)kKindNone) {
      rs = s.x & kPosMask;
      rl = s.y & kPosMask;
      rc = s.y >> 30;
    }
    s.z = (s.x & kPosMask) | (rc << 30);
    s.w = s.y & kPosMask;
    s.x = (uint32_t)gpos | ((uint32_t)pc << 30);
    s.y = (uint32_t)gpos | (1u << 30);
  }
  w.cell[c] = s;
}

// Applies the access of the task whose first candidate sits at `gpos` to every
// cell of box [x0,x1]x[y0,y1] with privilege `p` (use_scr: per-cell privilege
// from the scratch bytes, consumed so a cell is applied once).
__device__ void sweep_box(Ctx& x, const WarpSmem& w, const SweepOut& o, int x0, int x1, int y0,
                          int y1, int gpos, int p, bool use_scr, int dst) {
  if (x1 < x0 || y1 < y0) return;  // a candidate outside the strip (warp-uniform)
  const int bw = x1 - x0 + 1, bh = y1 - y0 + 1;
  const int total = bw * bh;
  int qx = x.lane % bw, qy = x.lane / bw;
  const int dx = 32 % bw, dy = 32 / bw;
  const int iters = (total + 31) >> 5;
  for (int it = 0; it < iters; ++it) {
    bool act = it * 32 + x.lane < total;
    const int cx = x0 + qx, cy = y0 + qy;
    int c = 0, pc = p;
    if (act) {
      c = cy * x.tw + cx;
      if (use_scr) {
        uint32_t sv = w.scr[c];
        if (sv == 0xFFu) {
          act = false;
        } else {
          pc = (int)sv;
          w.scr[c] = 0xFFu;
        }
      }
    }
    int m1 = -1, m2 = -1;
    uint32_t rs = 0, rl = 0, rc = 0;
    if (act) {
      apply_cell(w, c, gpos, pc, rs, rl, rc);
      if (rc >= 1u) m1 = (int)(uint32_t)entry_at(x, w, (int)rs);
      if (rc >= 2u) m2 = (int)(uint32_t)entry_at(x, w, (int)rl);
    }
    warp_insert(w, o, m1, dst);
    warp_insert(w, o, m2, dst);
    // three or more members: the candidates strictly between the first and
    // the last member that cover the cell are the others. Short spans are
    // scanned by their own lane, all lanes at once; each long span is scanned
    // by the whole warp, 32 consecutive candidates per step.
    const bool longspan = act && rc == 3u && rl - rs > (uint32_t)kLongSpan;
    if (act && rc == 3u && !longspan) {
      for (uint32_t q = rs + 1; q < rl; ++q) {
        const Box b = unpack_c(x, w, entry_at(x, w, (int)q));
        if (b.x0 <= cx && cx <= b.x1 && b.y0 <= cy && cy <= b.y1) hash_insert(w, o, b.task, dst);
      }
    }
    unsigned need = __ballot_sync(kFull, longspan);
    while (need) {
      const int l = __ffs((int)need) - 1;
      need &= need - 1;
      const int qs = __shfl_sync(kFull, (int)rs, l) + 1, qe = __shfl_sync(kFull, (int)rl, l);
      const int lx = __shfl_sync(kFull, cx, l), ly = __shfl_sync(kFull, cy, l);
      for (int q0 = qs; q0 < qe; q0 += 32) {
        const int q = q0 + x.lane;
        if (q < qe) {
          const Box b = unpack_c(x, w, entry_at(x, w, q));
          if (b.x0 <= lx && lx <= b.x1 && b.y0 <= ly && ly <= b.y1) hash_insert(w, o, b.task, dst);
        }
      }
    }
    qx += dx;
    qy += dy;
    if (qx >= bw) {
      qx -= bw;
      qy += 1;
    }
  }
}

// the cells of a box, lane-strided; marks the combined privilege in scratch
__device__ void mark_box(const Ctx& x, const WarpSmem& w, const Box& b) {
  const int bw = b.x1 - b.x0 + 1, total = bw * (b.y1 - b.y0 + 1);
  for (int i = x.lane; i < total; i += 32) {
    int c = (b.y0 + i / bw) * x.tw + b.x0 + i % bw;
    w.scr[c] = (uint8_t)combine_priv(w.scr[c], (uint32_t)b.priv);
  }
}

// adds one predecessor to this lane's buffer (lane-parallel path)
__device__ __forceinline__ void lane_add(const WarpSmem& w, const SweepOut& o, int lane, int& nb, int src,
                                         int dst) {
  for (int k = 0; k < nb; ++k)
    if (w.lbuf[lane * kLaneBuf + k] == src) return;
  if (nb < kLaneBuf) {
    w.lbuf[lane * kLaneBuf + nb++] = src;
  } else {
    put_pair(w, o, atomicAdd(o.cursor, 1ull), pair_key(src, dst, o.key_bits));
    atomicAdd(w.npairs, 1);
  }
}

// Lane-parallel processing of a staged window whose candidates [0, end) are all
// small boxes: one candidate per lane. Candidates of different tasks whose
// boxes overlap are ordered by levels (a candidate runs one round after every
// earlier candidate it overlaps), so within a round lanes touch disjoint cells
// and each cell still sees its accesses in program order. A task's several
// candidates must be disjoint here (no privilege combination needed). Returns
// false (nothing done) when the window does not qualify.
__device__ bool stage_lanes(Ctx& x, const WarpSmem& w, const SweepOut& o, unsigned starts, int end) {
  const int lane = x.lane;
  const bool mine = lane < end;
  Box b = unpack_c(x, w, mine ? w.stage[lane] : 0ull);
  const int cells = mine ? (b.x1 - b.x0 + 1) * (b.y1 - b.y0 + 1) : 0;
  if (!__all_sync(kFull, cells <= kSmallCells)) return false;
  // position of this candidate's task (its group's first candidate)
  const unsigned upto = lane == 31 ? starts : (starts & ((2u << lane) - 1u));
  const int gpos = x.pos + (upto ? 31 - __clz((int)upto) : 0);
  int level = 0;
  bool bad = false;
  for (int j = 0; j < end; ++j) {
    const int x0 = __shfl_sync(kFull, b.x0, j), x1 = __shfl_sync(kFull, b.x1, j);
    const int y0 = __shfl_sync(kFull, b.y0, j), y1 = __shfl_sync(kFull, b.y1, j);
    const int tj = __shfl_sync(kFull, b.task, j), lj = __shfl_sync(kFull, level, j);
    if (mine && lane > j && b.x0 <= x1 && x0 <= b.x1 && b.y0 <= y1 && y0 <= b.y1) {
      if (tj == b.task) bad = true;
      else if (lj + 1 > level) level = lj + 1;
    }
  }
  if (__any_sync(kFull, bad)) return false;
  int maxl = level;
#pragma unroll
  for (int o2 = 16; o2 >= 1; o2 >>= 1) maxl = max(maxl, __shfl_xor_sync(kFull, maxl, o2));
  if (maxl >= kMaxRounds) return false;  // nothing applied yet: the warp-wide path takes the window
  // each lane runs in one round (its level) and buffers its candidate's
  // predecessors; the buffers are written out once, after the last round
  int nb = 0;
  for (int r = 0; r <= maxl; ++r) {
    if (mine && level == r) {
      const int bw = b.x1 - b.x0 + 1;
      for (int i = 0; i < cells; ++i) {
        const int cx = b.x0 + i % bw, cy = b.y0 + i / bw;
        uint32_t rs, rl, rc;
        apply_cell(w, cy * x.tw + cx, gpos, b.priv, rs, rl, rc);
        if (rc >= 1u) lane_add(w, o, lane, nb, (int)(uint32_t)entry_at(x, w, (int)rs), b.task);
        if (rc >= 2u) lane_add(w, o, lane, nb, (int)(uint32_t)entry_at(x, w, (int)rl), b.task);
        if (rc == 3u) {
          for (uint32_t q = rs + 1; q < rl; ++q) {
            Box e = unpack_c(x, w, entry_at(x, w, (int)q));
            if (e.x0 <= cx && cx <= e.x1 && e.y0 <= cy && cy <= e.y1) lane_add(w, o, lane, nb, e.task, b.task);
          }
        }
      }
    }
    __syncwarp();  // this level's cell updates before the next level reads them
  }
  // emit every lane's buffer into the warp's chunk (with the filter: only the
  // keys it has not seen)
  uint32_t fresh = nb > 0 ? (1u << nb) - 1u : 0u;
  if (o.filt) {
    fresh = 0u;
#pragma unroll
    for (int k = 0; k < kLaneBuf; ++k)
      if (k < nb && filt_fresh(o, pair_key(w.lbuf[lane * kLaneBuf + k], b.task, o.key_bits))) fresh |= 1u << k;
  }
  const int nf = __popc(fresh);
  int incl = nf;
#pragma unroll
  for (int o2 = 1; o2 < 32; o2 <<= 1) {
    const int y = __shfl_up_sync(kFull, incl, o2);
    if (lane >= o2) incl += y;
  }
  const int total = __shfl_sync(kFull, incl, 31);
  // the tile's count bounds a rerun, which writes every pair: count them all
  const int all = __reduce_add_sync(kFull, (unsigned)nb);
  if (lane == 0 && all) atomicAdd(w.npairs, all);
  if (total > 0) {
    const PairDst pd = reserve_pairs(x, o, (uint32_t)total);
    int pos = incl - nf;
    for (int k = 0; k < nb; ++k)
      if ((fresh >> k) & 1u)
        put_pair(w, o, pair_pos(pd, (uint32_t)pos++), pair_key(w.lbuf[lane * kLaneBuf + k], b.task, o.key_bits));
  }
  __syncwarp();
  return true;
}

// ---- segment mode ---------------------------------------------------------
// Tiles whose candidates cover many classes keep each class row as segments of
// equal run state: bit x of the row's mask is set where a segment starts, and
// only a segment's first cell holds the state (and the privilege mark). A
// candidate splits the segments at its box's edges, updates each covered
// segment once, and merges neighbours left equal. The previous-run fields of a
// state whose current run is a write are never read (nothing joins a write),
// so they are zeroed, which lets the segments a write covers merge. One lane
// owns one row of the box; predecessors of a segment are those of any of its
// cells (they share the state), and the members of a run of three or more are
// the candidates between its first and last member whose box meets the segment.

__device__ __forceinline__ int seg_start_le(const uint32_t* row, int X) {  // bit 0 is always set
  int k = X >> 5;
  uint32_t m = row[k] & (0xffffffffu >> (31 - (X & 31)));
  while (!m) m = row[--k];
  return (k << 5) + 31 - __clz((int)m);
}

__device__ __forceinline__ int seg_next(const uint32_t* row, int X, int cw) {  // first start > X, or cw
  if (X + 1 >= cw) return cw;
  int k = (X + 1) >> 5;
  const int W = (cw + 31) >> 5;
  uint32_t m = row[k] & (0xffffffffu << ((X + 1) & 31));
  while (!m) {
    if (++k >= W) return cw;
    m = row[k];
  }
  const int b = (k << 5) + __ffs((int)m) - 1;
  return b < cw ? b : cw;
}

__device__ __forceinline__ void seg_split(const Ctx& x, const WarpSmem& w, uint32_t* row, int y, int X) {
  if (X <= 0 || X >= x.tw) return;
  if (row[X >> 5] & (1u << (X & 31))) return;
  const int s0 = seg_start_le(row, X);
  w.cell[y * x.tw + X] = w.cell[y * x.tw + s0];
  w.scr[y * x.tw + X] = w.scr[y * x.tw + s0];
  row[X >> 5] |= 1u << (X & 31);
}

// merges the segments starting in [x0, x1 + 1] into their left neighbour when
// their state and mark equal it
__device__ void seg_merge(const Ctx& x, const WarpSmem& w, uint32_t* row, int y, int x0, int x1) {
  const int end = x1 + 1 < x.tw ? x1 + 1 : x.tw - 1;
  int prev = x0 > 0 ? seg_start_le(row, x0 - 1) : -1;
  for (int t = x0; t <= end; t = seg_next(row, t, x.tw)) {
    if (!(row[t >> 5] & (1u << (t & 31)))) continue;  // only when t == x0 is not a start (x0 == 0 case)
    if (prev >= 0) {
      const uint4 a = w.cell[y * x.tw + prev], b = w.cell[y * x.tw + t];
      if (a.x == b.x && a.y == b.y && a.z == b.z && a.w == b.w && w.scr[y * x.tw + prev] == w.scr[y * x.tw + t]) {
        row[t >> 5] &= ~(1u << (t & 31));
        continue;
      }
    }
    prev = t;
  }
}

// the access of the task whose first candidate is at `gpos` to the box's
// segments (use_scr: privileges from the marks, each segment applied once;
// the caller has split the rows already)
__device__ void seg_box(Ctx& x, const WarpSmem& w, const SweepOut& o, const Box& b, int gpos, int p, bool use_scr,
                        int dst) {
  if (b.x1 < b.x0 || b.y1 < b.y0) return;  // a candidate outside the strip (warp-uniform)
  const int W = (x.tw + 31) >> 5;
  for (int r0 = b.y0; r0 <= b.y1; r0 += 32) {
    const int y = r0 + x.lane;
    const bool rowact = y <= b.y1;
    uint32_t* row = w.seg + (rowact ? y : 0) * W;
    if (rowact && !use_scr) {
      seg_split(x, w, row, y, b.x0);
      seg_split(x, w, row, y, b.x1 + 1);
    }
    int sx = b.x0;
    bool more = rowact;
    while (__any_sync(kFull, more)) {
      int m1 = -1, m2 = -1, ex = 0;
      uint32_t rs = 0, rl = 0, rc = 0;
      bool act = false;
      if (more) {
        ex = seg_next(row, sx, x.tw) - 1;
        const int c = y * x.tw + sx;
        int pc = p;
        act = true;
        if (use_scr) {
          const uint32_t sv = w.scr[c];
          if (sv == 0xFFu) {
            act = false;
          } else {
            pc = (int)sv;
            w.scr[c] = 0xFFu;
          }
        }
        if (act) {
          apply_cell(w, c, gpos, pc, rs, rl, rc);
          if (pc == kKindWrite) {
            w.cell[c].z = 0u;
            w.cell[c].w = 0u;
          }
          if (rc >= 1u) m1 = (int)(uint32_t)entry_at(x, w, (int)rs);
          if (rc >= 2u) m2 = (int)(uint32_t)entry_at(x, w, (int)rl);
        }
      }
      warp_insert(w, o, m1, dst);
      warp_insert(w, o, m2, dst);
      const bool longspan = act && rc == 3u && rl - rs > (uint32_t)kLongSpan;
      if (act && rc == 3u && !longspan) {
        for (uint32_t q = rs + 1; q < rl; ++q) {
          const Box e = unpack_c(x, w, entry_at(x, w, (int)q));
          if (e.y0 <= y && y <= e.y1 && e.x0 <= ex && sx <= e.x1) hash_insert(w, o, e.task, dst);
        }
      }
      unsigned need = __ballot_sync(kFull, longspan);
      while (need) {
        const int l = __ffs((int)need) - 1;
        need &= need - 1;
        const int qs = __shfl_sync(kFull, (int)rs, l) + 1, qe = __shfl_sync(kFull, (int)rl, l);
        const int ly = __shfl_sync(kFull, y, l), lx0 = __shfl_sync(kFull, sx, l), lx1 = __shfl_sync(kFull, ex, l);
        for (int q0 = qs; q0 < qe; q0 += 32) {
          const int q = q0 + x.lane;
          if (q < qe) {
            const Box e = unpack_c(x, w, entry_at(x, w, q));
            if (e.y0 <= ly && ly <= e.y1 && e.x0 <= lx1 && lx0 <= e.x1) hash_insert(w, o, e.task, dst);
          }
        }
      }
      if (more) {
        sx = ex + 1;
        if (sx > b.x1) more = false;
      }
    }
    // a group's boxes merge only after all of them ran (their edges must stay)
    if (rowact && !use_scr) seg_merge(x, w, row, y, b.x0, b.x1);
    __syncwarp();
  }
}

// over the rows of box b: split at its edges (op 0), combine p into the marks
// of the segments it covers (op 1), or merge equal neighbours (op 2)
__device__ void seg_prepare(const Ctx& x, const WarpSmem& w, const Box& b, int p, int op) {
  if (b.x1 < b.x0 || b.y1 < b.y0) return;
  const int W = (x.tw + 31) >> 5;
  for (int y = b.y0 + x.lane; y <= b.y1; y += 32) {
    uint32_t* row = w.seg + y * W;
    if (op == 0) {
      seg_split(x, w, row, y, b.x0);
      seg_split(x, w, row, y, b.x1 + 1);
    } else if (op == 2) {
      seg_merge(x, w, row, y, b.x0, b.x1);
    } else {
      for (int t = b.x0; t <= b.x1; t = seg_next(row, t, x.tw)) {
        const int c = y * x.tw + t;
        w.scr[c] = (uint8_t)combine_priv(w.scr[c], (uint32_t)p);
      }
    }
  }
  __syncwarp();
}

// one task's candidates at positions [a, b), segment mode
__device__ void process_group_seg(Ctx& x, const WarpSmem& w, const SweepOut& o, int a, int b) {
  const uint64_t first = entry_at(x, w, a);
  const int dst = (int)(uint32_t)first;
  if (b - a == 1) {
    const Box bx = unpack_c(x, w, first);
    seg_box(x, w, o, bx, a, bx.priv, false, dst);
  } else {
    // all edges first, so every segment is wholly inside or outside each box;
    // then one combined privilege per segment, applied once
    for (int e = a; e < b; ++e) seg_prepare(x, w, unpack_c(x, w, entry_at(x, w, e)), 0, 0);
    for (int e = a; e < b; ++e) {
      const Box bx = unpack_c(x, w, entry_at(x, w, e));
      seg_prepare(x, w, bx, bx.priv, 1);
    }
    for (int e = a; e < b; ++e) seg_box(x, w, o, unpack_c(x, w, entry_at(x, w, e)), a, 0, true, dst);
    for (int e = a; e < b; ++e) seg_prepare(x, w, unpack_c(x, w, entry_at(x, w, e)), 0, 2);
  }
  flush(x, w, o, dst);
}

// ---- row mode ----------------------------------------------------------------
// In a segment tile the cells of different class rows never interact, so a lane
// can take whole class rows and run every candidate of a staged window over its
// rows in program order, without waiting for the other lanes between
// candidates (the segment path above runs one candidate at a time, one lane per
// row of its box). A predecessor inside the window is recorded as a bit of the
// window: a run's first and last members by their own positions, the members
// between them (runs of three or more) as the window's candidates that cover
// the row, overlap the segment and lie between the two. Each lane ORs its bits
// into the task's mask in shared memory; the masks become pairs once per
// window. Members from before the window (the runs a window's first accesses
// meet) go through a per-warp hash set of (predecessor, task) keys.

__device__ __forceinline__ uint32_t pack_cbox(const Box& b) {
  return (uint32_t)b.x0 | ((uint32_t)b.x1 << 8) | ((uint32_t)b.y0 << 16) | ((uint32_t)b.y1 << 24);
}

// (src, window task j) into the warp's set; once the set is full (or a key
// finds no slot within kExtProbes) the pair is written at once, through the
// pair-key filter on dense inputs (lane-level, may run divergently)
__device__ __forceinline__ void ext_add(const WarpSmem& w, const SweepOut& o, int src, int j, int dst) {
  // the tile's count bounds a rerun, which writes every pair: each call writes
  // at most one (in the set or at once), whatever order the lanes reach the
  // set in, so every call is counted
  atomicAdd(w.npairs, 1);
  const unsigned long long key = ((unsigned long long)(uint32_t)src << 5) | (unsigned long long)(uint32_t)j;
  if (*(volatile int*)w.xcount < kExtMax) {
    uint32_t h = (uint32_t)((key * 0x9E3779B97F4A7C15ull) >> 56);  // 8 bits: kExtSlots
    for (int t = 0; t < kExtProbes; ++t) {
      const unsigned long long old = atomicCAS(w.xtab + h, (unsigned long long)kEmpty64, key);
      if (old == key) return;
      if (old == (unsigned long long)kEmpty64) {
        atomicAdd(w.xcount, 1);
        return;
      }
      h = (h + 1) & (kExtSlots - 1);
    }
  }
  const uint64_t pk = pair_key(src, dst, o.key_bits);
  if (!o.filt || filt_fresh(o, pk)) put_pair(w, o, atomicAdd(o.cursor, 1ull), pk);
}

// The access with privilege pk of window task j (first candidate at window
// index j, task id dst) to segment [sx, ex] of class row y: updates the state
// and records the members of the run it follows (window ones as bits of acc).
// cover: the window candidates whose box holds row y.
__device__ __forceinline__ void row_seg(const Ctx& x, const WarpSmem& w, const SweepOut& o, int y, int sx, int ex,
                                        int pk, int j, unsigned cover, unsigned& acc, int dst) {
  const int c = y * x.tw + sx;
  uint32_t rs, rl, rc;
  apply_cell(w, c, x.pos + j, pk, rs, rl, rc);
  if (pk == kKindWrite) {
    w.cell[c].z = 0u;
    w.cell[c].w = 0u;
  }
  if (rc == 0u) return;
  const int pos = x.pos;
  // members in the window: the first and the last by their positions, the
  // ones strictly between them (runs of three or more) as the candidates that
  // cover row y, overlap the segment and lie between the two (rl precedes
  // this task, so rl - pos <= 30)
  if ((int)rs >= pos) acc |= 1u << ((int)rs - pos);
  if (rc >= 2u && (int)rl >= pos) acc |= 1u << ((int)rl - pos);
  if (rc == 3u) {
    const int a = (int)rs + 1 > pos ? (int)rs + 1 : pos, b = (int)rl - 1;
    if (b >= a) acc |= ((2u << (b - pos)) - 1u) & ~((1u << (a - pos)) - 1u) & cover & w.rlo[ex] & w.rhi[sx];
  }
  if ((int)rs >= pos) return;
  // members from before the window, in one pass: the first, the candidates
  // strictly between the first and the last that meet the segment (runs of
  // three or more), then the last
  const int last = (rc >= 2u && (int)rl < pos) ? (int)rl : -1;
  const int qe = rc == 3u ? ((int)rl < pos ? (int)rl : pos) : (int)rs + 1;  // end of the scan
  for (int q = (int)rs;;) {
    int src = -1;
    if (q == (int)rs || q == last) {
      src = (int)(uint32_t)entry_at(x, w, q);
    } else {
      const Box e = unpack_c(x, w, entry_at(x, w, q));
      if (e.y0 <= y && y <= e.y1 && e.x0 <= ex && sx <= e.x1) src = e.task;
    }
    if (src >= 0) ext_add(w, o, src, j, dst);
    if (q + 1 < qe) ++q;
    else if (q < last) q = last;
    else break;
  }
}

// privilege of window candidate k from the window's privilege planes
__device__ __forceinline__ int row_priv(unsigned wp, unsigned dp, int k) {
  return ((wp >> k) & 1u) ? kKindWrite : (((dp >> k) & 1u) ? kKindReduce : kKindRead);
}

// Segment starts of one row for row mode: in shared memory, or (ONE: class
// width up to 32) one word held in a register by the row's lane.
template <bool ONE>
struct RowSeg;

template <>
struct RowSeg<false> {
  static __device__ __forceinline__ void split(const Ctx& x, const WarpSmem& w, uint32_t* row, uint32_t&, int y,
                                               int X) {
    seg_split(x, w, row, y, X);
  }
  static __device__ __forceinline__ int next(const uint32_t* row, uint32_t, int X, int cw) {
    return seg_next(row, X, cw);
  }
  static __device__ __forceinline__ void merge(const Ctx& x, const WarpSmem& w, uint32_t* row, uint32_t&, int y,
                                               int x0, int x1) {
    seg_merge(x, w, row, y, x0, x1);
  }
};

template <>
struct RowSeg<true> {
  static __device__ __forceinline__ int start_le(uint32_t m, int X) {  // X <= 31; bit 0 is always set
    return 31 - __clz((int)(m & ((2u << X) - 1u)));
  }
  static __device__ __forceinline__ int next(const uint32_t*, uint32_t m, int X, int cw) {  // first start > X, or cw
    const uint32_t r = m & ~((2u << X) - 1u);
    const int b = r ? __ffs((int)r) - 1 : cw;
    return b < cw ? b : cw;
  }
  static __device__ __forceinline__ void split(const Ctx& x, const WarpSmem& w, uint32_t*, uint32_t& m, int y,
                                               int X) {
    if (X <= 0 || X >= x.tw || ((m >> X) & 1u)) return;
    const int s0 = start_le(m, X);
    w.cell[y * x.tw + X] = w.cell[y * x.tw + s0];
    w.scr[y * x.tw + X] = w.scr[y * x.tw + s0];
    m |= 1u << X;
  }
  static __device__ __forceinline__ void merge(const Ctx& x, const WarpSmem& w, uint32_t*, uint32_t& m, int y,
                                               int x0, int x1) {
    const int end = x1 + 1 < x.tw ? x1 + 1 : x.tw - 1;
    int prev = x0 > 0 ? start_le(m, x0 - 1) : -1;
    for (int t = x0; t <= end; t = next(nullptr, m, t, x.tw)) {
      if (!((m >> t) & 1u)) continue;
      if (prev >= 0) {
        const uint4 a = w.cell[y * x.tw + prev], b = w.cell[y * x.tw + t];
        if (a.x == b.x && a.y == b.y && a.z == b.z && a.w == b.w && w.scr[y * x.tw + prev] == w.scr[y * x.tw + t]) {
          m &= ~(1u << t);
          continue;
        }
      }
      prev = t;
    }
  }
};

// one class row y of a row-mode window: every staged candidate that holds the
// row, in program order (ONE: the row's segment starts fit one word, kept in
// a register for the window)
template <bool ONE>
__device__ __forceinline__ void row_pass(const Ctx& x, const WarpSmem& w, const SweepOut& o, int y, unsigned starts,
                                         int end, unsigned wp, unsigned dp) {
  uint32_t* row = w.seg + y * ((x.tw + 31) >> 5);
  uint32_t m = ONE ? row[0] : 0u;
  unsigned cover = 0u;
  for (int k = 0; k < end; ++k) {
    const uint32_t bx = w.rbox[k];
    if ((int)((bx >> 16) & 255u) <= y && y <= (int)(bx >> 24)) cover |= 1u << k;
  }
  for (unsigned tm = cover; tm;) {
    const int k = __ffs((int)tm) - 1;
    // k's task: its first candidate j and the window bits G of its candidates
    const unsigned upto = starts & ((2u << k) - 1u), later = starts & ~((2u << k) - 1u);
    const int j = 31 - __clz((int)upto);
    const unsigned G = (later ? (1u << (__ffs((int)later) - 1)) - 1u : kFull) & ~((1u << j) - 1u);
    const unsigned K = tm & G;  // its candidates on this row
    tm &= ~G;
    const int dst = (int)(uint32_t)w.stage[j];
    // split at the edges of the task's candidates on this row, then run each
    // segment of their union once, with the privileges of the candidates
    // holding it combined (one candidate: its own)
    unsigned acc = 0u;
    int u0 = 1 << 30, u1 = -1;
    for (unsigned kk = K; kk; kk &= kk - 1u) {
      const uint32_t bx = w.rbox[__ffs((int)kk) - 1];
      const int x0 = (int)(bx & 255u), x1 = (int)((bx >> 8) & 255u);
      RowSeg<ONE>::split(x, w, row, m, y, x0);
      RowSeg<ONE>::split(x, w, row, m, y, x1 + 1);
      u0 = x0 < u0 ? x0 : u0;
      u1 = x1 > u1 ? x1 : u1;
    }
    for (int sx = u0; sx <= u1;) {
      const int ex = RowSeg<ONE>::next(row, m, sx, x.tw) - 1;
      uint32_t pk = 0xFFu;
      for (unsigned kk = K; kk; kk &= kk - 1u) {
        const int q = __ffs((int)kk) - 1;
        const uint32_t bx = w.rbox[q];
        if ((int)(bx & 255u) <= sx && sx <= (int)((bx >> 8) & 255u)) pk = combine_priv(pk, (uint32_t)row_priv(wp, dp, q));
      }
      if (pk != 0xFFu) row_seg(x, w, o, y, sx, ex, (int)pk, j, cover, acc, dst);
      sx = ex + 1;
    }
    RowSeg<ONE>::merge(x, w, row, m, y, u0, u1);
    if (acc) atomicOr(w.rpred + j, acc);
  }
  if (ONE) row[0] = m;
}

// Row mode over the staged window's candidates [0, end) (whole tasks; bit k of
// starts: candidate k is its task's first) in a segment tile (convergent).
__device__ void row_window(Ctx& x, const WarpSmem& w, const SweepOut& o, unsigned starts, int end) {
  const int lane = x.lane;
  const bool mine = lane < end;
  Box b;
  b.x0 = b.y0 = 1;
  b.x1 = b.y1 = 0;
  b.priv = kKindRead;
  if (mine) b = unpack_c(x, w, w.stage[lane]);
  w.rbox[lane] = pack_cbox(b);
  w.rpred[lane] = 0u;
  const unsigned wp = __ballot_sync(kFull, mine && b.priv == kKindWrite);
  const unsigned dp = __ballot_sync(kFull, mine && b.priv == kKindReduce);
  const bool live = mine && b.x0 <= b.x1 && b.y0 <= b.y1;
  for (int cx = 0; cx < x.tw; ++cx) {
    const unsigned lo = __ballot_sync(kFull, live && b.x0 <= cx);
    const unsigned hi = __ballot_sync(kFull, live && b.x1 >= cx);
    if (lane == 0) {
      w.rlo[cx] = lo;
      w.rhi[cx] = hi;
    }
  }
  __syncwarp();
  const int rows = x.yhi - x.ylo + 1, W = (x.tw + 31) >> 5;
  for (int y = lane; y < rows; y += 32) {
    if (W == 1) row_pass<true>(x, w, o, y, starts, end, wp, dp);
    else row_pass<false>(x, w, o, y, starts, end, wp, dp);
  }
  __syncwarp();

  // pairs: lane j (a task's first candidate) turns its mask into the tasks it
  // follows; lane l takes the set's slots l, l + 32, ...
  const bool lead = mine && ((starts >> lane) & 1u);
  const unsigned P = lead ? w.rpred[lane] : 0u;
  const int dst = lead ? (int)(uint32_t)w.stage[lane] : 0;
  unsigned src = 0u;  // first candidates of the tasks this one follows
  for (unsigned r = P; r;) {
    const int q = 31 - __clz((int)r);
    const int g = 31 - __clz((int)(starts & ((2u << q) - 1u)));
    src |= 1u << g;
    r &= (1u << g) - 1u;
  }
  const bool any_ext = *(volatile int*)w.xcount > 0;
  constexpr int kPer = kExtSlots / 32;
  unsigned fresh = src, xfresh = 0u;  // xfresh bit i: slot lane + 32 i holds a pair to write
  if (any_ext) {
#pragma unroll
    for (int i = 0; i < kPer; ++i) {
      const unsigned long long e = w.xtab[lane + 32 * i];
      if (e != (unsigned long long)kEmpty64) {
        if (!o.filt || filt_fresh(o, pair_key((int)(uint32_t)(e >> 5), (int)(uint32_t)w.stage[e & 31u], o.key_bits)))
          xfresh |= 1u << i;
      }
    }
  }
  if (o.filt) {
    fresh = 0u;
    for (unsigned r = src; r; r &= r - 1u) {
      const int g = __ffs((int)r) - 1;
      if (filt_fresh(o, pair_key((int)(uint32_t)w.stage[g], dst, o.key_bits))) fresh |= 1u << g;
    }
  }
  // the tile's count bounds a rerun, which writes every pair: the window's own
  // (the set's were counted as they were added)
  const unsigned all = __reduce_add_sync(kFull, (unsigned)__popc(src));
  if (lane == 0 && all) atomicAdd(w.npairs, (int)all);
  const int mine_n = __popc(fresh) + __popc(xfresh);
  int incl = mine_n;
#pragma unroll
  for (int o2 = 1; o2 < 32; o2 <<= 1) {
    const int t = __shfl_up_sync(kFull, incl, o2);
    if (lane >= o2) incl += t;
  }
  const int total = __shfl_sync(kFull, incl, 31);
  if (total > 0) {
    const PairDst pd = reserve_pairs(x, o, (uint32_t)total);
    uint32_t at = (uint32_t)(incl - mine_n);
    for (unsigned r = fresh; r; r &= r - 1u)
      put_pair(w, o, pair_pos(pd, at++), pair_key((int)(uint32_t)w.stage[__ffs((int)r) - 1], dst, o.key_bits));
    for (unsigned r = xfresh; r; r &= r - 1u) {
      const unsigned long long e = w.xtab[lane + 32 * (__ffs((int)r) - 1)];
      put_pair(w, o, pair_pos(pd, at++), pair_key((int)(uint32_t)(e >> 5), (int)(uint32_t)w.stage[e & 31u], o.key_bits));
    }
  }
  if (any_ext) {
    __syncwarp();
#pragma unroll
    for (int i = 0; i < kPer; ++i) w.xtab[lane + 32 * i] = (unsigned long long)kEmpty64;
  }
  __syncwarp();
  if (lane == 0) *w.xcount = 0;
  __syncwarp();
}

// one task's candidates at positions [a, b) of the tile list
__device__ void process_group(Ctx& x, const WarpSmem& w, const SweepOut& o, int a, int b) {
  const uint64_t first = entry_at(x, w, a);
  const int dst = (int)(uint32_t)first;
  const int g = b - a;
  if (g == 1) {
    Box bx = unpack_c(x, w, first);
    sweep_box(x, w, o, bx.x0, bx.x1, bx.y0, bx.y1, a, bx.priv, false, dst);
  } else {
    // disjoint rectangles need no privilege combination
    bool overlap = g > 32;
    if (!overlap) {
      bool mine = false;
      if (x.lane < g) {
        Box bi = unpack_c(x, w, entry_at(x, w, a + x.lane));
        for (int j = x.lane + 1; j < g; ++j) {
          Box bj = unpack_c(x, w, entry_at(x, w, a + j));
          if (bi.x0 <= bj.x1 && bj.x0 <= bi.x1 && bi.y0 <= bj.y1 && bj.y0 <= bi.y1) mine = true;
        }
      }
      overlap = __any_sync(kFull, mine);
    }
    if (!overlap) {
      for (int e = a; e < b; ++e) {
        Box bx = unpack_c(x, w, entry_at(x, w, e));
        sweep_box(x, w, o, bx.x0, bx.x1, bx.y0, bx.y1, a, bx.priv, false, dst);
      }
    } else {
      for (int e = a; e < b; ++e) {
        mark_box(x, w, unpack_c(x, w, entry_at(x, w, e)));
        __syncwarp();
      }
      for (int e = a; e < b; ++e) {
        Box bx = unpack_c(x, w, entry_at(x, w, e));
        sweep_box(x, w, o, bx.x0, bx.x1, bx.y0, bx.y1, a, 0, true, dst);
        __syncwarp();
      }
    }
  }
  flush(x, w, o, dst);
}

__global__ void __launch_bounds__(256, 3) k_sweep(const uint64_t* __restrict__ payload,
                                               const uint32_t* __restrict__ seg_begin,
                                               const uint32_t* __restrict__ seg_end, AnalysisDims d,
                                               SweepOut o) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int C = class_cap(d.tw, d.th);
  unsigned char* base = smem + (size_t)warp * per_warp_bytes(d.tw, d.th);
  WarpSmem w;
  w.cell = reinterpret_cast<uint4*>(base);
  w.scr = base + 16 * C;
  w.stage = reinterpret_cast<uint64_t*>(base + 16 * C + ((C + 15) & ~15));
  w.htab = reinterpret_cast<int*>(w.stage + 32);
  w.hlist = w.htab + kHashSlots;
  w.hslot = w.hlist + kListCap;
  w.hcount = w.hslot + kListCap;
  w.lbuf = w.hcount + 4;
  w.cmx = reinterpret_cast<uint16_t*>(w.lbuf + 32 * kLaneBuf);
  w.cmy = w.cmx + d.tw;
  w.seg = reinterpret_cast<uint32_t*>(reinterpret_cast<unsigned char*>(w.cmx) + class_map_bytes(d.tw, d.th));
  w.rbox = reinterpret_cast<uint32_t*>(reinterpret_cast<unsigned char*>(w.seg) + seg_bytes(d.tw, d.th));
  w.rpred = w.rbox + 32;
  w.rlo = w.rpred + 32;
  w.rhi = w.rlo + d.tw;
  static_assert(kExtSlots * 8 <= 32 * kLaneBuf * 4, "the set fits the lane-parallel path's buffer");
  w.xtab = reinterpret_cast<unsigned long long*>(w.lbuf);
  w.dropped = w.hcount + 1;
  w.npairs = w.hcount + 2;
  w.xcount = w.hcount + 3;
  // row mode runs in 2-D segment tiles, whose class columns the tables cover
  const bool rowmode = d.ndim == 2 && row_table_bytes(d.tw) > 0;
  for (int i = lane; i < kHashSlots; i += 32) w.htab[i] = -1;
  if (lane == 0) {
    *w.hcount = 0;
    *w.dropped = 0;
    *w.npairs = 0;
    *w.xcount = 0;
  }
  __syncwarp();

  Ctx x;
  x.tw = d.tw;
  x.ndim = d.ndim;
  x.chunk_base = 0;
  x.chunk_left = 0;
  x.lane = lane;
  const int ntiles = d.ntx * d.nty;
  for (;;) {
    int t = 0;
    if (lane == 0) t = (int)atomicAdd(o.tile_counter, 1u);
    t = __shfl_sync(kFull, t, 0);
    if (t >= ntiles) break;
    const uint32_t sb = seg_begin[t], se = seg_end[t];
    if (sb >= se) continue;
    if (o.only && !o.only[t]) continue;  // a rerun sweeps the tiles that dropped pairs
    x.L = payload + sb;
    x.n = (int)(se - sb);
    // class maps of this tile: mark every rectangle boundary inside it, then
    // number the classes by a prefix sum
    for (int i = lane; i < d.tw; i += 32) w.cmx[i] = 0;
    for (int i = lane; i < d.th; i += 32) w.cmy[i] = 0;
    __syncwarp();
    for (int k = lane; k < x.n; k += 32) {
      const Box b = unpack_entry(x.L[k], x.ndim);
      if (b.x0 > 0) w.cmx[b.x0] = 1;
      if (b.x1 + 1 < d.tw) w.cmx[b.x1 + 1] = 1;
      if (b.y0 > 0) w.cmy[b.y0] = 1;
      if (b.y1 + 1 < d.th) w.cmy[b.y1 + 1] = 1;
    }
    __syncwarp();
    scan_flags(w.cmx, d.tw, lane);
    scan_flags(w.cmy, d.th, lane);
    const int cw = w.cmx[d.tw - 1] + 1, ch = w.cmy[d.th - 1] + 1;
    x.tw = cw;  // row stride of the class grid
    // segment mode when the candidates cover many classes each
    unsigned long long area = 0;
    for (int k = lane; k < x.n; k += 32) {
      const Box b = unpack_entry(x.L[k], x.ndim);
      area += (unsigned long long)(w.cmx[b.x1] - w.cmx[b.x0] + 1) * (unsigned long long)(w.cmy[b.y1] - w.cmy[b.y0] + 1);
    }
#pragma unroll
    for (int o2 = 16; o2 >= 1; o2 >>= 1) area += __shfl_xor_sync(kFull, area, o2);
    x.segmode = area >= (unsigned long long)kSegMinArea * (unsigned long long)x.n;
    // a class grid larger than the cell state is swept in strips of class
    // rows, each pass over every candidate (those outside see empty boxes)
    const int cap = class_cap(d.tw, d.th);
    const int strip = cw * ch <= cap ? ch : cap / cw;
    for (x.ylo = 0; x.ylo < ch; x.ylo += strip) {
      x.yhi = min(x.ylo + strip, ch) - 1;
      const int rows = x.yhi - x.ylo + 1;
      if (x.segmode) {
        const int W = (cw + 31) >> 5;
        for (int i = lane; i < rows * W; i += 32) w.seg[i] = (i % W == 0) ? 1u : 0u;
        for (int y = lane; y < rows; y += 32) {
          w.cell[y * cw] = make_uint4((uint32_t)kKindNone << 30, 0u, 0u, 0u);
          w.scr[y * cw] = 0xFFu;
        }
        // row mode's set shares its memory with the lane-parallel path's buffers
        if (rowmode)
          for (int i = lane; i < kExtSlots; i += 32) w.xtab[i] = (unsigned long long)kEmpty64;
      } else {
        for (int c = lane; c < cw * rows; c += 32) {
          w.cell[c] = make_uint4((uint32_t)kKindNone << 30, 0u, 0u, 0u);
          w.scr[c] = 0xFFu;
        }
      }
      __syncwarp();
      int pos = 0;
      while (pos < x.n) {
        const int cnt = x.n - pos < 32 ? x.n - pos : 32;
        const uint64_t my = lane < cnt ? x.L[pos + lane] : kEmpty64;
        w.stage[lane] = my;
        const uint64_t nxt = (pos + 32 < x.n) ? x.L[pos + 32] : kEmpty64;
        x.pos = pos;
        x.cnt = cnt;
        __syncwarp();
        const int mytask = (int)(uint32_t)my;
        const int prevtask = __shfl_up_sync(kFull, mytask, 1);
        const bool start = lane < cnt && (lane == 0 || mytask != prevtask);
        const unsigned starts = __ballot_sync(kFull, start);
        const int lasttask = __shfl_sync(kFull, mytask, cnt - 1);
        const bool last_complete = (pos + cnt == x.n) || ((int)(uint32_t)nxt != lasttask);
        const int last_start = 31 - __clz((int)starts);
        const int end = last_complete ? cnt : last_start;
        if (end == 0) {
          // one task with more than 32 candidates in this tile: find its end
          int gend = pos + 32;
          for (;;) {
            int idx = gend + lane;
            int tk = idx < x.n ? (int)(uint32_t)x.L[idx] : -2;
            unsigned diff = __ballot_sync(kFull, tk != lasttask);
            if (diff) {
              gend += __ffs((int)diff) - 1;
              break;
            }
            gend += 32;
          }
          if (x.segmode) {
            process_group_seg(x, w, o, pos, gend);
          } else {
            process_group(x, w, o, pos, gend);
          }
          pos = gend;
          __syncwarp();
          continue;
        }
        unsigned gs = starts & (end == 32 ? kFull : ((1u << end) - 1u));
        if (x.segmode && rowmode) {
          row_window(x, w, o, gs, end);
          gs = 0;
        } else if (!x.segmode && stage_lanes(x, w, o, gs, end)) {
          gs = 0;
        }
        while (gs) {
          const int a = __ffs((int)gs) - 1;
          gs &= gs - 1;
          const int b = gs ? __ffs((int)gs) - 1 : end;
          if (x.segmode) {
            process_group_seg(x, w, o, pos + a, pos + b);
          } else {
            process_group(x, w, o, pos + a, pos + b);
          }
        }
        pos += end;
        __syncwarp();
      }
    }
    // a tile that dropped a pair is marked for the rerun, with its pair count
    __syncwarp();
    if (lane == 0) {
      if (*(volatile int*)w.dropped) {
        if (o.flag_out) o.flag_out[t] = 1;
        atomicAdd(o.rerun, (unsigned long long)*(volatile int*)w.npairs);
      }
      *w.dropped = 0;
      *w.npairs = 0;
    }
    __syncwarp();
  }
  for (uint32_t i = lane; i < x.chunk_left; i += 32) put_pair(w, o, x.chunk_base + i, kEmpty64);
}
}  // namespace

int sweep_warps_per_block(int tw, int th) {
  // three blocks per SM (the kernel's launch bounds): 228 KB of shared memory,
  // less 1 KB the hardware keeps per block, is 75 KB a block
  int w = (int)((75 * 1024) / per_warp_bytes(tw, th));
  return w < 1 ? 1 : (w > 8 ? 8 : w);
}

size_t sweep_smem_bytes(int tw, int th, int warps) { return per_warp_bytes(tw, th) * warps; }

void launch_sweep(const uint64_t* payload, const uint32_t* seg_begin, const uint32_t* seg_end,
                  AnalysisDims d, SweepOut o, int blocks, cudaStream_t s) {
  const int warps = sweep_warps_per_block(d.tw, d.th);
  const size_t bytes = sweep_smem_bytes(d.tw, d.th, warps);
  // The shared-memory limit is one attribute of the kernel per device, shared
  // by every thread of the process. It only ever grows, under a lock, so an
  // analysis on another thread with a smaller tile never lowers it below what
  // a launch in flight here needs.
  {
    static std::mutex mu;
    static std::map<int, size_t> limit;
    int dev = 0;
    cudaGetDevice(&dev);
    std::lock_guard<std::mutex> lk(mu);
    size_t& cur = limit[dev];
    if (bytes > cur) {
      cudaFuncSetAttribute(k_sweep, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
      cur = bytes;
    }
  }
  count_launch();
  k_sweep<<<blocks, warps * 32, bytes, s>>>(payload, seg_begin, seg_end, d, o);
}

void preload_sweep() {
  cudaFuncAttributes a;
  cudaFuncGetAttributes(&a, k_sweep);
}

}  // namespace grt
