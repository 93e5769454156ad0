// primitives.cu -- device exclusive scan and stable LSD radix sort.
//
// Scan: reduce-then-scan over blocks of 2048 items (256 threads x 8), the
// block totals scanned recursively. out[n] receives the total, so arrays are
// sized n+1; in == out is allowed.
//
// Radix sort: 8-bit digits, least significant first. Per pass: a per-block
// digit histogram, an exclusive scan of the digit-major histogram matrix, and
// a scatter whose in-block ranks are computed warp by warp with match_any (so
// the sort is stable: keys keep their input order within a digit); the block
// reorders its keys by digit in shared memory before writing them, so each
// digit's run goes out in coalesced writes.

#include <mutex>
#include <set>

#include "grt_internal.cuh"

namespace grt {

std::atomic<long long> g_kernel_launches{0};

namespace {
constexpr int kScanThreads = 256;
constexpr int kScanItems = 8;
constexpr int kScanTile = kScanThreads * kScanItems;

template <typename T>
__device__ T block_exclusive_sum(T v, T* warp_tot, T* block_total) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  T incl = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    T y = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += y;
  }
  if (lane == 31) warp_tot[warp] = incl;
  __syncthreads();
  if (warp == 0) {
    T w = lane < (kScanThreads / 32) ? warp_tot[lane] : T(0);
    T wi = w;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      T y = __shfl_up_sync(0xffffffffu, wi, o);
      if (lane >= o) wi += y;
    }
    if (lane < (kScanThreads / 32)) warp_tot[lane] = wi - w;
    if (lane == (kScanThreads / 32) - 1) *block_total = wi;
  }
  __syncthreads();
  return incl - v + warp_tot[warp];
}

template <typename T>
__global__ void __launch_bounds__(kScanThreads) k_scan_reduce(const T* in, int64_t n, T* partial) {
  __shared__ T warp_tot[32];
  __shared__ T tot;
  const int64_t base = (int64_t)blockIdx.x * kScanTile;
  T s = 0;
#pragma unroll
  for (int j = 0; j < kScanItems; ++j) {
    int64_t k = base + j * kScanThreads + threadIdx.x;  // coalesced
    if (k < n) s += in[k];
  }
  (void)block_exclusive_sum<T>(s, warp_tot, &tot);
  if (threadIdx.x == 0) partial[blockIdx.x] = tot;
}

template <typename T>
__global__ void __launch_bounds__(kScanThreads) k_scan_down(const T* in, T* out, int64_t n,
                                                           const T* block_base) {
  __shared__ T stage[kScanTile];
  __shared__ T warp_tot[32];
  __shared__ T tot;
  const int64_t base = (int64_t)blockIdx.x * kScanTile;
  // coalesced load into shared memory, then each thread owns 8 consecutive items
#pragma unroll
  for (int j = 0; j < kScanItems; ++j) {
    int64_t k = base + j * kScanThreads + threadIdx.x;
    stage[j * kScanThreads + threadIdx.x] = k < n ? in[k] : T(0);
  }
  __syncthreads();
  T v[kScanItems];
  T s = 0;
#pragma unroll
  for (int j = 0; j < kScanItems; ++j) {
    v[j] = stage[threadIdx.x * kScanItems + j];
    s += v[j];
  }
  T run = block_exclusive_sum<T>(s, warp_tot, &tot);
  if (block_base) run += block_base[blockIdx.x];
#pragma unroll
  for (int j = 0; j < kScanItems; ++j) {
    stage[threadIdx.x * kScanItems + j] = run;
    run += v[j];
  }
  __syncthreads();
#pragma unroll
  for (int j = 0; j < kScanItems; ++j) {
    int64_t k = base + j * kScanThreads + threadIdx.x;
    if (k < n) out[k] = stage[j * kScanThreads + threadIdx.x];
  }
  if (base + kScanTile >= n && threadIdx.x == 0) {
    // the last block writes the grand total
    T total = tot + (block_base ? block_base[blockIdx.x] : T(0));
    out[n] = total;
  }
}
}  // namespace

template <typename T>
size_t scan_ws_elems(int64_t n) {
  size_t total = 0;
  while (n > kScanTile) {
    int64_t nb = (n + kScanTile - 1) / kScanTile;
    total += 2 * nb + 1;
    n = nb;
  }
  return total + 1;
}

template <typename T>
void scan_exclusive(const T* in, T* out, int64_t n, T* ws, cudaStream_t s) {
  if (n <= 0) {
    cudaMemsetAsync(out, 0, sizeof(T), s);
    return;
  }
  int64_t nb = (n + kScanTile - 1) / kScanTile;
  if (nb == 1) {
    count_launch();
    k_scan_down<T><<<1, kScanThreads, 0, s>>>(in, out, n, nullptr);
    return;
  }
  T* part = ws;
  T* part_scan = ws + nb;
  count_launch();
  k_scan_reduce<T><<<(unsigned)nb, kScanThreads, 0, s>>>(in, n, part);
  scan_exclusive<T>(part, part_scan, nb, ws + 2 * nb + 1, s);
  count_launch();
  k_scan_down<T><<<(unsigned)nb, kScanThreads, 0, s>>>(in, out, n, part_scan);
}

template size_t scan_ws_elems<uint32_t>(int64_t);
template size_t scan_ws_elems<uint64_t>(int64_t);
template void scan_exclusive<uint32_t>(const uint32_t*, uint32_t*, int64_t, uint32_t*, cudaStream_t);
template void scan_exclusive<uint64_t>(const uint64_t*, uint64_t*, int64_t, uint64_t*, cudaStream_t);

// ---------------------------------------------------------------------------
// radix sort
// ---------------------------------------------------------------------------
namespace {
constexpr int kRadixThreads = 256;
constexpr int kRadixWarps = kRadixThreads / 32;
constexpr int kRadixIpt = 16;                                 // keys per thread
constexpr int kRadixTile = kRadixThreads * kRadixIpt;         // 4096 keys per block
constexpr int kRadixWarpKeys = kRadixTile / kRadixWarps;      // 512 keys per warp

template <typename K>
__global__ void __launch_bounds__(kRadixThreads) k_radix_hist(const K* keys, int64_t n, int shift,
                                                             uint32_t mask, uint32_t* hist,
                                                             int64_t nblocks) {
  __shared__ uint32_t h[256];
  h[threadIdx.x] = 0;
  __syncthreads();
  const int64_t base = (int64_t)blockIdx.x * kRadixTile;
#pragma unroll 4
  for (int j = 0; j < kRadixIpt; ++j) {
    int64_t k = base + j * kRadixThreads + threadIdx.x;
    if (k < n) atomicAdd(&h[(uint32_t)(keys[k] >> shift) & mask], 1u);
  }
  __syncthreads();
  hist[(int64_t)threadIdx.x * nblocks + blockIdx.x] = h[threadIdx.x];
}

// dynamic shared memory of one scatter block: its keys (and values) in
// block-sorted order
template <typename K, bool HAS_V>
constexpr size_t scatter_smem_bytes() {
  return (size_t)kRadixTile * (sizeof(K) + (HAS_V ? sizeof(uint64_t) : 0));
}

// One pass of the LSD radix sort over a block of kRadixTile keys: every key is
// ranked within its warp and digit (match_any), the ranks become positions in
// the block's digit-sorted order, the keys are reordered in shared memory, and
// consecutive threads then write consecutive keys of each digit run to the
// run's global offset, so the global writes are coalesced. Stable.
template <typename K, bool HAS_V>
__global__ void __launch_bounds__(kRadixThreads) k_radix_scatter(
    const K* __restrict__ keys, const uint64_t* __restrict__ vals, K* __restrict__ keys_out,
    uint64_t* __restrict__ vals_out, int64_t n, int shift, uint32_t mask,
    const uint32_t* __restrict__ offs, int64_t nblocks) {
  __shared__ uint32_t wcnt[kRadixWarps][256];
  __shared__ uint32_t boff[256];    // the digit's first position in the output
  __shared__ uint32_t bstart[257];  // the digit's first position in the block's sorted order
  __shared__ uint32_t wsum[kRadixWarps];
  extern __shared__ __align__(16) unsigned char rsmem[];
  K* sk = reinterpret_cast<K*>(rsmem);
  uint64_t* sv = reinterpret_cast<uint64_t*>(rsmem + (size_t)kRadixTile * sizeof(K));
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int w = 0; w < kRadixWarps; ++w) wcnt[w][threadIdx.x] = 0;
  boff[threadIdx.x] = offs[(int64_t)threadIdx.x * nblocks + blockIdx.x];
  __syncthreads();
  const int64_t wbase = (int64_t)blockIdx.x * kRadixTile + (int64_t)warp * kRadixWarpKeys;
  K kv[kRadixIpt];
  uint64_t vv[HAS_V ? kRadixIpt : 1];
  uint32_t rk[kRadixIpt];
  const unsigned lt = lanemask_lt();
#pragma unroll
  for (int r = 0; r < kRadixIpt; ++r) {
    int64_t idx = wbase + r * 32 + lane;
    bool valid = idx < n;
    K k = valid ? keys[idx] : K(0);
    kv[r] = k;
    if (HAS_V) vv[HAS_V ? r : 0] = valid ? vals[idx] : 0ull;
    uint32_t d = valid ? ((uint32_t)(k >> shift) & mask) : 256u;
    unsigned peers = __match_any_sync(0xffffffffu, d);
    uint32_t before = __popc(peers & lt);
    uint32_t base = valid ? wcnt[warp][d] : 0u;
    __syncwarp();
    if (valid && before == 0) wcnt[warp][d] = base + __popc(peers);
    __syncwarp();
    rk[r] = base + before;
  }
  __syncthreads();
  // per digit (thread d): warp prefixes, and the digit's block total
  uint32_t tot = 0;
#pragma unroll
  for (int w = 0; w < kRadixWarps; ++w) {
    uint32_t t = wcnt[w][threadIdx.x];
    wcnt[w][threadIdx.x] = tot;
    tot += t;
  }
  // exclusive scan of the totals over the 256 digits (warp scans, then warps)
  uint32_t incl = tot;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += y;
  }
  if (lane == 31) wsum[warp] = incl;
  __syncthreads();
  uint32_t wpre = 0;
#pragma unroll
  for (int w = 0; w < kRadixWarps; ++w) wpre += w < warp ? wsum[w] : 0u;
  bstart[threadIdx.x] = wpre + incl - tot;
  if (threadIdx.x == kRadixThreads - 1) bstart[256] = wpre + incl;
  __syncthreads();
#pragma unroll
  for (int r = 0; r < kRadixIpt; ++r) {
    int64_t idx = wbase + r * 32 + lane;
    if (idx < n) {
      const uint32_t d = (uint32_t)(kv[r] >> shift) & mask;
      const uint32_t lp = bstart[d] + wcnt[warp][d] + rk[r];
      sk[lp] = kv[r];
      if (HAS_V) sv[lp] = vv[HAS_V ? r : 0];
    }
  }
  __syncthreads();
  const uint32_t nvalid = bstart[256];
  for (uint32_t i = threadIdx.x; i < nvalid; i += kRadixThreads) {
    const K k = sk[i];
    const uint32_t d = (uint32_t)(k >> shift) & mask;
    const uint32_t dst = boff[d] + (i - bstart[d]);
    keys_out[dst] = k;
    if (HAS_V) vals_out[dst] = sv[i];
  }
}

template <typename K, bool HAS_V>
void launch_scatter(const K* kin, const uint64_t* vin, K* kout, uint64_t* vout, int64_t n, int shift, uint32_t mask,
                    const uint32_t* offs, int64_t nb, cudaStream_t s) {
  // above the default 48 KB of dynamic shared memory for some instantiations:
  // one fixed size per instantiation, set once per device
  static std::mutex mu;
  static std::set<int> done;
  int dev = 0;
  cudaGetDevice(&dev);
  {
    std::lock_guard<std::mutex> lk(mu);
    if (!done.count(dev)) {
      cudaFuncSetAttribute(k_radix_scatter<K, HAS_V>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)scatter_smem_bytes<K, HAS_V>());
      done.insert(dev);
    }
  }
  count_launch();
  k_radix_scatter<K, HAS_V><<<(unsigned)nb, kRadixThreads, scatter_smem_bytes<K, HAS_V>(), s>>>(
      kin, vin, kout, vout, n, shift, mask, offs, nb);
}
}  // namespace

size_t radix_ws_bytes(int64_t n) {
  int64_t nb = (n + kRadixTile - 1) / kRadixTile;
  int64_t h = 256 * (nb > 0 ? nb : 1);
  return (size_t)(2 * h + 1 + scan_ws_elems<uint32_t>(h)) * sizeof(uint32_t) + 256;
}

template <typename K>
int radix_sort(K* keys, K* keys_alt, uint64_t* vals, uint64_t* vals_alt, int64_t n, int nbits,
               void* ws, cudaStream_t s) {
  if (n <= 1 || nbits <= 0) return 0;
  int64_t nb = (n + kRadixTile - 1) / kRadixTile;
  int64_t h = 256 * nb;
  uint32_t* hist = (uint32_t*)ws;
  uint32_t* offs = hist + h;
  uint32_t* sws = offs + h + 1;
  K* kin = keys;
  K* kout = keys_alt;
  uint64_t* vin = vals;
  uint64_t* vout = vals_alt;
  int flips = 0;
  for (int shift = 0; shift < nbits; shift += 8) {
    int bits = nbits - shift < 8 ? nbits - shift : 8;
    uint32_t mask = (1u << bits) - 1u;
    count_launch();
    k_radix_hist<K><<<(unsigned)nb, kRadixThreads, 0, s>>>(kin, n, shift, mask, hist, nb);
    scan_exclusive<uint32_t>(hist, offs, h, sws, s);
    if (vals) {
      launch_scatter<K, true>(kin, vin, kout, vout, n, shift, mask, offs, nb, s);
    } else {
      launch_scatter<K, false>(kin, nullptr, kout, nullptr, n, shift, mask, offs, nb, s);
    }
    K* t = kin;
    kin = kout;
    kout = t;
    uint64_t* tv = vin;
    vin = vout;
    vout = tv;
    flips ^= 1;
  }
  return flips;
}

template int radix_sort<uint32_t>(uint32_t*, uint32_t*, uint64_t*, uint64_t*, int64_t, int, void*,
                                  cudaStream_t);
template int radix_sort<uint64_t>(uint64_t*, uint64_t*, uint64_t*, uint64_t*, int64_t, int, void*,
                                  cudaStream_t);

// Loads every kernel of this file now (lazy module loading would otherwise
// load a kernel at its first launch, which can wait on a running persistent
// kernel, e.g. the serving kernel).
void preload_primitives() {
  cudaFuncAttributes a;
  cudaFuncGetAttributes(&a, k_scan_reduce<uint32_t>);
  cudaFuncGetAttributes(&a, k_scan_reduce<uint64_t>);
  cudaFuncGetAttributes(&a, k_scan_down<uint32_t>);
  cudaFuncGetAttributes(&a, k_scan_down<uint64_t>);
  cudaFuncGetAttributes(&a, k_radix_hist<uint32_t>);
  cudaFuncGetAttributes(&a, k_radix_hist<uint64_t>);
  cudaFuncGetAttributes(&a, k_radix_scatter<uint32_t, true>);
  cudaFuncGetAttributes(&a, k_radix_scatter<uint32_t, false>);
  cudaFuncGetAttributes(&a, k_radix_scatter<uint64_t, true>);
  cudaFuncGetAttributes(&a, k_radix_scatter<uint64_t, false>);
}

void preload_all() {
  preload_primitives();
  preload_analysis();
  preload_sweep();
  preload_exec();
  preload_serve();
  preload_events();
  preload_task_kernel();
  preload_stitch();
  preload_static();
  preload_microbench();
}

}  // namespace grt
