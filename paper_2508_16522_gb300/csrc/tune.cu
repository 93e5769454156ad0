// tune.cu -- the autotuner: analysis tile shape and executor launch shape.
//
// Results never depend on these knobs (tile size, persistent blocks per SM,
// warps per block, ring slots claimed at once, ready successors kept per
// warp); only speed does, and the best values depend on the workload and the
// device. Each tuner measures candidates on the caller's own workload and
// keeps the fastest:
//   rt_tune_tile   -- analyses the trace once per candidate tile (timed by
//                     the analysis's own events) and returns the fastest;
//   rt_tune_exec   -- runs an analysed graph under candidate launch shapes and
//                     configures it with the fastest;
//   rt_tune_batch  -- the same for a batch launch with its replay count.
// The executor search is coordinate descent for the ring policy: (warps,
// blocks per SM) jointly, then the claim width, then the keep width, then
// (warps, blocks per SM) again; then a pass over the grids of the owned
// policy, and its group sizes (lanes per task) on the best grid; each ring
// trial the best of two runs, each owned trial the best of three.
// Results go to an optional plain-text cache, one line per workload key
// (device, SM count, kind, sizes, an input hash), so a later call with the
// same workload answers without running anything.
#include <stdio.h>
#include <string.h>

#include <chrono>
#include <mutex>
#include <string>
#include <vector>

#include "grt_internal.cuh"

using namespace grt;

namespace {

std::mutex g_cache_mu;

rt_status tfail(rt_status st, const std::string& m) {
  set_last_error(m.c_str());
  return st;
}

std::string device_tag() {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaDeviceProp prop;
  std::string name = "gpu";
  if (cudaGetDeviceProperties(&prop, dev) == cudaSuccess) name = prop.name;
  for (char& c : name)
    if (c == ' ' || c == '\t') c = '_';
  return name + "/" + std::to_string(sms);
}

uint64_t fnv(uint64_t h, const void* p, size_t bytes) {
  const unsigned char* c = static_cast<const unsigned char*>(p);
  for (size_t i = 0; i < bytes; ++i) {
    h ^= c[i];
    h *= 1099511628211ull;
  }
  return h;
}

// the cached values of `key`, if the cache file has them
bool cache_get(const char* path, const std::string& key, std::vector<double>* vals) {
  if (!path || !*path) return false;
  std::lock_guard<std::mutex> lk(g_cache_mu);
  FILE* f = fopen(path, "r");
  if (!f) return false;
  char line[1024];
  bool found = false;
  while (fgets(line, sizeof line, f)) {
    char* sp = strchr(line, ' ');
    if (!sp) continue;
    *sp = 0;
    if (key != line) continue;
    vals->clear();
    char* q = sp + 1;
    for (;;) {
      char* end = nullptr;
      const double v = strtod(q, &end);
      if (end == q) break;
      vals->push_back(v);
      q = end;
    }
    found = true;  // the last line for a key wins
  }
  fclose(f);
  return found;
}

void cache_put(const char* path, const std::string& key, const std::vector<double>& vals) {
  if (!path || !*path) return;
  std::lock_guard<std::mutex> lk(g_cache_mu);
  FILE* f = fopen(path, "a");
  if (!f) return;
  fprintf(f, "%s", key.c_str());
  for (double v : vals) fprintf(f, " %.6g", v);
  fprintf(f, "\n");
  fclose(f);
}

struct Shape {
  int warps, bps, claim, keep;
};

// Coordinate descent over launch shapes; `run` returns the time of one run
// (ms) or a negative value on failure.
template <class Run>
rt_status search(int sms, Shape start, Run run, Shape* best, float* best_ms, int* trials) {
  auto trial = [&](const Shape& s, double* ms) -> rt_status {
    double t = 1e30;
    for (int rep = 0; rep < 2; ++rep) {
      const double m = run(s);
      if (m < 0) return RT_ERR_CUDA;
      if (m < t) t = m;
    }
    ++*trials;
    *ms = t;
    return RT_OK;
  };
  Shape cur = start;
  double cur_ms = 0;
  rt_status st = trial(cur, &cur_ms);
  if (st != RT_OK) return st;
  const int warps_c[] = {2, 4, 8};
  auto shape_pass = [&]() -> rt_status {
    for (int w : warps_c) {
      const int maxb = std::max(exec_max_blocks_per_sm(w), 1);
      for (int b = 1; b <= std::min(maxb, 3); ++b) {
        Shape s = cur;
        s.warps = w;
        s.bps = b;
        if (s.warps == cur.warps && s.bps == cur.bps) continue;
        double ms = 0;
        rt_status r = trial(s, &ms);
        if (r != RT_OK) return r;
        if (ms < cur_ms) {
          cur = s;
          cur_ms = ms;
        }
      }
    }
    return RT_OK;
  };
  if ((st = shape_pass()) != RT_OK) return st;
  const int claim_c[] = {1, 2, 4, 8, 16, 32};
  const Shape after_shape = cur;
  for (int c : claim_c) {
    if (c == after_shape.claim) continue;
    Shape s = after_shape;
    s.claim = c;
    double ms = 0;
    if ((st = trial(s, &ms)) != RT_OK) return st;
    if (ms < cur_ms) {
      cur = s;
      cur_ms = ms;
    }
  }
  const int keep_c[] = {2, 4, 8, 16, 32, 64};
  const Shape after_claim = cur;
  for (int k : keep_c) {
    if (k == after_claim.keep) continue;
    Shape s = after_claim;
    s.keep = k;
    double ms = 0;
    if ((st = trial(s, &ms)) != RT_OK) return st;
    if (ms < cur_ms) {
      cur = s;
      cur_ms = ms;
    }
  }
  // the best grid can move with the widths: one more pass over it
  if ((st = shape_pass()) != RT_OK) return st;
  (void)sms;
  *best = cur;
  *best_ms = (float)cur_ms;
  return RT_OK;
}

}  // namespace

extern "C" {

rt_status rt_tune_tile(const rt_graph_desc* desc, int32_t n, const int32_t* req_off, const int64_t* lo,
                       const int64_t* hi, const uint8_t* priv, const char* cache_path, int32_t* tile_w,
                       int32_t* tile_h, float* ms) {
  if (!desc || !req_off || !tile_w || !tile_h || n < 0) return tfail(RT_ERR_INVALID, "bad arguments");
  const int D = desc->ndim;
  if (D != 1 && D != 2) return tfail(RT_ERR_INVALID, "ndim must be 1 or 2");
  const int64_t R = req_off[n];
  if (R < 0 || (R > 0 && (!lo || !hi || !priv))) return tfail(RT_ERR_INVALID, "rect arrays missing");
  uint64_t h = 1469598103934665603ull;
  h = fnv(h, req_off, (size_t)(n + 1) * 4);
  const int64_t Rh = std::min<int64_t>(R, 1 << 20);
  if (Rh > 0) {
    h = fnv(h, lo, (size_t)Rh * D * 8);
    h = fnv(h, hi, (size_t)Rh * D * 8);
    h = fnv(h, priv, (size_t)Rh);
  }
  char hb[32];
  snprintf(hb, sizeof hb, "%016llx", (unsigned long long)h);
  // "tile3": entries of the sweep with its row mode for segment tiles, and of
  // the candidate list below (older entries are never read)
  const std::string key = "tile3/" + device_tag() + "/" + std::to_string(D) + "/" +
                          std::to_string(desc->dom_hi[0] - desc->dom_lo[0] + 1) + "x" +
                          std::to_string(D == 2 ? desc->dom_hi[1] - desc->dom_lo[1] + 1 : 1) + "/" +
                          std::to_string(n) + "/" + std::to_string(R) + "/" + hb;
  std::vector<double> cached;
  if (cache_get(cache_path, key, &cached) && cached.size() >= 3) {
    *tile_w = (int32_t)cached[0];
    *tile_h = (int32_t)cached[1];
    if (ms) *ms = (float)cached[2];
    return RT_OK;
  }
  std::vector<std::pair<int, int>> cands;
  if (D == 2) {
    // squares, and flat or tall ones (a Task Bench step is a row of the domain:
    // 8 x 16 sweeps its stencil graph in 0.81 ms against 1.12 ms for 16 x 16;
    // dense tiles sweep their class rows one lane each, so 32 rows keep a
    // warp's lanes busy)
    for (int t : {8, 16, 32, 64}) cands.push_back({t, t});
    for (auto wh : {std::pair<int, int>{8, 16}, {16, 8}, {32, 4}, {32, 8}, {64, 4}, {8, 32}, {16, 32}, {32, 16}})
      cands.push_back(wh);
  } else {
    for (int t : {128, 256, 512, 1024}) cands.push_back({t, 1});
  }
  double best = 1e30;
  int bw = 0, bh = 0;
  std::string last;
  for (auto [cw, ch] : cands) {
    rt_graph_desc d = *desc;
    d.tile_w = cw;
    d.tile_h = ch;
    d.body = RT_BODY_EMPTY;  // analysis only
    d.state = nullptr;
    d.state_elems = 0;
    d.out = nullptr;
    d.out_elems = 0;
    d.flags = RT_GRAPH_PROFILE;
    rt_graph_t g = nullptr;
    if (rt_graph_create(&d, &g) != RT_OK) {
      last = rt_last_error();
      continue;
    }
    double t = -1;
    for (int rep = 0; rep < 2; ++rep) {  // the first run grows the buffers
      rt_graph_stats_t st{};
      if (rt_graph_clear(g) != RT_OK ||
          rt_launch_batch(g, n, req_off, lo, hi, priv, nullptr, nullptr, nullptr, RT_LAUNCH_DEFER_CHECK) != RT_OK ||
          rt_analyze(g) != RT_OK || rt_graph_stats(g, &st) != RT_OK) {
        last = rt_last_error();
        t = -1;
        break;
      }
      t = st.ms_analyze;
    }
    rt_graph_destroy(g);
    if (t >= 0 && t < best) {
      best = t;
      bw = cw;
      bh = ch;
    }
  }
  if (bw == 0) return tfail(RT_ERR_INVALID, "no tile candidate analysed: " + last);
  *tile_w = bw;
  *tile_h = bh;
  if (ms) *ms = (float)best;
  cache_put(cache_path, key, {(double)bw, (double)bh, best});
  return RT_OK;
}

rt_status rt_tune_exec(rt_graph_t g, const char* cache_path, rt_exec_config* best) {
  if (!g || !best) return tfail(RT_ERR_INVALID, "NULL argument");
  rt_graph_stats_t st{};
  rt_status s = rt_graph_stats(g, &st);
  if (s != RT_OK) return s;
  int sms = 0;
  if ((s = rt_device_info(&sms, nullptr)) != RT_OK) return s;
  // "exec7": entries for the owned kernel whose decrements are reductions, with
  // its grids and group sizes (entries of older kernels are never read)
  const std::string key = "exec7/" + device_tag() + "/" + std::to_string(st.n_tasks) + "/" +
                          std::to_string(st.n_edges) + "/" + std::to_string(st.n_roots);
  auto apply = [&](const rt_exec_config& c) -> rt_status {
    rt_status r = rt_graph_exec_policy(g, c.policy);
    return r != RT_OK ? r : rt_graph_exec_config(g, c.blocks, c.warps, c.claim, c.keep);
  };
  std::vector<double> c;
  if (cache_get(cache_path, key, &c) && c.size() >= 6) {
    *best = rt_exec_config{(int32_t)c[0], (int32_t)c[1], (int32_t)c[2], (int32_t)c[3], (float)c[4], 0,
                           (int32_t)c[5]};
    return apply(*best);
  }
  auto run = [&](const Shape& sh) -> double {
    if (rt_graph_exec_config(g, sms * sh.bps, sh.warps, sh.claim, sh.keep) != RT_OK) return -1;
    const auto t0 = std::chrono::steady_clock::now();
    if (rt_execute(g) != RT_OK || rt_sync(g) != RT_OK) return -1;
    return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  };
  Shape b{};
  float ms = 0;
  int trials = 0;
  rt_graph_exec_policy(g, RT_EXEC_RING);
  if ((s = search(sms, Shape{2, 1, 8, 16}, run, &b, &ms, &trials)) != RT_OK) {
    rt_graph_exec_config(g, 0, 0, 0, 0);
    return tfail(s, std::string("executor trial failed: ") + rt_last_error());
  }
  *best = rt_exec_config{sms * b.bps, b.warps, b.claim, b.keep, ms, trials, RT_EXEC_RING};
  rt_graph_exec_policy(g, RT_EXEC_OWNED);
  // the owned policy: grids from 32 warps (a Task Bench step's 32 chunks, each
  // warp always on the same column of chunks) up to several warps per SM, one
  // lane per task; then groups of 2 and 4 lanes per task (chunks of 16 and 8
  // tasks) on the best grid and on one that many times wider
  auto run_owned = [&](int blocks, int warps, int group) -> double {
    if (rt_graph_exec_config(g, blocks, warps, group, 16) != RT_OK) return -1;
    const auto t0 = std::chrono::steady_clock::now();
    if (rt_execute(g) != RT_OK || rt_sync(g) != RT_OK) return -1;
    return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  };
  bool failed = false;
  auto owned_trial = [&](int blocks, int warps, int group) {
    double t = 1e30;
    for (int rep = 0; rep < 3 && !failed; ++rep) {
      const double m = run_owned(blocks, warps, group);
      if (m < 0) failed = true;
      t = std::min(t, m);
    }
    ++trials;
    if (!failed && t < best->ms)
      *best = rt_exec_config{blocks, warps, group, 16, (float)t, trials, RT_EXEC_OWNED};
  };
  const int owned_c[][2] = {{32, 1}, {64, 1}, {96, 1}, {128, 1}, {152, 1}, {152, 2}, {152, 4}, {304, 2}};
  for (const auto& bw : owned_c) {
    const int blocks = bw[0] * sms / 152 > 0 ? bw[0] * sms / 152 : 1;  // scaled to this GPU's SM count
    if (blocks > sms * std::max(exec_max_blocks_per_sm(bw[1]), 1)) continue;
    owned_trial(blocks, bw[1], 1);
  }
  if (!failed && best->policy == RT_EXEC_OWNED) {
    const int gb = best->blocks, gwp = best->warps;
    for (int group : {2, 4}) {
      owned_trial(gb, gwp, group);
      const int wider = std::min(gb * group, sms * std::max(exec_max_blocks_per_sm(gwp), 1));
      if (wider > gb) owned_trial(wider, gwp, group);
    }
  }
  if (failed) {
    rt_graph_exec_policy(g, RT_EXEC_RING);
    rt_graph_exec_config(g, 0, 0, 0, 0);
    return tfail(RT_ERR_CUDA, std::string("executor trial failed: ") + rt_last_error());
  }
  best->trials = trials;
  cache_put(cache_path, key, {(double)best->blocks, (double)best->warps, (double)best->claim, (double)best->keep,
                              best->ms, (double)best->policy});
  return apply(*best);
}

rt_status rt_tune_batch(rt_batch_t b, int32_t replays, const char* cache_path, rt_exec_config* best) {
  if (!b || !best || replays < 1) return tfail(RT_ERR_INVALID, "bad arguments");
  int64_t G = 0, T = 0, E = 0;
  rt_status s = batch_shape(b, &G, &T, &E);
  if (s != RT_OK) return s;
  int sms = 0;
  if ((s = rt_device_info(&sms, nullptr)) != RT_OK) return s;
  // "batch2": entries that also weigh the owned policy (the batch as one DAG)
  const std::string key = "batch2/" + device_tag() + "/" + std::to_string(G) + "/" + std::to_string(T) + "/" +
                          std::to_string(E) + "/" + std::to_string(replays);
  std::vector<double> c;
  if (cache_get(cache_path, key, &c) && c.size() >= 6) {
    *best = rt_exec_config{(int32_t)c[0], (int32_t)c[1], (int32_t)c[2], (int32_t)c[3], (float)c[4], 0, (int32_t)c[5]};
    return rt_batch_exec_policy(b, best->policy);
  }
  auto run = [&](const Shape& sh) -> double {
    float ms = 0;
    if (rt_batch_execute(b, replays, sms * sh.bps, sh.warps, sh.claim, sh.keep) != RT_OK ||
        rt_batch_sync(b, &ms) != RT_OK)
      return -1;
    return ms;
  };
  Shape sh{};
  float ms = 0;
  int trials = 0;
  rt_batch_exec_policy(b, RT_EXEC_RING);
  const int bps4 = std::max(exec_max_blocks_per_sm(4), 1);
  if ((s = search(sms, Shape{4, std::min(bps4, 3), 32, 32}, run, &sh, &ms, &trials)) != RT_OK)
    return tfail(s, std::string("batch trial failed: ") + rt_last_error());
  *best = rt_exec_config{sms * sh.bps, sh.warps, sh.claim, sh.keep, ms, trials, RT_EXEC_RING};
  // the owned policy: one probe at two blocks of 8 warps per SM (one run: on
  // a batch of unrelated graphs a warp's chunks lie in many graphs and one
  // graph's progress waits for the others', so it can be many times slower);
  // only if that probe comes within 1.5x of the ring, the other grids (one to
  // three blocks of 4 or 8 warps per SM) and 2 and 4 lanes per task
  rt_batch_exec_policy(b, RT_EXEC_OWNED);
  bool failed = false;
  auto owned_trial = [&](int blocks, int warps, int group, int reps) {
    if (blocks > sms * std::max(exec_max_blocks_per_sm(warps), 1)) return;
    double t = 1e30;
    for (int rep = 0; rep < reps && !failed; ++rep) {
      float m = 0;
      if (rt_batch_execute(b, replays, blocks, warps, group, 16) != RT_OK || rt_batch_sync(b, &m) != RT_OK)
        failed = true;
      t = std::min<double>(t, m);
    }
    ++trials;
    if (!failed && t < best->ms) *best = rt_exec_config{blocks, warps, group, 16, (float)t, trials, RT_EXEC_OWNED};
  };
  const double ring_ms = best->ms;
  double probe_ms = 1e30;
  {
    float m = 0;
    if (rt_batch_execute(b, replays, sms * 2, 8, 1, 16) == RT_OK && rt_batch_sync(b, &m) == RT_OK)
      probe_ms = m;
    ++trials;
  }
  if (probe_ms < 1.5 * ring_ms) {
    const int grids[][2] = {{1, 4}, {1, 8}, {2, 4}, {2, 8}, {3, 8}};  // (blocks per SM, warps)
    for (const auto& gw : grids) owned_trial(sms * gw[0], gw[1], 1, 2);
    if (!failed && best->policy == RT_EXEC_OWNED) {
      const int gb = best->blocks, gwp = best->warps;
      for (int group : {2, 4}) owned_trial(gb, gwp, group, 2);
    }
  }
  if (failed) {
    rt_batch_exec_policy(b, RT_EXEC_RING);
    return tfail(RT_ERR_CUDA, std::string("batch trial failed: ") + rt_last_error());
  }
  best->trials = trials;
  rt_batch_exec_policy(b, best->policy);
  cache_put(cache_path, key, {(double)best->blocks, (double)best->warps, (double)best->claim, (double)best->keep,
                              best->ms, (double)best->policy});
  return RT_OK;
}

}  // extern "C"
