// Autotuner of the persistent kernel: the GPU counterpart of Section 5.4's
// ring-size tuning, which pre-runs short walks and keeps the ring sizes that
// run them fastest.  Here the knobs are threads per block, resident blocks
// per SM, the work-queue chunk and the degrees from which the warp takes over
// a MetaPath label scan or a Node2Vec neighbour search.  A calibration walk
// of length 10 sizes the pre-walks so that each trial lasts about 2 ms with
// walks as long as the real ones (up to 80 moves): trials that short of the
// launch overhead would let noise pick between configurations within 10 % of
// each other.  Each candidate keeps the median of three trials.  Walk results
// never depend on these knobs.
#include <algorithm>
#include <vector>

#include <cuda_runtime.h>

#include "trw_api_internal.h"

using namespace trw;

extern "C" trw_status trw_autotune(trw_graph* g, trw_algo algo, const trw_params* params, int32_t max_len,
                                   trw_tuning* best_out) {
  if (!g) return trw_fail(TRW_ERR_INVALID, "graph is NULL");
  if (trw_status dc = trw_check_device(g); dc != TRW_OK) return dc;
  if (g->nv == 0) return trw_fail(TRW_ERR_INVALID, "empty graph");
  const int32_t len0 = std::max(1, std::min<int32_t>(max_len, 10));
  const int32_t len_max = std::max(1, std::min<int32_t>(max_len, 80));
  // Sources: an even stride over the vertices, enough walks to fill the GPU a few times.
  const int64_t n = std::min<int64_t>(g->nv, (int64_t)g->num_sms * 2048 * 2);
  const int64_t n_min = std::min<int64_t>(n, (int64_t)g->num_sms * 256);
  std::vector<int32_t> src((size_t)n);
  for (int64_t i = 0; i < n; ++i) src[(size_t)i] = (int32_t)((i * g->nv) / n);
  trw_params p;
  if (params) p = *params;
  else trw_params_default(&p);
  p.walks_per_source = 1;
  p.walk_offset = 0;
  WalkSpec sp;
  trw_status st = trw_make_spec(g, algo, &p, n, len_max, 0x5eedULL, &sp);
  if (st != TRW_OK) return st;
  const size_t out_elems = sp.endpoints ? (size_t)n : (size_t)n * ((size_t)len_max + 1);
  int32_t *d_src = nullptr, *d_out = nullptr, *d_len = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t e = trw_dev_malloc((void**)&d_src, sizeof(int32_t) * (size_t)n);
  if (e == cudaSuccess) e = trw_dev_malloc((void**)&d_out, sizeof(int32_t) * out_elems);
  if (e == cudaSuccess) e = trw_dev_malloc((void**)&d_len, sizeof(int32_t) * (size_t)n);
  if (e == cudaSuccess) e = cudaMemcpy(d_src, src.data(), sizeof(int32_t) * (size_t)n, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  trw_tuning best = g->tuning;
  float best_ms = 1e30f;
  if (e == cudaSuccess) {
    std::lock_guard<std::mutex> lk(g->mu);
    sp.sources = d_src;
    sp.out_paths = d_out;
    sp.out_lengths = d_len;
    const DevGraph dg = trw_dev_graph(g);
    // One timed launch of the kernel as it is configured now.
    auto timed = [&](const LaunchCfg& cfg, float* ms) {
      cudaError_t r = cudaMemsetAsync(g->ctrl, 0, sizeof(Ctrl), g->stream);
      if (r == cudaSuccess) r = cudaEventRecord(e0, g->stream);
      if (r == cudaSuccess) r = launch_walk_persistent(dg, sp, g->ctrl, g->stream, cfg);
      if (r == cudaSuccess) r = cudaEventRecord(e1, g->stream);
      if (r == cudaSuccess) r = cudaEventSynchronize(e1);
      if (r == cudaSuccess) r = cudaEventElapsedTime(ms, e0, e1);
      return r;
    };
    // Calibration: length-10 walks under the current tuning, then walks as
    // long as the real ones (capped at 80 moves) on as many sources as keep a
    // trial near 2 ms, never fewer than fill the GPU once.
    {
      const LaunchCfg base = trw_launch_cfg(g, sp.algo);
      sp.max_len = len0;
      float ms0 = 0.f;
      for (int rep = 0; rep < 2 && e == cudaSuccess; ++rep) e = timed(base, &ms0);
      const double per = e == cudaSuccess ? (double)ms0 / ((double)n * len0) : 0.0;  // ms per walk-move
      int64_t nt = n;
      int32_t lt = len_max;
      if (per > 0) {
        const double target = 2.0;
        if ((double)nt * lt * per > target) nt = std::max<int64_t>(n_min, (int64_t)(target / (lt * per)));
        if ((double)nt * lt * per > target) lt = std::max<int32_t>(len0, (int32_t)(target / (nt * per)));
      }
      sp.max_len = lt;
      sp.nwalks = nt;
      if (nt < n && e == cudaSuccess) {  // fewer sources, still spread over every vertex
        for (int64_t i = 0; i < nt; ++i) src[(size_t)i] = (int32_t)((i * g->nv) / nt);
        e = cudaMemcpy(d_src, src.data(), sizeof(int32_t) * (size_t)nt, cudaMemcpyHostToDevice);
      }
    }
    // Degree thresholds tried: MetaPath scans (coop_degree) or Node2Vec
    // searches (search_degree); 0x7fffffff keeps every row with its own lane.
    const int kOff = 0x7fffffff;
    const int threads_c[] = {64, 128, 256, 512};
    const int chunk_c[] = {8, 32, 128};
    std::vector<int> deg_c;
    if (algo == TRW_METAPATH && !g->lerec) deg_c = {64, 256, 1024, kOff};
    else if ((algo == TRW_NODE2VEC || algo == TRW_NODE2VEC_WEIGHTED) && !g->nh_slots) deg_c = {64, 1024, kOff};
    else deg_c = {kOff};
    for (int threads : threads_c) {
      for (int cd : deg_c) {
      const bool coop = cd != kOff;
      const int occ = persistent_blocks_per_sm(sp.algo, threads, coop);
      for (int bps_div = 1; bps_div <= 2; ++bps_div) {
        const int bps = std::max(1, occ / bps_div);
        if (bps_div == 2 && bps == occ) continue;
        for (int chunk : chunk_c) {
          {
            LaunchCfg cfg;
            cfg.block_threads = threads;
            cfg.grid_blocks = g->num_sms * bps;
            cfg.chunk = chunk;
            cfg.coop_degree = algo == TRW_METAPATH ? cd : g->tuning.coop_degree;
            cfg.search_degree = (algo == TRW_NODE2VEC || algo == TRW_NODE2VEC_WEIGHTED) ? cd : g->tuning.search_degree;
            float t[4] = {0.f, 0.f, 0.f, 0.f};
            for (int rep = 0; rep < 4 && e == cudaSuccess; ++rep) e = timed(cfg, &t[rep]);  // rep 0 warms up
            if (e != cudaSuccess) break;
            std::sort(t + 1, t + 4);
            const float ms_med = t[2];
            if (ms_med < best_ms) {
              best_ms = ms_med;
              best.block_threads = threads;
              best.blocks_per_sm = bps;
              best.chunk = chunk;
              best.coop_degree = cfg.coop_degree;
              best.search_degree = cfg.search_degree;
            }
          }
        }
      }
      }
    }
    Ctrl c{};
    if (e == cudaSuccess) e = cudaMemcpy(&c, g->ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && c.err != 0) st = trw_fail(TRW_ERR_INTERNAL, "autotune pre-walk status %d", c.err);
    if (e == cudaSuccess && st == TRW_OK) g->tuning = best;
  }
  cudaFree(d_src);
  cudaFree(d_out);
  cudaFree(d_len);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (e != cudaSuccess) return trw_cuda_fail(e, "autotune");
  if (st != TRW_OK) return st;
  if (best_out) *best_out = best;
  return TRW_OK;
}
