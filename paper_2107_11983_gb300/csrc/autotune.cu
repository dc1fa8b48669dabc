// Autotuner of the persistent kernel: the GPU counterpart of Section 5.4's
// ring-size tuning, which pre-runs length-10 walks and keeps the ring sizes
// that run them fastest.  Here the knobs are threads per block, resident
// blocks per SM, the work-queue chunk and the degrees from which the warp
// takes over a MetaPath label scan or a Node2Vec neighbour search.  Walk
// results never depend on these knobs.
#include <algorithm>
#include <vector>

#include <cuda_runtime.h>

#include "trw_api_internal.h"

using namespace trw;

extern "C" trw_status trw_autotune(trw_graph* g, trw_algo algo, const trw_params* params, int32_t max_len,
                                   trw_tuning* best_out) {
  if (!g) return trw_fail(TRW_ERR_INVALID, "graph is NULL");
  if (g->nv == 0) return trw_fail(TRW_ERR_INVALID, "empty graph");
  const int32_t len = std::max(1, std::min<int32_t>(max_len, 10));
  // Sources: an even stride over the vertices, enough walks to fill the GPU a few times.
  const int64_t n = std::min<int64_t>(g->nv, (int64_t)g->num_sms * 2048 * 2);
  std::vector<int32_t> src((size_t)n);
  for (int64_t i = 0; i < n; ++i) src[(size_t)i] = (int32_t)((i * g->nv) / n);
  trw_params p;
  if (params) p = *params;
  else trw_params_default(&p);
  p.walks_per_source = 1;
  p.walk_offset = 0;
  WalkSpec sp;
  trw_status st = trw_make_spec(g, algo, &p, n, len, 0x5eedULL, &sp);
  if (st != TRW_OK) return st;
  const size_t out_elems = sp.endpoints ? (size_t)n : (size_t)n * ((size_t)len + 1);
  int32_t *d_src = nullptr, *d_out = nullptr, *d_len = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t e = cudaMalloc(&d_src, sizeof(int32_t) * (size_t)n);
  if (e == cudaSuccess) e = cudaMalloc(&d_out, sizeof(int32_t) * out_elems);
  if (e == cudaSuccess) e = cudaMalloc(&d_len, sizeof(int32_t) * (size_t)n);
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
    // Degree thresholds tried: MetaPath scans (coop_degree) or Node2Vec
    // searches (search_degree); 0x7fffffff keeps every row with its own lane.
    const int kOff = 0x7fffffff;
    const int threads_c[] = {128, 256, 512};
    const int chunk_c[] = {8, 32, 128};
    std::vector<int> deg_c;
    if (algo == TRW_METAPATH && !g->lerec) deg_c = {64, 256, 1024, kOff};
    else if (algo == TRW_NODE2VEC && !g->nh_slots) deg_c = {64, 1024, kOff};
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
            cfg.search_degree = algo == TRW_NODE2VEC ? cd : g->tuning.search_degree;
            float ms_min = 1e30f;
            for (int rep = 0; rep < 3 && e == cudaSuccess; ++rep) {
              e = cudaMemsetAsync(g->ctrl, 0, sizeof(Ctrl), g->stream);
              if (e == cudaSuccess) e = cudaEventRecord(e0, g->stream);
              if (e == cudaSuccess) e = launch_walk_persistent(dg, sp, g->ctrl, g->stream, cfg);
              if (e == cudaSuccess) e = cudaEventRecord(e1, g->stream);
              if (e == cudaSuccess) e = cudaEventSynchronize(e1);
              float ms = 0;
              if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
              if (rep > 0) ms_min = std::min(ms_min, ms);
            }
            if (e != cudaSuccess) break;
            if (ms_min < best_ms) {
              best_ms = ms_min;
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
