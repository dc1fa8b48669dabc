// Streaming output: walks whose paths need not fit in device or host memory
// at once (the paper's double-buffered dump of the output, Appendix "Input
// and output").  The batch runs in source-aligned slices; slice i walks into
// device staging buffer i % 2 while the copy engine moves slice i - 1 into
// pinned host buffer (i - 1) % 2 and the calling thread hands slice i - 2's
// buffer to the consumer: walking, copying and consuming overlap, and memory
// stays O(slice).
#include <algorithm>
#include <cstdio>
#include <cstring>
#include <vector>

#include <cuda_runtime.h>

#include "trw_api_internal.h"

using namespace trw;

namespace {

trw_status grow_pinned(void** p, size_t* cap, size_t need) {
  if (*cap >= need && *p) return TRW_OK;
  if (*p) cudaFreeHost(*p);
  *p = nullptr;
  *cap = 0;
  const size_t bytes = std::max<size_t>(need, 64);
  if (trw_host_alloc(p, bytes, cudaHostAllocDefault) != cudaSuccess) {
    cudaGetLastError();
    *p = nullptr;
    return trw_fail(TRW_ERR_OOM, "pinned host allocation of %zu bytes failed", bytes);
  }
  *cap = bytes;
  return TRW_OK;
}

// Waits for everything the call queued, so that no copy or kernel still
// reads or writes the staging buffers when the call returns.
void drain(cudaStream_t a, cudaStream_t b) {
  cudaStreamSynchronize(a);
  cudaStreamSynchronize(b);
}

}  // namespace

void trw_free_stream_buffers(trw_graph* g) {
  for (int b = 0; b < 2; ++b) {
    if (g->pin_paths[b]) cudaFreeHost(g->pin_paths[b]);
    if (g->pin_lens[b]) cudaFreeHost(g->pin_lens[b]);
    g->pin_paths[b] = g->pin_lens[b] = nullptr;
    g->pin_paths_cap[b] = g->pin_lens_cap[b] = 0;
  }
  if (g->pin_ctrl) cudaFreeHost(g->pin_ctrl);
  g->pin_ctrl = nullptr;
}

extern "C" trw_status trw_walk_stream(trw_graph* g, trw_algo algo, const trw_params* params, const int32_t* sources,
                                      int64_t n_sources, int32_t max_len, uint64_t seed, int64_t slice_walks,
                                      trw_stream_fn fn, void* user) {
  if (!g || !fn) return trw_fail(TRW_ERR_INVALID, "NULL graph or consumer");
  if (trw_status dc = trw_check_device(g); dc != TRW_OK) return dc;
  if (slice_walks < 1) return trw_fail(TRW_ERR_INVALID, "slice_walks must be >= 1");
  WalkSpec sp;
  trw_status st = trw_make_spec(g, algo, params, n_sources, max_len, seed, &sp);
  if (st != TRW_OK) return st;
  if (n_sources > 0 && !sources) return trw_fail(TRW_ERR_INVALID, "NULL sources");
  std::lock_guard<std::mutex> lk(g->mu);
  g->last.walks = sp.nwalks;
  g->last.moves = 0;
  g->last.kernel_ms = 0;
  g->last.launches = 0;
  g->timed = false;
  if (sp.nwalks == 0) return TRW_OK;
  cudaStream_t stream = g->stream, cs = g->copy_stream;
  const int64_t wps = (int64_t)sp.wps;
  const int64_t row = sp.endpoints ? 1 : (int64_t)max_len + 1;
  const int64_t src_per = std::max<int64_t>(1, slice_walks / wps);
  const int64_t walks_per = src_per * wps;

  // Sources on the device, checked before anything is walked.
  const int32_t* d_src = sources;
  if (!trw_is_device_ptr(sources)) {
    if (!trw_sources_in_range(sources, n_sources, g->nv)) return trw_fail(TRW_ERR_INVALID, "a source is outside [0, nv)");
    st = trw_grow((void**)&g->src_stage, &g->src_cap, sizeof(int32_t) * (size_t)n_sources);
    if (st != TRW_OK) return st;
    CUDA_TRY(cudaMemcpyAsync(g->src_stage, sources, sizeof(int32_t) * (size_t)n_sources, cudaMemcpyHostToDevice, stream),
             "copy sources");
    d_src = g->src_stage;
  } else {
    Ctrl c;
    CUDA_TRY(cudaMemsetAsync(g->ctrl, 0, sizeof(Ctrl), stream), "reset ctrl");
    CUDA_TRY(launch_validate_sources(d_src, n_sources, (int32_t)g->nv, g->ctrl, stream), "validate sources");
    CUDA_TRY(cudaMemcpyAsync(&c, g->ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, stream), "read status");
    CUDA_TRY(cudaStreamSynchronize(stream), "validate sources");
    if (c.err != 0) return trw_fail(TRW_ERR_INVALID, "a source vertex is outside [0, nv)");
  }

  st = trw_grow((void**)&g->out_stage, &g->out_cap, sizeof(int32_t) * (size_t)(2 * walks_per * row));
  if (st == TRW_OK) st = trw_grow((void**)&g->len_stage, &g->len_cap, sizeof(int32_t) * (size_t)(2 * walks_per));
  for (int b = 0; b < 2 && st == TRW_OK; ++b) {
    st = grow_pinned((void**)&g->pin_paths[b], &g->pin_paths_cap[b], sizeof(int32_t) * (size_t)(walks_per * row));
    if (st == TRW_OK)
      st = grow_pinned((void**)&g->pin_lens[b], &g->pin_lens_cap[b], sizeof(int32_t) * (size_t)walks_per);
  }
  if (st == TRW_OK && !g->pin_ctrl) {
    size_t cap = 0;
    st = grow_pinned((void**)&g->pin_ctrl, &cap, 2 * sizeof(Ctrl));
  }
  if (st != TRW_OK) return st;

  const DevGraph dg = trw_dev_graph(g);
  const LaunchCfg cfg = trw_launch_cfg(g, sp.algo);
  const bool coop = (sp.algo == METAPATH && cfg.coop_degree < 0x7fffffff) ||
                    (is_n2v(sp.algo) && cfg.search_degree < 0x7fffffff);
  Ctrl* kc[2] = {g->ctrl, g->ctrl2};
  const int64_t nslices = (n_sources + src_per - 1) / src_per;
  int64_t moves = 0;
  trw_kernel kernel = TRW_KERNEL_PERSISTENT;  // of the last slice
  CUDA_TRY(cudaEventRecord(g->ev0, stream), "event");
  for (int64_t i = 0; i <= nslices; ++i) {
    if (i < nslices) {
      const int b = (int)(i & 1);
      const int64_t s0 = i * src_per, s1 = std::min(n_sources, s0 + src_per);
      WalkSpec sl = sp;
      sl.sources = d_src + s0;
      sl.nwalks = (s1 - s0) * wps;
      sl.walk_offset = sp.walk_offset + (uint32_t)(s0 * wps);
      sl.out_paths = g->out_stage + (size_t)b * (size_t)(walks_per * row);
      sl.out_lengths = g->len_stage + (size_t)b * (size_t)walks_per;
      // device buffer b is free once slice i - 2 was copied out
      if (i >= 2) CUDA_TRY(cudaStreamWaitEvent(stream, g->ev_copied[b], 0), "wait for a drained buffer");
      CUDA_TRY(cudaMemsetAsync(kc[b], 0, sizeof(Ctrl), stream), "reset ctrl");
      if (!coop && sl.nwalks <= (int64_t)cfg.grid_blocks * cfg.block_threads) {
        CUDA_TRY(launch_walk_plain(dg, sl, kc[b], stream, 256), "plain walk launch");
        kernel = TRW_KERNEL_PLAIN;
      } else {
        CUDA_TRY(launch_walk_persistent(dg, sl, kc[b], stream, cfg), "persistent walk launch");
        kernel = TRW_KERNEL_PERSISTENT;
      }
      CUDA_TRY(cudaEventRecord(g->ev_walked[b], stream), "event");
      // host buffer b is free: slice i - 2 was consumed in the previous iteration
      CUDA_TRY(cudaStreamWaitEvent(cs, g->ev_walked[b], 0), "wait for a walked slice");
      CUDA_TRY(cudaMemcpyAsync(g->pin_paths[b], sl.out_paths, sizeof(int32_t) * (size_t)(sl.nwalks * row),
                               cudaMemcpyDeviceToHost, cs),
               "copy paths");
      CUDA_TRY(cudaMemcpyAsync(g->pin_lens[b], sl.out_lengths, sizeof(int32_t) * (size_t)sl.nwalks,
                               cudaMemcpyDeviceToHost, cs),
               "copy lengths");
      CUDA_TRY(cudaMemcpyAsync(g->pin_ctrl + b, kc[b], sizeof(Ctrl), cudaMemcpyDeviceToHost, cs), "copy status");
      CUDA_TRY(cudaEventRecord(g->ev_copied[b], cs), "event");
    }
    if (i >= 1) {
      // consume slice i - 1 while slice i walks
      const int64_t j = i - 1;
      const int bj = (int)(j & 1);
      const cudaError_t e = cudaEventSynchronize(g->ev_copied[bj]);
      if (e != cudaSuccess) {
        drain(stream, cs);
        return trw_cuda_fail(e, "walk slice");
      }
      const Ctrl c = g->pin_ctrl[bj];
      if (c.err != 0) {
        drain(stream, cs);
        if (c.err == kErrRejectCap)
          return trw_fail(TRW_ERR_REJECT_CAP, "a rejection step exceeded %d trials", TRW_REJECT_CAP);
        if (c.err == kErrInvalid) return trw_fail(TRW_ERR_INVALID, "a source vertex is outside [0, nv)");
        return trw_fail(TRW_ERR_INTERNAL, "device status %d", c.err);
      }
      moves += (int64_t)c.moves;
      const int64_t first = j * src_per * wps;
      const int64_t n = (std::min(n_sources, (j + 1) * src_per) - j * src_per) * wps;
      if (fn(user, first, n, g->pin_paths[bj], g->pin_lens[bj]) != 0) {
        drain(stream, cs);
        g->last.moves = moves;
        return trw_fail(TRW_ERR_STOPPED, "the consumer stopped the stream after walk %lld", (long long)(first + n));
      }
    }
  }
  CUDA_TRY(cudaEventRecord(g->ev1, stream), "event");
  CUDA_TRY(cudaStreamSynchronize(stream), "walk stream");
  float ms = 0.f;
  if (cudaEventElapsedTime(&ms, g->ev0, g->ev1) == cudaSuccess) g->last.kernel_ms = ms;
  g->last.moves = moves;
  g->last.kernel = kernel;
  g->last.launches = (int32_t)std::min<int64_t>(nslices, INT32_MAX);
  g->last.grid_blocks = cfg.grid_blocks;
  g->last.block_threads = cfg.block_threads;
  return TRW_OK;
}

namespace {

// The file consumer of trw_walk_to_file: compacts each slice (the vertices of
// every walk, walk after walk) and appends it and the lengths to the files.
struct FileSink {
  FILE* paths = nullptr;
  FILE* lengths = nullptr;
  int64_t row = 0;
  bool endpoints = false;
  std::vector<int32_t> buf;
  bool failed = false;
};

int file_sink(void* user, int64_t first, int64_t n, const int32_t* paths, const int32_t* lengths) {
  (void)first;
  FileSink* s = static_cast<FileSink*>(user);
  size_t count = 0;
  const int32_t* data = paths;
  if (s->endpoints) {
    count = (size_t)n;
  } else {
    size_t total = 0;
    for (int64_t i = 0; i < n; ++i) total += (size_t)lengths[i];
    s->buf.resize(total);
    for (int64_t i = 0; i < n; ++i) {
      std::memcpy(s->buf.data() + count, paths + i * s->row, sizeof(int32_t) * (size_t)lengths[i]);
      count += (size_t)lengths[i];
    }
    data = s->buf.data();
  }
  if (std::fwrite(data, sizeof(int32_t), count, s->paths) != count ||
      std::fwrite(lengths, sizeof(int32_t), (size_t)n, s->lengths) != (size_t)n) {
    s->failed = true;
    return 1;
  }
  return 0;
}

}  // namespace

extern "C" trw_status trw_walk_to_file(trw_graph* g, trw_algo algo, const trw_params* params, const int32_t* sources,
                                       int64_t n_sources, int32_t max_len, uint64_t seed, const char* paths_file,
                                       const char* lengths_file) {
  if (!g || !paths_file || !lengths_file) return trw_fail(TRW_ERR_INVALID, "NULL argument");
  if (trw_status dc = trw_check_device(g); dc != TRW_OK) return dc;
  WalkSpec sp;
  trw_status st = trw_make_spec(g, algo, params, n_sources, max_len, seed, &sp);
  if (st != TRW_OK) return st;
  FileSink s;
  s.row = sp.endpoints ? 1 : (int64_t)max_len + 1;
  s.endpoints = sp.endpoints != 0;
  s.paths = std::fopen(paths_file, "wb");
  s.lengths = s.paths ? std::fopen(lengths_file, "wb") : nullptr;
  if (!s.paths || !s.lengths) {
    if (s.paths) std::fclose(s.paths);
    return trw_fail(TRW_ERR_IO, "cannot open %s or %s for writing", paths_file, lengths_file);
  }
  // slices of about 64 MB of padded paths
  const int64_t slice = std::max<int64_t>(1, ((int64_t)64 << 20) / (int64_t)(sizeof(int32_t) * s.row));
  st = trw_walk_stream(g, algo, params, sources, n_sources, max_len, seed, slice, file_sink, &s);
  const bool closed = std::fclose(s.paths) == 0 && std::fclose(s.lengths) == 0;
  if (s.failed || (st == TRW_OK && !closed)) return trw_fail(TRW_ERR_IO, "writing %s or %s failed", paths_file, lengths_file);
  return st;
}
