// Compact path output (TRW_OUT_COMPACT): the vertices of walk 0, then of walk
// 1, ... with no padding, so that a walk that stops early (a dead end, a PPR
// coin, a missing MetaPath label) ships no unused row entries across the
// host link, which bounds end-to-end throughput.  The batch walks in slices
// into padded device staging; each slice is compacted on the device (an
// exclusive scan of its lengths, then a row-prefix copy) while the next one
// walks, and its compact block is copied to the caller's buffer at the
// running offset once its total is known on the host.
#include <algorithm>
#include <cstdint>

#include <cuda_runtime.h>

#include "trw_api_internal.h"

using namespace trw;

namespace {

constexpr int kScanBlock = 1024;  // lengths per scan block

// Exclusive prefix of the lengths within each block of 1024 walks, and the
// block totals.
__global__ void __launch_bounds__(kScanBlock) scan_blocks(const int32_t* __restrict__ len, int64_t n,
                                                          int64_t* __restrict__ off, int64_t* __restrict__ bsum) {
  __shared__ long long warp_tot[kScanBlock / 32];
  const int64_t i = (int64_t)blockIdx.x * kScanBlock + threadIdx.x;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const long long v = i < n ? (long long)len[i] : 0;
  long long incl = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const long long t = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += t;
  }
  if (lane == 31) warp_tot[wid] = incl;
  __syncthreads();
  if (wid == 0) {
    long long w = warp_tot[lane];
    long long wi = w;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const long long t = __shfl_up_sync(0xffffffffu, wi, o);
      if (lane >= o) wi += t;
    }
    warp_tot[lane] = wi - w;  // exclusive prefix of the warp totals
    if (lane == 31) bsum[blockIdx.x] = wi;
  }
  __syncthreads();
  if (i < n) off[i] = warp_tot[wid] + incl - v;
}

// The block totals turned into their exclusive prefix (one block, a carry
// across chunks of 1024); *total receives the sum.
__global__ void __launch_bounds__(kScanBlock) scan_sums(int64_t* __restrict__ bsum, int64_t nb,
                                                        int64_t* __restrict__ total) {
  __shared__ long long warp_tot[kScanBlock / 32];
  __shared__ long long carry;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  for (int64_t base = 0; base < nb; base += kScanBlock) {
    const int64_t i = base + threadIdx.x;
    const long long v = i < nb ? bsum[i] : 0;
    long long incl = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const long long t = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += t;
    }
    if (lane == 31) warp_tot[wid] = incl;
    __syncthreads();
    if (wid == 0) {
      long long w = warp_tot[lane];
      long long wi = w;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const long long t = __shfl_up_sync(0xffffffffu, wi, o);
        if (lane >= o) wi += t;
      }
      warp_tot[lane] = wi - w;
    }
    __syncthreads();
    const long long c = carry;
    if (i < nb) bsum[i] = c + warp_tot[wid] + incl - v;
    __syncthreads();
    if (threadIdx.x == kScanBlock - 1) carry = c + warp_tot[wid] + incl;
    __syncthreads();
  }
  if (threadIdx.x == 0) *total = carry;
}

// Row prefixes of the padded rows to their compact positions.
__global__ void compact_rows(const int32_t* __restrict__ padded, const int32_t* __restrict__ len,
                             const int64_t* __restrict__ off, const int64_t* __restrict__ bsum, int64_t n, int32_t row,
                             int32_t* __restrict__ out) {
  const int64_t total = n * (int64_t)row;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e / row;
    const int32_t k = (int32_t)(e - i * row);
    if (k < len[i]) out[bsum[i / kScanBlock] + off[i] + k] = padded[e];
  }
}

}  // namespace

trw_status trw_walk_compact(trw_graph* g, WalkSpec sp, trw_kernel kernel, const int32_t* d_src, int64_t n_sources,
                            int32_t* out_paths, int32_t* out_lengths, cudaStream_t stream) {
  const int64_t wps = (int64_t)sp.wps;
  const int64_t nwalks = sp.nwalks;
  const int32_t row = sp.max_len + 1;
  // Slices of about 2^18 walks, at most 16, on one compute stream: each
  // slice's walk and compaction run in order while the copy engine drains
  // the previous slice.  (Two compute streams, as the padded output uses,
  // were slower here: the compaction kernels of one slice then compete with
  // the other slice's walk.)
  int64_t nslices = std::max<int64_t>(1, std::min<int64_t>(16, nwalks >> 18));
  const int64_t src_per = (n_sources + nslices - 1) / nslices;
  const int64_t walks_per = src_per * wps;
  const int64_t nb_per = (walks_per + kScanBlock - 1) / kScanBlock;
  const size_t pad_bytes = sizeof(int32_t) * (size_t)(walks_per * row);
  trw_status st = trw_grow((void**)&g->out_stage, &g->out_cap, 2 * pad_bytes);
  if (st == TRW_OK) st = trw_grow((void**)&g->len_stage, &g->len_cap, sizeof(int32_t) * (size_t)(2 * walks_per));
  if (st == TRW_OK) st = trw_grow((void**)&g->cmp_stage, &g->cmp_cap, 2 * pad_bytes);
  if (st == TRW_OK)
    st = trw_grow((void**)&g->cmp_scratch, &g->cmp_scratch_cap,
                  sizeof(int64_t) * (size_t)(2 * (walks_per + nb_per) + 2));
  if (st != TRW_OK) return st;
  if (!g->cmp_host) CUDA_TRY(trw_host_alloc((void**)&g->cmp_host, 2 * sizeof(int64_t), cudaHostAllocDefault), "pinned totals");
  const DevGraph dg = trw_dev_graph(g);
  const LaunchCfg cfg = trw_launch_cfg(g, sp.algo);
  cudaStream_t cs = g->copy_stream;
  int64_t* off_d[2] = {g->cmp_scratch, g->cmp_scratch + walks_per};
  int64_t* bsum_d[2] = {g->cmp_scratch + 2 * walks_per, g->cmp_scratch + 2 * walks_per + nb_per};
  int64_t* tot_d = g->cmp_scratch + 2 * (walks_per + nb_per);
  CUDA_TRY(cudaMemsetAsync(g->ctrl, 0, sizeof(Ctrl), stream), "reset ctrl");
  CUDA_TRY(cudaEventRecord(g->ev0, stream), "event");
  int64_t host_off = 0, slice_first[2] = {0, 0}, slice_n[2] = {0, 0};
  for (int64_t i = 0; i <= nslices; ++i) {
    if (i < nslices) {
      const int b = (int)(i & 1);
      const int64_t s0 = i * src_per, s1 = std::min(n_sources, s0 + src_per);
      WalkSpec sl = sp;
      sl.sources = d_src + s0;
      sl.nwalks = std::max<int64_t>(0, s1 - s0) * wps;
      sl.walk_offset = sp.walk_offset + (uint32_t)(s0 * wps);
      sl.out_paths = g->out_stage + (size_t)b * (size_t)(walks_per * row);
      sl.out_lengths = g->len_stage + (size_t)b * (size_t)walks_per;
      int32_t* cmp = g->cmp_stage + (size_t)b * (size_t)(walks_per * row);
      slice_first[b] = s0 * wps;
      slice_n[b] = sl.nwalks;
      // staging b is free once slice i - 2 was copied out
      if (i >= 2) CUDA_TRY(cudaStreamWaitEvent(stream, g->ev_copied[b], 0), "wait for a drained buffer");
      CUDA_TRY(cudaMemsetAsync(&g->ctrl->head, 0, sizeof(unsigned long long), stream), "reset queue");
      if (sl.nwalks > 0) {
        if (kernel == TRW_KERNEL_PLAIN) CUDA_TRY(launch_walk_plain(dg, sl, g->ctrl, stream, 256), "plain walk launch");
        else CUDA_TRY(launch_walk_persistent(dg, sl, g->ctrl, stream, cfg), "persistent walk launch");
        const int64_t nb = (sl.nwalks + kScanBlock - 1) / kScanBlock;
        scan_blocks<<<(unsigned)nb, kScanBlock, 0, stream>>>(sl.out_lengths, sl.nwalks, off_d[b], bsum_d[b]);
        scan_sums<<<1, kScanBlock, 0, stream>>>(bsum_d[b], nb, tot_d + b);
        int64_t blocks = (sl.nwalks * row + 255) / 256;
        if (blocks > 8 * 152) blocks = 8 * 152;
        compact_rows<<<(unsigned)blocks, 256, 0, stream>>>(sl.out_paths, sl.out_lengths, off_d[b], bsum_d[b], sl.nwalks,
                                                           row, cmp);
        CUDA_TRY(cudaGetLastError(), "compaction launch");
      } else {
        CUDA_TRY(cudaMemsetAsync(tot_d + b, 0, sizeof(int64_t), stream), "empty slice");
      }
      CUDA_TRY(cudaMemcpyAsync(g->cmp_host + b, tot_d + b, sizeof(int64_t), cudaMemcpyDeviceToHost, stream),
               "read slice total");
      CUDA_TRY(cudaEventRecord(g->ev_walked[b], stream), "event");
    }
    if (i >= 1) {
      // slice i - 1: its total is on the host once its compaction is done
      const int bj = (int)((i - 1) & 1);
      CUDA_TRY(cudaEventSynchronize(g->ev_walked[bj]), "compacted slice");
      const int64_t tot = g->cmp_host[bj];
      CUDA_TRY(cudaStreamWaitEvent(cs, g->ev_walked[bj], 0), "wait for a compacted slice");
      if (tot > 0)
        CUDA_TRY(cudaMemcpyAsync(out_paths + host_off, g->cmp_stage + (size_t)bj * (size_t)(walks_per * row),
                                 sizeof(int32_t) * (size_t)tot, cudaMemcpyDefault, cs),
                 "copy paths");
      if (slice_n[bj] > 0)
        CUDA_TRY(cudaMemcpyAsync(out_lengths + slice_first[bj], g->len_stage + (size_t)bj * (size_t)walks_per,
                                 sizeof(int32_t) * (size_t)slice_n[bj], cudaMemcpyDefault, cs),
                 "copy lengths");
      CUDA_TRY(cudaEventRecord(g->ev_copied[bj], cs), "event");
      host_off += tot;
    }
  }
  CUDA_TRY(cudaStreamWaitEvent(stream, g->ev_copied[(nslices - 1) & 1], 0), "join");
  CUDA_TRY(cudaEventRecord(g->ev1, stream), "event");
  g->timed = true;
  g->last.grid_blocks = cfg.grid_blocks;
  g->last.block_threads = cfg.block_threads;
  g->last.kernel = kernel == TRW_KERNEL_PLAIN ? TRW_KERNEL_PLAIN : TRW_KERNEL_PERSISTENT;
  g->last.launches = (int32_t)nslices;
  CUDA_TRY(cudaStreamSynchronize(cs), "copy stream");
  return TRW_OK;
}
