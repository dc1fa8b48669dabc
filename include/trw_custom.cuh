/*
 * trw_custom.cuh -- user-defined walks on a loaded graph (header-only CUDA
 * C++ for sm_103a): the paper's programming interface (Section 4.3, "APIs"),
 * where a walk is a sampling method plus the user functions Weight, Update
 * and, for O-REJ, MaxWeight, run by the same engine model as the built-in
 * walks (one persistent grid, a device work queue, per-lane refill).
 *
 * A walk type W provides
 *
 *   static constexpr trw_custom::Sampler sampler;  // NAIVE or OREJ
 *   struct Params;                                // copied to the kernel by value
 *   __device__ static uint32_t weight(const Params&, const trw_custom::Graph&,
 *                                     const trw_custom::Query&, const trw_custom::Edge&);
 *   __device__ static uint32_t max_weight(const Params&);
 *   __device__ static bool update(const Params&, const trw_custom::Graph&,
 *                                 const trw_custom::Query&, const trw_custom::Edge&);
 *
 * weight and max_weight (O-REJ only) are relative chances in any fixed-point
 * scale, max_weight >= 1; a weight above max_weight is accepted like one
 * equal to it.  update is called after every move, with the query already
 * moved (cur is e.dst, length counts the move); true ends the walk there.
 *
 * Draws are those of the built-in walks (trw_draws.cuh): step s, attempt a of
 * walk i is block (walk_offset + i, s, a, 0).  NAIVE moves to E_cur[x],
 * x = below(B, d).  O-REJ throws darts x = below(B, d) and accepts when the
 * 32-bit word y = B.z passes (y + 1) * max_weight <= weight * 2^32 (exact in
 * 64-bit integers), i.e. y < floor(weight * 2^32 / max_weight); after
 * TRW_REJECT_CAP rejected darts the call fails with TRW_ERR_REJECT_CAP.  A
 * walk also ends after max_len moves and at a vertex without out-edges.
 *
 * trw_custom::walk<W>(...) runs a batch on the graph's device (device
 * buffers only) and waits for it.
 */
#ifndef TRW_CUSTOM_CUH
#define TRW_CUSTOM_CUH

#include <cstdint>
#include <cuda_runtime.h>

#include "trw.h"
#include "trw_draws.cuh"

namespace trw_custom {

enum class Sampler { NAIVE, OREJ };

// The graph as user functions see it (device pointers of trw_graph_get_view).
struct Graph {
  const int32_t* row_ptr;  // [nv + 1]
  const int32_t* col;      // [ne]
  const float* weights;    // [ne] or null
  const uint8_t* labels;   // [ne] or null
  int32_t nv, ne;
  int32_t sorted;          // rows strictly increasing

  __device__ int32_t degree(int32_t v) const { return __ldg(row_ptr + v + 1) - __ldg(row_ptr + v); }
  // Is c an out-neighbour of u?  (binary search; needs sorted rows)
  __device__ bool is_neighbor(int32_t u, int32_t c) const {
    int32_t lo = __ldg(row_ptr + u), n = __ldg(row_ptr + u + 1) - lo;
    while (n > 0) {
      const int32_t half = n >> 1;
      if (__ldg(col + lo + half) < c) {
        lo += half + 1;
        n -= half + 1;
      } else {
        n = half;
      }
    }
    return lo < __ldg(row_ptr + u + 1) && __ldg(col + lo) == c;
  }
};

// A walk as user functions see it.
struct Query {
  uint32_t walk;    // Philox walk index (walk_offset + i)
  int32_t source;
  int32_t length;   // moves taken
  int32_t cur;
  int32_t prev;     // -1 before the first move
};

// The edge (cur, dst) at CSR slot index.
struct Edge {
  int32_t src, dst, index;
};

namespace detail {

struct Ctrl {
  unsigned long long head;   // work queue
  unsigned long long moves;
  int err;
  int pad;
};

struct Batch {
  const int32_t* sources;
  int64_t nwalks;
  int32_t wps;
  int32_t max_len;
  uint32_t walk_offset;
  uint64_t seed;
  int32_t* paths;     // [nwalks * (max_len + 1)]
  int32_t* lengths;   // [nwalks]
};

constexpr int kErrInvalid = -1;
constexpr int kErrRejectCap = -6;

// One persistent grid; each warp claims 32 walks at a time from the queue
// and a lane takes the next walk as soon as its own ends.
template <class W>
__global__ void __launch_bounds__(256) custom_walk(Graph g, typename W::Params prm, Batch b, Ctrl* ctrl) {
  const unsigned full = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  bool active = false, exhausted = false;
  int64_t walk = 0, wlo = 0, whi = 0;
  Query q{};
  int32_t off = 0, d = 0;
  uint32_t att = 0;
  unsigned long long moves = 0;
  for (;;) {
    unsigned idle = __ballot_sync(full, !active);
    while (idle != 0u && !exhausted) {
      if (wlo >= whi) {
        unsigned long long base = 0;
        if (lane == 0) base = atomicAdd(&ctrl->head, 32ull);
        base = __shfl_sync(full, base, 0);
        if ((int64_t)base >= b.nwalks) {
          exhausted = true;
          break;
        }
        wlo = (int64_t)base;
        whi = min((int64_t)base + 32, b.nwalks);
      }
      const int take = (int)min((int64_t)__popc(idle), whi - wlo);
      const int rank = __popc(idle & ((1u << lane) - 1u));
      if (((idle >> lane) & 1u) && rank < take) {
        walk = wlo + rank;
        const int32_t src = b.sources[walk / b.wps];
        if (src >= 0 && src < g.nv) {
          q = Query{b.walk_offset + (uint32_t)walk, src, 0, src, -1};
          att = 0;
          b.paths[walk * ((int64_t)b.max_len + 1)] = src;
          active = true;
        } else {
          atomicCAS(&ctrl->err, 0, kErrInvalid);
        }
      }
      wlo += take;
      idle = __ballot_sync(full, !active);
    }
    if (!__any_sync(full, active)) break;
    if (active) {
      bool stop = q.length == b.max_len;
      if (!stop) {
        if (att == 0) {
          off = __ldg(g.row_ptr + q.cur);
          d = __ldg(g.row_ptr + q.cur + 1) - off;
        }
        stop = d == 0;
      }
      if (!stop) {
        const uint4 B = trw_draws::draw(b.seed, q.walk, (uint32_t)q.length, att);
        const int32_t x = (int32_t)trw_draws::below(B, (uint32_t)d);
        const Edge e{q.cur, __ldg(g.col + off + x), off + x};
        bool take = true;
        if (W::sampler == Sampler::OREJ) {
          const unsigned long long mw = W::max_weight(prm);
          const unsigned long long w = W::weight(prm, g, q, e);
          take = ((unsigned long long)B.z + 1ull) * mw <= (w << 32);
        }
        if (take) {
          q.prev = q.cur;
          q.cur = e.dst;
          q.length += 1;
          att = 0;
          b.paths[walk * ((int64_t)b.max_len + 1) + q.length] = e.dst;
          stop = W::update(prm, g, q, e);
        } else if (++att >= (uint32_t)TRW_REJECT_CAP) {
          atomicCAS(&ctrl->err, 0, kErrRejectCap);
          stop = true;
        }
      }
      if (stop) {
        b.lengths[walk] = q.length + 1;
        moves += (unsigned long long)q.length;
        active = false;
      }
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) moves += __shfl_xor_sync(full, moves, o);
  if (lane == 0 && moves) atomicAdd(&ctrl->moves, moves);
}

}  // namespace detail

// Runs n_sources * walks_per_source walks of type W (walk i starts at
// sources[i / walks_per_source]) into device buffers paths [nwalks *
// (max_len + 1)] and lengths [nwalks], on stream (NULL: the legacy default
// stream) of the current device, which must be the graph's, and waits.
// *moves (may be NULL) receives the moves made.  Errors: TRW_ERR_INVALID
// (arguments, another current device, a source outside [0, nv): the outputs
// are then unspecified), TRW_ERR_REJECT_CAP, TRW_ERR_OOM, TRW_ERR_CUDA.
template <class W>
trw_status walk(const trw_graph* graph, const typename W::Params& prm, const int32_t* sources, int64_t n_sources,
                int32_t walks_per_source, int32_t max_len, uint64_t seed, uint32_t walk_offset, int32_t* paths,
                int32_t* lengths, cudaStream_t stream, int64_t* moves) {
  trw_graph_view v;
  trw_status st = trw_graph_get_view(graph, &v);
  if (st != TRW_OK) return st;
  if (n_sources < 0 || walks_per_source < 1 || max_len < 0) return TRW_ERR_INVALID;
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev != v.device) return TRW_ERR_INVALID;  // not the graph's device
  const int64_t nwalks = n_sources * (int64_t)walks_per_source;
  if ((int64_t)walk_offset + nwalks > 4294967296LL) return TRW_ERR_INVALID;
  if (moves) *moves = 0;
  if (nwalks == 0) return TRW_OK;
  if (!sources || !paths || !lengths) return TRW_ERR_INVALID;
  Graph g{v.row_ptr, v.col, v.weights, v.labels, (int32_t)v.nv, (int32_t)v.ne, v.sorted};
  detail::Batch b{sources, nwalks, walks_per_source, max_len, walk_offset, seed, paths, lengths};
  detail::Ctrl* ctrl = nullptr;
  if (cudaMalloc(&ctrl, sizeof(detail::Ctrl)) != cudaSuccess) {
    cudaGetLastError();
    return TRW_ERR_OOM;
  }
  int sms = 1, per_sm = 1;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, v.device);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, detail::custom_walk<W>, 256, 0);
  int64_t blocks = (int64_t)sms * (per_sm > 0 ? per_sm : 1);
  blocks = blocks < (nwalks + 255) / 256 ? blocks : (nwalks + 255) / 256;
  detail::Ctrl host{};
  cudaError_t e = cudaMemsetAsync(ctrl, 0, sizeof(detail::Ctrl), stream);
  if (e == cudaSuccess) {
    detail::custom_walk<W><<<(unsigned)blocks, 256, 0, stream>>>(g, prm, b, ctrl);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(&host, ctrl, sizeof(host), cudaMemcpyDeviceToHost, stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
  cudaFree(ctrl);
  if (e != cudaSuccess) return TRW_ERR_CUDA;
  if (moves) *moves = (int64_t)host.moves;
  if (host.err == detail::kErrRejectCap) return TRW_ERR_REJECT_CAP;
  if (host.err != 0) return TRW_ERR_INVALID;
  return TRW_OK;
}

}  // namespace trw_custom

#endif  // TRW_CUSTOM_CUH
