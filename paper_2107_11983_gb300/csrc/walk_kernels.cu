// Walk kernels: one step of Algorithm 2 (Gather, Move, Update) per call of
// step_once, and the two ways of driving it:
//   walk_plain       the baseline: one thread per walk for its whole length,
//                    one launch for the batch, no refill, direct path stores;
//   walk_persistent  one resident grid; each warp claims chunks of walks from a
//                    device work queue and refills a lane as soon as its walk
//                    ends (Algorithm 4's "replace a completed query" done on
//                    the GPU), stages paths in shared memory and flushes whole
//                    32-byte sectors, and hands long rows to the whole warp.
#include <cstdint>
#include <cuda_runtime.h>

#include "trw_device.cuh"
#include "trw_internal.h"
#include "walk_step.cuh"

namespace trw {

namespace {

using namespace step;

// ------------------------------------------------------------ plain baseline

template <int A>
__global__ void __launch_bounds__(256) walk_plain(DevGraph g, WalkSpec sp, Ctrl* ctrl) {
  if (*(volatile int*)&ctrl->err != 0) return;  // the call was rejected: write nothing
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  unsigned long long moves = 0;
  if (i < sp.nwalks) {
    const int32_t src = sp.sources[i / sp.wps];
    if (src >= 0 && src < g.nv) {
      Walker W;
      walker_init(W, sp.walk_offset + (uint32_t)i, src);
      const int64_t base = sp.endpoints ? i : i * ((int64_t)sp.max_len + 1);
      if (!sp.endpoints) sp.out_paths[base] = src;
      for (;;) {
        int32_t next = -1;
        const int r = step_dispatch<A, false, 0>(g, sp, W, next);
        if (r == kMoved) {
          advance(W, next);
          if (!sp.endpoints) sp.out_paths[base + W.s] = next;
        } else if (r == kRetry) {
          W.att += 1;
        } else {
          if (r == kFail) set_err(ctrl, kErrRejectCap);
          if (r == kBroken) set_err(ctrl, kErrInternal);
          break;
        }
      }
      if (sp.endpoints) sp.out_paths[i] = W.cur;
      sp.out_lengths[i] = W.s + 1;
      moves = (unsigned long long)W.s;
    } else {
      set_err(ctrl, kErrInvalid);
    }
  }
  moves = warp_sum(moves);
  if ((threadIdx.x & 31) == 0 && moves) atomicAdd(&ctrl->moves, moves);
}

// -------------------------------------------------------- persistent kernel

// COOP compiles in the warp-cooperative MetaPath scan and Node2Vec search;
// without it every row stays with its lane (fewer registers).
template <int A, bool COOP>
__global__ void __launch_bounds__(512) walk_persistent(DevGraph g, WalkSpec sp0, const WalkSpec* __restrict__ specs,
                                                       const int64_t* __restrict__ prefix, int nreq, int64_t total,
                                                       Ctrl* ctrl, int chunk, Coop coop) {
  extern __shared__ int32_t stage_mem[];
  if (*(volatile int*)&ctrl->err != 0) return;
  const int lane = threadIdx.x & 31;
  const unsigned lt_mask = (1u << lane) - 1u;

  Stage st;
  st.buf = stage_mem + threadIdx.x * 8;
  st.gpos = 0;
  st.lo = 0;
  Walker W;
  walker_init(W, 0u, 0);
  bool active = false;
  int req = 0;
  int64_t walk = 0;  // walk index within its request

  int64_t wlo = 0, whi = 0;
  bool exhausted = false;
  unsigned long long moves = 0;

  for (;;) {
    // ---- refill idle lanes from the work queue (warp-uniform control flow)
    unsigned idle = __ballot_sync(kFull, !active);
    while (idle != 0u && !exhausted) {
      if (wlo >= whi) {
        unsigned long long base = 0;
        if (lane == 0) base = atomicAdd(&ctrl->head, (unsigned long long)chunk);
        base = __shfl_sync(kFull, base, 0);
        if ((int64_t)base >= total) {
          exhausted = true;
          break;
        }
        wlo = (int64_t)base;
        whi = min((int64_t)base + chunk, total);
      }
      const int take = (int)min((int64_t)__popc(idle), whi - wlo);
      const int rank = __popc(idle & lt_mask);
      if (((idle >> lane) & 1u) && rank < take) {
        const int64_t gidx = wlo + rank;
        if (A == MIXED) {
          req = 0;
          while (req + 1 < nreq && __ldg(prefix + req + 1) <= gidx) ++req;
          walk = gidx - __ldg(prefix + req);
        } else {
          walk = gidx;
        }
        const WalkSpec& sp = (A == MIXED) ? specs[req] : sp0;
        const int32_t src = sp.sources[walk / sp.wps];
        if (src >= 0 && src < g.nv) {
          walker_init(W, sp.walk_offset + (uint32_t)walk, src);
          if (!sp.endpoints) {
            st.gpos = walk * ((int64_t)sp.max_len + 1);
            st.lo = (int)(st.gpos & 7);
            stage_put(st, sp.out_paths, src, (reinterpret_cast<uintptr_t>(sp.out_paths) & 31) == 0);
          }
          active = true;
        } else {
          set_err(ctrl, kErrInvalid);
        }
      }
      wlo += take;
      idle = __ballot_sync(kFull, !active);
    }
    if (!__any_sync(kFull, active)) break;

    // ---- one unit of work per active lane; long rows go to the whole warp
    const WalkSpec& sp = (A == MIXED) ? specs[req] : sp0;
    int r = kIdle;
    int32_t next = -1;
    Pend pend;
    pend.kind = 0;
    pend.res = 0;
    if (active)
      r = step_begin_dispatch<A, false, kFoldDarts>(g, sp, W, next, pend, COOP ? coop : Coop{0x7fffffff, 0x7fffffff});
    if constexpr (COOP) {
      if (__any_sync(kFull, r == kDefer)) {
        warp_resolve(g, r, W, pend);
        if (r == kDefer) r = step_finish(g, sp, W, pend, next);
      }
    }
    if (active) {
      const bool aligned = (reinterpret_cast<uintptr_t>(sp.out_paths) & 31) == 0;
      if (r == kMoved) {
        advance(W, next);
        if (!sp.endpoints) stage_put(st, sp.out_paths, next, aligned);
      } else if (r == kRetry) {
        W.att += 1;
      } else {
        if (r == kFail) set_err(ctrl, kErrRejectCap);
        if (r == kBroken) set_err(ctrl, kErrInternal);
        if (sp.endpoints) {
          __stcs(sp.out_paths + walk, W.cur);
        } else {
          stage_finish(st, sp.out_paths, aligned);
        }
        __stcs(sp.out_lengths + walk, W.s + 1);
        moves += (unsigned long long)W.s;
        active = false;
      }
    }
  }
  moves = warp_sum(moves);
  if (lane == 0 && moves) atomicAdd(&ctrl->moves, moves);
}

// ------------------------------------------------ step-synchronous baseline
// The BSP execution of KnightKing and C-SAW: one launch per step moves every
// live walker by one step (a whole step: the trials of a rejection sampler
// run inside it), and the walkers still alive are appended to the next
// step's list.  Walker state lives in device memory between launches; the
// host reads the live count after every launch.  Same draws, same walks.

struct BspWalker {
  Walker W;
  uint32_t walk;  // index within the request
};

// Finishes a walk: its length (and endpoint) out, its moves counted.
__device__ __forceinline__ void bsp_finish(const WalkSpec& sp, const Walker& W, uint32_t walk,
                                           unsigned long long& moves) {
  if (sp.endpoints) sp.out_paths[walk] = W.cur;
  sp.out_lengths[walk] = W.s + 1;
  moves += (unsigned long long)W.s;
}

// Appends the live lanes' walkers to out with one atomic per warp.
__device__ __forceinline__ void bsp_append(bool live, const BspWalker& b, BspWalker* __restrict__ out,
                                           unsigned long long* n_out) {
  const int lane = threadIdx.x & 31;
  const unsigned mask = __ballot_sync(kFull, live);
  if (mask == 0u) return;
  const int leader = __ffs(mask) - 1;
  unsigned long long base = 0;
  if (lane == leader) base = atomicAdd(n_out, (unsigned long long)__popc(mask));
  base = __shfl_sync(kFull, base, leader);
  if (live) out[base + __popc(mask & ((1u << lane) - 1u))] = b;
}

__global__ void __launch_bounds__(256) bsp_init(DevGraph g, WalkSpec sp, BspWalker* __restrict__ out,
                                                unsigned long long* n_out, Ctrl* ctrl) {
  if (*(volatile int*)&ctrl->err != 0) return;  // the call was rejected: write nothing
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  bool live = false;
  BspWalker b;
  unsigned long long moves = 0;
  if (i < sp.nwalks) {
    const int32_t src = sp.sources[i / sp.wps];
    if (src >= 0 && src < g.nv) {
      walker_init(b.W, sp.walk_offset + (uint32_t)i, src);
      b.walk = (uint32_t)i;
      if (!sp.endpoints) sp.out_paths[i * ((int64_t)sp.max_len + 1)] = src;
      live = sp.max_len > 0;
      if (!live) bsp_finish(sp, b.W, b.walk, moves);
    } else {
      set_err(ctrl, kErrInvalid);
    }
  }
  bsp_append(live, b, out, n_out);
}

template <int A>
__global__ void __launch_bounds__(256) bsp_step(DevGraph g, WalkSpec sp, const BspWalker* __restrict__ in, int64_t n,
                                                BspWalker* __restrict__ out, unsigned long long* n_out, Ctrl* ctrl) {
  if (*(volatile int*)&ctrl->err != 0) return;  // a source was invalid: write nothing more
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  bool live = false;
  BspWalker b;
  unsigned long long moves = 0;
  if (i < n) {
    b = in[i];
    int r;
    int32_t next;
    for (;;) {
      next = -1;
      r = step_dispatch<A, false, 0>(g, sp, b.W, next);
      if (r != kRetry) break;
      b.W.att += 1;
    }
    if (r == kMoved) {
      advance(b.W, next);
      if (!sp.endpoints) sp.out_paths[(int64_t)b.walk * ((int64_t)sp.max_len + 1) + b.W.s] = next;
      live = b.W.s < sp.max_len;
      if (!live) bsp_finish(sp, b.W, b.walk, moves);
    } else {
      if (r == kFail) set_err(ctrl, kErrRejectCap);
      if (r == kBroken) set_err(ctrl, kErrInternal);
      bsp_finish(sp, b.W, b.walk, moves);
    }
  }
  bsp_append(live, b, out, n_out);
  moves = warp_sum(moves);
  if ((threadIdx.x & 31) == 0 && moves) atomicAdd(&ctrl->moves, moves);
}

__global__ void validate_sources(const int32_t* __restrict__ src, int64_t n, int32_t nv, Ctrl* ctrl) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const int32_t v = src[i];
    if (v < 0 || v >= nv) set_err(ctrl, kErrInvalid);
  }
}

__global__ void debug_is_neighbor(DevGraph g, const int32_t* __restrict__ u, const int32_t* __restrict__ v, int64_t n,
                                  uint8_t* __restrict__ out) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const int32_t a = u[i];
    const int32_t off = g.row_ptr[a];
    out[i] = step::is_neighbor(g, a, off, g.row_ptr[a + 1] - off, v[i]) ? 1 : 0;
  }
}

__global__ void debug_philox(const uint4* __restrict__ ctr, int64_t n, uint32_t k0, uint32_t k1,
                             uint4* __restrict__ out) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = philox10(ctr[i], k0, k1);
}

template <typename K>
int blocks_per_sm_of(K kernel, int threads) {
  int nb = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kernel, threads, (size_t)threads * 32) != cudaSuccess)
    return 1;
  return nb > 0 ? nb : 1;
}

}  // namespace

namespace {

// Whether a launch needs the cooperative variant.
bool wants_coop(int algo, const LaunchCfg& cfg) {
  if (algo == MIXED) return true;
  if (algo == METAPATH) return cfg.coop_degree < 0x7fffffff;
  if (is_n2v(algo)) return cfg.search_degree < 0x7fffffff;
  return false;
}

}  // namespace

int persistent_blocks_per_sm(int algo, int block_threads, bool coop) {
  switch (algo) {
    case DEEPWALK: return blocks_per_sm_of(walk_persistent<DEEPWALK, false>, block_threads);
    case DEEPWALK_WEIGHTED: return blocks_per_sm_of(walk_persistent<DEEPWALK_WEIGHTED, false>, block_threads);
    case PPR: return blocks_per_sm_of(walk_persistent<PPR, false>, block_threads);
    case NODE2VEC:
      return coop ? blocks_per_sm_of(walk_persistent<NODE2VEC, true>, block_threads)
                  : blocks_per_sm_of(walk_persistent<NODE2VEC, false>, block_threads);
    case METAPATH:
      return coop ? blocks_per_sm_of(walk_persistent<METAPATH, true>, block_threads)
                  : blocks_per_sm_of(walk_persistent<METAPATH, false>, block_threads);
    case DW_ITS: return blocks_per_sm_of(walk_persistent<DW_ITS, false>, block_threads);
    case DW_REJ: return blocks_per_sm_of(walk_persistent<DW_REJ, false>, block_threads);
    case DW_OREJ: return blocks_per_sm_of(walk_persistent<DW_OREJ, false>, block_threads);
    case N2V_W:
      return coop ? blocks_per_sm_of(walk_persistent<N2V_W, true>, block_threads)
                  : blocks_per_sm_of(walk_persistent<N2V_W, false>, block_threads);
    default:
      return coop ? blocks_per_sm_of(walk_persistent<MIXED, true>, block_threads)
                  : blocks_per_sm_of(walk_persistent<MIXED, false>, block_threads);
  }
}

cudaError_t launch_validate_sources(const int32_t* src, int64_t n, int32_t nv, Ctrl* ctrl, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  int64_t blocks = (n + 255) / 256;
  if (blocks > 4096) blocks = 4096;
  validate_sources<<<(unsigned)blocks, 256, 0, st>>>(src, n, nv, ctrl);
  return cudaGetLastError();
}

cudaError_t launch_walk_plain(const DevGraph& g, const WalkSpec& sp, Ctrl* ctrl, cudaStream_t st, int block) {
  (void)block;
  if (sp.nwalks <= 0) return cudaSuccess;
  const int threads = 256;
  const int64_t blocks = (sp.nwalks + threads - 1) / threads;
  switch (sp.algo) {
    case DEEPWALK: walk_plain<DEEPWALK><<<(unsigned)blocks, threads, 0, st>>>(g, sp, ctrl); break;
    case DEEPWALK_WEIGHTED: walk_plain<DEEPWALK_WEIGHTED><<<(unsigned)blocks, threads, 0, st>>>(g, sp, ctrl); break;
    case PPR: walk_plain<PPR><<<(unsigned)blocks, threads, 0, st>>>(g, sp, ctrl); break;
    case NODE2VEC: walk_plain<NODE2VEC><<<(unsigned)blocks, threads, 0, st>>>(g, sp, ctrl); break;
    case METAPATH: walk_plain<METAPATH><<<(unsigned)blocks, threads, 0, st>>>(g, sp, ctrl); break;
    case DW_ITS: walk_plain<DW_ITS><<<(unsigned)blocks, threads, 0, st>>>(g, sp, ctrl); break;
    case DW_REJ: walk_plain<DW_REJ><<<(unsigned)blocks, threads, 0, st>>>(g, sp, ctrl); break;
    case DW_OREJ: walk_plain<DW_OREJ><<<(unsigned)blocks, threads, 0, st>>>(g, sp, ctrl); break;
    case N2V_W: walk_plain<N2V_W><<<(unsigned)blocks, threads, 0, st>>>(g, sp, ctrl); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

cudaError_t launch_walk_persistent(const DevGraph& g, const WalkSpec& sp, Ctrl* ctrl, cudaStream_t st,
                                   const LaunchCfg& cfg) {
  if (sp.nwalks <= 0) return cudaSuccess;
  const int threads = cfg.block_threads;
  const size_t smem = (size_t)threads * 8 * sizeof(int32_t);
  int64_t blocks = cfg.grid_blocks;
  const int64_t need = (sp.nwalks + threads - 1) / threads;
  if (blocks > need) blocks = need;
  if (blocks < 1) blocks = 1;
  const dim3 grid((unsigned)blocks);
  const Coop coop{cfg.coop_degree, cfg.search_degree};
  const bool cv = wants_coop(sp.algo, cfg);
#define TRW_LAUNCH(A, C) \
  walk_persistent<A, C><<<grid, threads, smem, st>>>(g, sp, nullptr, nullptr, 1, sp.nwalks, ctrl, cfg.chunk, coop)
  switch (sp.algo) {
    case DEEPWALK: TRW_LAUNCH(DEEPWALK, false); break;
    case DEEPWALK_WEIGHTED: TRW_LAUNCH(DEEPWALK_WEIGHTED, false); break;
    case PPR: TRW_LAUNCH(PPR, false); break;
    case NODE2VEC:
      if (cv) TRW_LAUNCH(NODE2VEC, true);
      else TRW_LAUNCH(NODE2VEC, false);
      break;
    case METAPATH:
      if (cv) TRW_LAUNCH(METAPATH, true);
      else TRW_LAUNCH(METAPATH, false);
      break;
    case DW_ITS: TRW_LAUNCH(DW_ITS, false); break;
    case DW_REJ: TRW_LAUNCH(DW_REJ, false); break;
    case DW_OREJ: TRW_LAUNCH(DW_OREJ, false); break;
    case N2V_W:
      if (cv) TRW_LAUNCH(N2V_W, true);
      else TRW_LAUNCH(N2V_W, false);
      break;
    default: return cudaErrorInvalidValue;
  }
#undef TRW_LAUNCH
  return cudaGetLastError();
}

cudaError_t launch_walk_batch(const DevGraph& g, const WalkSpec* d_specs, const int64_t* d_prefix, int nreq,
                              int64_t total, Ctrl* ctrl, cudaStream_t st, const LaunchCfg& cfg) {
  if (total <= 0) return cudaSuccess;
  const int threads = cfg.block_threads;
  const size_t smem = (size_t)threads * 8 * sizeof(int32_t);
  int64_t blocks = cfg.grid_blocks;
  const int64_t need = (total + threads - 1) / threads;
  if (blocks > need) blocks = need;
  if (blocks < 1) blocks = 1;
  WalkSpec dummy{};
  const Coop coop{cfg.coop_degree, cfg.search_degree};
  if (cfg.batch_coop)
    walk_persistent<MIXED, true><<<(unsigned)blocks, threads, smem, st>>>(g, dummy, d_specs, d_prefix, nreq, total,
                                                                           ctrl, cfg.chunk, coop);
  else
    walk_persistent<MIXED, false><<<(unsigned)blocks, threads, smem, st>>>(g, dummy, d_specs, d_prefix, nreq, total,
                                                                            ctrl, cfg.chunk, coop);
  return cudaGetLastError();
}

size_t bsp_walker_bytes() { return sizeof(BspWalker); }

cudaError_t launch_bsp_init(const DevGraph& g, const WalkSpec& sp, void* out, unsigned long long* n_out, Ctrl* ctrl,
                            cudaStream_t st) {
  if (sp.nwalks <= 0) return cudaSuccess;
  bsp_init<<<(unsigned)((sp.nwalks + 255) / 256), 256, 0, st>>>(g, sp, static_cast<BspWalker*>(out), n_out, ctrl);
  return cudaGetLastError();
}

cudaError_t launch_bsp_step(const DevGraph& g, const WalkSpec& sp, const void* in, int64_t n, void* out,
                            unsigned long long* n_out, Ctrl* ctrl, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  const unsigned blocks = (unsigned)((n + 255) / 256);
  const BspWalker* a = static_cast<const BspWalker*>(in);
  BspWalker* b = static_cast<BspWalker*>(out);
  switch (sp.algo) {
    case DEEPWALK: bsp_step<DEEPWALK><<<blocks, 256, 0, st>>>(g, sp, a, n, b, n_out, ctrl); break;
    case DEEPWALK_WEIGHTED: bsp_step<DEEPWALK_WEIGHTED><<<blocks, 256, 0, st>>>(g, sp, a, n, b, n_out, ctrl); break;
    case PPR: bsp_step<PPR><<<blocks, 256, 0, st>>>(g, sp, a, n, b, n_out, ctrl); break;
    case NODE2VEC: bsp_step<NODE2VEC><<<blocks, 256, 0, st>>>(g, sp, a, n, b, n_out, ctrl); break;
    case METAPATH: bsp_step<METAPATH><<<blocks, 256, 0, st>>>(g, sp, a, n, b, n_out, ctrl); break;
    case DW_ITS: bsp_step<DW_ITS><<<blocks, 256, 0, st>>>(g, sp, a, n, b, n_out, ctrl); break;
    case DW_REJ: bsp_step<DW_REJ><<<blocks, 256, 0, st>>>(g, sp, a, n, b, n_out, ctrl); break;
    case DW_OREJ: bsp_step<DW_OREJ><<<blocks, 256, 0, st>>>(g, sp, a, n, b, n_out, ctrl); break;
    case N2V_W: bsp_step<N2V_W><<<blocks, 256, 0, st>>>(g, sp, a, n, b, n_out, ctrl); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

cudaError_t launch_debug_is_neighbor(const DevGraph& g, const int32_t* u, const int32_t* v, int64_t n, uint8_t* out,
                                     cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  int64_t blocks = (n + 255) / 256;
  if (blocks > 4096) blocks = 4096;
  debug_is_neighbor<<<(unsigned)blocks, 256, 0, st>>>(g, u, v, n, out);
  return cudaGetLastError();
}

cudaError_t launch_debug_philox(const uint32_t* d_ctr, int64_t n, uint32_t k0, uint32_t k1, uint32_t* d_out,
                                cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  debug_philox<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(reinterpret_cast<const uint4*>(d_ctr), n, k0, k1,
                                                             reinterpret_cast<uint4*>(d_out));
  return cudaGetLastError();
}

}  // namespace trw
