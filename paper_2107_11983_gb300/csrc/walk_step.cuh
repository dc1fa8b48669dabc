// One step of Algorithm 2 for one walker (Gather, Move, Update), the path
// staging of the persistent kernels, and warp helpers: shared by the batch
// kernels (walk_kernels.cu) and the serving kernel (serve.cu).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "trw_device.cuh"

namespace trw {
namespace step {

constexpr unsigned kFull = 0xffffffffu;

struct Walker {
  uint32_t w;       // Philox walk index (counter word 0)
  int32_t s;        // moves taken
  int32_t cur;
  int32_t prev;
  int32_t off, d;   // CSR row of cur (valid once attempt 0 of the step loaded it)
  int32_t poff, pd; // CSR row of prev
  uint32_t att;     // rejection trial within the step
};

enum StepResult : int { kMoved = 0, kStop = 1, kRetry = 2, kFail = 3, kBroken = 4 };

__device__ __forceinline__ void set_err(Ctrl* c, int e) { atomicCAS(&c->err, 0, e); }

// ---------------------------------------------------------- MetaPath Gather
// Weight(Q, e) is 1 when l_e equals the step's schema label, else 0.  Labels
// are scanned as aligned 32-bit words (the label array is padded by 16 bytes).

__device__ __forceinline__ uint32_t byte_mask(int64_t wa, int64_t lo, int64_t hi) {
  uint32_t m = 0xffffffffu;
  if (wa < lo) m &= 0xffffffffu << (8 * (int)(lo - wa));
  if (wa + 4 > hi) m &= 0xffffffffu >> (8 * (int)(wa + 4 - hi));
  return m;
}

__device__ __forceinline__ uint32_t label_count_serial(const uint8_t* __restrict__ labels, int64_t lo, int64_t hi,
                                                       uint32_t hrep) {
  uint32_t cnt = 0;
  const uint32_t* L32 = reinterpret_cast<const uint32_t*>(labels);
  for (int64_t wa = lo & ~int64_t(3); wa < hi; wa += 4) {
    const uint32_t eq = __vcmpeq4(__ldg(L32 + (wa >> 2)), hrep) & byte_mask(wa, lo, hi);
    cnt += __popc(eq) >> 3;
  }
  return cnt;
}

// Index (relative to lo) of the r-th (0-based) matching label.
__device__ __forceinline__ int32_t label_select_serial(const uint8_t* __restrict__ labels, int64_t lo, int64_t hi,
                                                       uint32_t hrep, uint32_t r) {
  const uint32_t* L32 = reinterpret_cast<const uint32_t*>(labels);
  for (int64_t wa = lo & ~int64_t(3); wa < hi; wa += 4) {
    uint32_t eq = __vcmpeq4(__ldg(L32 + (wa >> 2)), hrep) & byte_mask(wa, lo, hi);
    const uint32_t c = __popc(eq) >> 3;
    if (r < c) {
      for (int b = 0; b < 4; ++b) {
        if ((eq >> (8 * b)) & 0xffu) {
          if (r == 0) return (int32_t)(wa + b - lo);
          --r;
        }
      }
    }
    r -= c;
  }
  return -1;
}

// IsNeighbor(c, prev): lower-bound search of c in the sorted row of prev.
__device__ __forceinline__ bool is_neighbor_serial(const int32_t* __restrict__ col, int32_t poff, int32_t pd,
                                                   int32_t c) {
  int32_t lo = 0, n = pd;
  while (n > 0) {
    const int32_t half = n >> 1;
    if (ldg(col + poff + lo + half) < c) {
      lo += half + 1;
      n -= half + 1;
    } else {
      n = half;
    }
  }
  return lo < pd && ldg(col + poff + lo) == c;
}

// O-REJ acceptance for Node2Vec's Weight (Eq. 1, Section 4.2 listing's rules):
// MaxWeight on the first step, 1/a back to prev, 1 to a neighbour of prev,
// 1/b otherwise.  The class is only resolved when the 32-bit dart y falls
// between the two non-return thresholds.
template <typename NbFn>
__device__ __forceinline__ bool n2v_accept(const WalkSpec& sp, const Walker& W, int32_t c, uint32_t y, NbFn nb) {
  if (W.s == 0) return true;
  if (c == W.prev) return (uint64_t)y < sp.T_ret;
  if ((uint64_t)y < sp.T_lo) return true;
  if ((uint64_t)y >= sp.T_hi) return false;
  return (uint64_t)y < (nb() ? sp.T_nb : sp.T_far);
}

// One unit of work for one walker, thread-serial: a full step, or one
// rejection trial of a Node2Vec step.
// CHECK adds range checks of the walker's vertex and of the row it loads
// before any access through them (kBroken instead of an out-of-range read).
template <int A, bool CHECK = false>
__device__ __forceinline__ int step_serial(const DevGraph& g, const WalkSpec& sp, Walker& W, int32_t& next) {
  if (W.s == sp.max_len) return kStop;                         // Update: target length reached
  const uint4 B = draw_block(sp, W.w, (uint32_t)W.s, W.att);
  if (A == PPR && (uint64_t)B.w < sp.T_stop) return kStop;     // Update: PPR stop coin
  if (W.att == 0) {
    if (CHECK && (uint32_t)W.cur >= (uint32_t)g.nv) return kBroken;
    W.off = ldg(g.row_ptr + W.cur);
    W.d = ldg(g.row_ptr + W.cur + 1) - W.off;
    if (CHECK && (W.off < 0 || W.d < 0 || (int64_t)W.off + W.d > (int64_t)g.ne)) return kBroken;
  }
  if (W.d == 0) return kStop;                                  // dead end
  if (A == DEEPWALK || A == PPR) {
    // NAIVE: E_v[x], x uniform in [0, d_v).
    next = ldg(g.col + W.off + below(B, (uint32_t)W.d));
    return kMoved;
  } else if (A == DEEPWALK_WEIGHTED) {
    // ALIAS generation from the stored C_v (no Gather for static walks).
    const uint4 r = ldg(g.alias + W.off + below(B, (uint32_t)W.d));
    const int32_t pick = (B.z < r.x) ? (int32_t)r.y : (int32_t)r.z;
    if (pick < 0) return kStop;                                // no positive weight
    next = pick;
    return kMoved;
  } else if (A == METAPATH) {
    // Gather (0/1 weights by label) then ITS generation: the r-th match.
    const uint32_t h = schema_label(sp, (uint32_t)W.s % sp.schema_len);
    const uint32_t hrep = h * 0x01010101u;
    const int64_t lo = W.off, hi = (int64_t)W.off + W.d;
    const uint32_t cnt = label_count_serial(g.labels, lo, hi, hrep);
    if (cnt == 0) return kStop;
    const uint32_t r = below(B, cnt);
    const int32_t j = label_select_serial(g.labels, lo, hi, hrep, r);
    if (j < 0) return kBroken;                                 // count and select disagree: internal error
    next = ldg(g.col + W.off + j);
    return kMoved;
  } else {  // NODE2VEC, O-REJ
    const int32_t c = ldg(g.col + W.off + below(B, (uint32_t)W.d));
    if (n2v_accept(sp, W, c, B.z, [&] { return is_neighbor_serial(g.col, W.poff, W.pd, c); })) {
      next = c;
      return kMoved;
    }
    return (W.att + 1 >= kRejectCap) ? kFail : kRetry;
  }
}

__device__ __forceinline__ void advance(Walker& W, int32_t next) {
  W.prev = W.cur;
  W.poff = W.off;
  W.pd = W.d;
  W.cur = next;
  W.s += 1;
  W.att = 0;
}

template <int A, bool CHECK = false>
__device__ __forceinline__ int step_dispatch(const DevGraph& g, const WalkSpec& sp, Walker& W, int32_t& next) {
  if constexpr (A != MIXED) {
    return step_serial<A, CHECK>(g, sp, W, next);
  } else {
    switch (sp.algo) {
      case DEEPWALK: return step_serial<DEEPWALK, CHECK>(g, sp, W, next);
      case DEEPWALK_WEIGHTED: return step_serial<DEEPWALK_WEIGHTED, CHECK>(g, sp, W, next);
      case PPR: return step_serial<PPR, CHECK>(g, sp, W, next);
      case NODE2VEC: return step_serial<NODE2VEC, CHECK>(g, sp, W, next);
      case METAPATH: return step_serial<METAPATH, CHECK>(g, sp, W, next);
      default: return kBroken;
    }
  }
}

__device__ __forceinline__ unsigned long long warp_sum(unsigned long long v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
  return v;
}

// Path staging: each thread owns 8 int32 of shared memory that mirror one
// aligned 32-byte sector of out_paths.  A full sector leaves as two 16-byte
// streaming stores; a partial one (the walk's first or last sector, which it
// may share with a neighbouring walk) leaves element by element.
struct Stage {
  int32_t* buf;     // 8 entries in shared memory
  int64_t gpos;     // element index of the next vertex in out_paths
  int lo;           // first slot of the current sector that belongs to this walk
};

__device__ __forceinline__ void stage_flush(Stage& st, int32_t* __restrict__ out, int hi_slot, bool aligned) {
  const int64_t sec = (st.gpos - 1) & ~int64_t(7);
  if (st.lo == 0 && hi_slot == 8 && aligned && ((reinterpret_cast<uintptr_t>(out + sec) & 31) == 0)) {
    const int4 a = *reinterpret_cast<const int4*>(st.buf);
    const int4 b = *reinterpret_cast<const int4*>(st.buf + 4);
    __stcs(reinterpret_cast<int4*>(out + sec), a);
    __stcs(reinterpret_cast<int4*>(out + sec + 4), b);
  } else {
    for (int k = st.lo; k < hi_slot; ++k) __stcs(out + sec + k, st.buf[k]);
  }
}

__device__ __forceinline__ void stage_put(Stage& st, int32_t* __restrict__ out, int32_t v, bool aligned) {
  const int slot = (int)(st.gpos & 7);
  st.buf[slot] = v;
  st.gpos += 1;
  if (slot == 7) {
    stage_flush(st, out, 8, aligned);
    st.lo = 0;
  }
}

__device__ __forceinline__ void stage_finish(Stage& st, int32_t* __restrict__ out, bool aligned) {
  const int slot = (int)(st.gpos & 7);
  if (slot != 0) stage_flush(st, out, slot, aligned);
}

}  // namespace step
}  // namespace trw
