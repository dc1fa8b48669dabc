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
  int32_t off, d;   // CSR row of cur (valid once attempt 0 of the step loaded it, or when rowok)
  int32_t poff, pd; // CSR row of prev
  uint32_t att;     // rejection trial within the step
  int32_t nxo, nxd; // row of the vertex an ALIAS move picked (from its record)
  int32_t rev;      // Node2Vec: position of prev in cur's row (-1: not in it, -2: unknown)
  int32_t px;       // Node2Vec: position of cur in prev's row (-2: unknown)
  bool nxv;         // nxo/nxd hold the next vertex's row
  bool rowok;       // off/d already hold cur's row
};

__device__ __forceinline__ void walker_init(Walker& W, uint32_t w, int32_t src) {
  W.w = w;
  W.s = 0;
  W.cur = src;
  W.prev = -1;
  W.off = W.d = W.poff = W.pd = 0;
  W.att = 0;
  W.nxo = W.nxd = 0;
  W.rev = W.px = -2;
  W.nxv = false;
  W.rowok = false;
}

// FOLD: how many of Node2Vec's return-only darts one unit decides before it
// yields.  0 for the kernels whose threads run free (a per-lane loop splits
// the warp); the persistent kernel takes kFoldDarts (its warp runs as many
// Philox blocks as its busiest lane: more folded darts idle more lanes, fewer
// cost more units); kFoldAll folds until the dart needs its candidate.
constexpr int kFoldDarts = 2;
constexpr int kFoldAll = 1 << 30;

enum StepResult : int { kIdle = -1, kMoved = 0, kStop = 1, kRetry = 2, kFail = 3, kBroken = 4, kDefer = 5 };

// Row lengths from which a lane hands its work to the warp.
struct Coop {
  int32_t scan;    // MetaPath label rows at least this long: warp-cooperative Gather
  int32_t search;  // Node2Vec neighbour checks in rows of prev at least this long: warp search
};

// Work a lane hands to its warp: a MetaPath Gather over a long row (kind 1)
// or a Node2Vec IsNeighbor check in a long row of prev (kind 2).
struct Pend {
  uint32_t kind;            // 0 none, 1 MetaPath scan, 2 neighbour check
  int32_t c;                // kind 2: candidate vertex
  uint32_t y;               // kind 2: the dart
  uint32_t hrep;            // kind 1: schema label replicated in four bytes
  unsigned long long r64;   // kind 1: the draw that picks the r-th match
  int32_t res;              // warp result: kind 1 index of the match (-1: none), kind 2 neighbour (0/1)
};

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

// Word k (0..7) of a 32-byte record held as two uint4 (selects, no local memory).
__device__ __forceinline__ uint32_t word8(const uint4& a, const uint4& b, uint32_t k) {
  const uint4& v = k < 4 ? a : b;
  const uint32_t i = k & 3;
  return i == 0 ? v.x : i == 1 ? v.y : i == 2 ? v.z : v.w;
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

// IsNeighbor(c, u) by u's table of the neighbour hash (u's row at poff,
// pd entries): about 1.5 probes, nearly always within one sector.
__device__ __forceinline__ bool is_neighbor_hashed(const NeighborHash& h, int32_t poff, int32_t pd, int32_t c) {
  const uint32_t cap = 2u * (uint32_t)pd;
  const int32_t* tab = h.slots + 2 * (int64_t)poff;
  uint32_t b = slot_of(c, cap);
  for (uint32_t probe = 0; probe < cap; ++probe) {
    const int32_t v = ldg(tab + b);
    if (v == c) return true;
    if (v == kHashEmpty) return false;
    b = b + 1 == cap ? 0u : b + 1;
  }
  return false;
}

// IsNeighbor(c, prev): the hash for rows it holds, else the row's binary search.
__device__ __forceinline__ bool is_neighbor(const DevGraph& g, int32_t prev, int32_t poff, int32_t pd, int32_t c) {
  if (g.nh.slots && pd >= g.nh.min_degree) return is_neighbor_hashed(g.nh, poff, pd, c);
  return is_neighbor_serial(g.col, poff, pd, c);
}

// One unit of work for one walker: a full step, or one rejection trial of a
// Node2Vec step.  Rows at least coop long are not scanned or searched by the
// lane alone: the step returns kDefer with the work in p, the warp resolves it
// (warp_metapath / warp_neighbor) and step_finish completes the step.
// CHECK adds range checks of the walker's vertex and of the row it loads
// before any access through them (kBroken instead of an out-of-range read).
// RET lets Node2Vec keep the positions that decide return-only darts; the
// per-request dispatch of mixed batches leaves it off, which keeps that
// kernel's code and live state those of the other algorithms.
template <int A, bool CHECK = false, int FOLD = kFoldAll, bool RET = true>
__device__ __forceinline__ int step_begin(const DevGraph& g, const WalkSpec& sp, Walker& W, int32_t& next, Pend& p,
                                          Coop coop) {
  p.kind = 0;
  if (W.s == sp.max_len) return kStop;                         // Update: target length reached
  const uint4 B = draw_block(sp, W.w, (uint32_t)W.s, W.att);
  if (A == PPR && (uint64_t)B.w < sp.T_stop) return kStop;     // Update: PPR stop coin
  if (W.att == 0) {
    if (!W.rowok) {
      if (CHECK && (uint32_t)W.cur >= (uint32_t)g.nv) return kBroken;
      if (A == METAPATH && g.lidx.vrec) {
        // Indexed MetaPath: (off, d) is the group of this step's label.
        const uint32_t h = schema_label(sp, (uint32_t)W.s % sp.schema_len);
        if (h < (uint32_t)g.lidx.nl) {
          const int32_t* vr = g.lidx.vrec + (int64_t)W.cur * g.lidx.stride;
          W.off = ldg(vr + 1 + h);
          W.d = ldg(vr + 2 + h) - W.off;
        } else {
          W.off = W.d = 0;
        }
      } else {
        W.off = ldg(g.row_ptr + W.cur);
        W.d = ldg(g.row_ptr + W.cur + 1) - W.off;
      }
    }
    if (CHECK && (W.off < 0 || W.d < 0 || (int64_t)W.off + W.d > (int64_t)g.ne)) return kBroken;
  }
  if (W.d == 0) return kStop;                                  // dead end
  if (A == DEEPWALK || A == PPR) {
    // NAIVE: E_v[x], x uniform in [0, d_v).  A row record also carries the
    // picked vertex's row for the next step.
    const int64_t e = (int64_t)W.off + below(B, (uint32_t)W.d);
    if (g.rrec) {
      const int4 r = __ldg(&g.rrec[e].a);
      next = r.x;
      W.nxo = r.y;
      W.nxd = r.z;
      W.nxv = true;
    } else {
      next = ldg(g.col + e);
    }
    return kMoved;
  } else if (A == DEEPWALK_WEIGHTED) {
    // ALIAS generation from the stored C_v (no Gather for static walks); the
    // record also carries the picked vertex's row for the next step.
    const AliasRec* rec = g.alias + W.off + below(B, (uint32_t)W.d);
    uint4 ra, rb;
    ldg32(rec, ra, rb);
    const bool first = B.z < ra.x;
    const int32_t pick = first ? (int32_t)ra.y : (int32_t)ra.z;
    if (pick < 0) return kStop;                                // no positive weight
    next = pick;
    W.nxo = first ? (int32_t)ra.w : (int32_t)rb.x;
    W.nxd = first ? (int32_t)rb.y : (int32_t)rb.z;
    W.nxv = true;
    return kMoved;
  } else if (A == METAPATH) {
    if (g.lidx.erec) {
      // Indexed: the r-th entry of the label group is the r-th match; its
      // record holds the next vertex and the bounds of its label groups.
      const uint32_t h2 = schema_label(sp, (uint32_t)(W.s + 1) % sp.schema_len);
      const int64_t e = (int64_t)W.off + below(B, (uint32_t)W.d);
      int32_t lo, hi;
      if (h2 >= (uint32_t)g.lidx.nl) {
        next = ldg(g.lidx.erec + e * g.lidx.stride);
        lo = hi = 0;
      } else if (g.lidx.stride == 8) {
        const uint4* rp = reinterpret_cast<const uint4*>(g.lidx.erec + e * 8);
        uint4 ra, rb;
        ldg32(rp, ra, rb);
        next = (int32_t)ra.x;
        lo = (int32_t)word8(ra, rb, 1 + h2);
        hi = (int32_t)word8(ra, rb, 2 + h2);
      } else {
        const int32_t* rp = g.lidx.erec + e * g.lidx.stride;
        next = ldg(rp);
        lo = ldg(rp + 1 + h2);
        hi = ldg(rp + 2 + h2);
      }
      W.nxo = lo;
      W.nxd = hi - lo;
      W.nxv = true;
      return kMoved;
    }
    // Gather (0/1 weights by label) then ITS generation: the r-th match.
    const uint32_t h = schema_label(sp, (uint32_t)W.s % sp.schema_len);
    const uint32_t hrep = h * 0x01010101u;
    if (W.d >= coop.scan) {
      p.kind = 1;
      p.hrep = hrep;
      p.r64 = ((unsigned long long)B.y << 32) | B.x;
      return kDefer;
    }
    const int64_t lo = W.off, hi = (int64_t)W.off + W.d;
    const uint32_t cnt = label_count_serial(g.labels, lo, hi, hrep);
    if (cnt == 0) return kStop;
    const uint32_t r = below(B, cnt);
    const int32_t j = label_select_serial(g.labels, lo, hi, hrep, r);
    if (j < 0) return kBroken;                                 // count and select disagree: internal error
    next = ldg(g.col + W.off + j);
    return kMoved;
  } else if (A == DW_ITS && g.its_rec) {
    // Guided ITS: the cell's record bounds the answer, usually to one or two
    // candidates; the answer's record holds the next vertex and its row.
    const ItsRec* R = g.its_rec + W.off;
    const unsigned long long r = max(((unsigned long long)B.y << 32) | B.x, 1ull);
    const uint32_t k = below(B, (uint32_t)W.d);
    uint4 ja = __ldg(&R[k].a), jb = __ldg(&R[k].b);
    int32_t a = (int32_t)jb.y;
    const int32_t hi = (int32_t)jb.z;
    if (a < 0) return kStop;                                   // no positive weight
    if (CHECK && (a >= W.d || hi >= W.d || hi < a)) return kBroken;
    if (a != (int32_t)k) {
      ja = __ldg(&R[a].a);
      jb = __ldg(&R[a].b);
    }
    if (r > (((unsigned long long)ja.y << 32) | ja.x)) {
      // smallest j in (a, hi] with r <= U_j; it exists, at hi at the latest
      int32_t n = hi - a - 1;
      a += 1;
      while (n > 0) {
        const int32_t half = n >> 1;
        const uint4 m = __ldg(&R[a + half].a);
        if ((((unsigned long long)m.y << 32) | m.x) < r) {
          a += half + 1;
          n -= half + 1;
        } else {
          n = half;
        }
      }
      ja = __ldg(&R[a].a);
      jb = __ldg(&R[a].b);
    }
    next = (int32_t)ja.z;
    W.nxo = (int32_t)ja.w;
    W.nxd = (int32_t)jb.x;
    W.nxv = true;
    return kMoved;
  } else if (A == DW_ITS) {
    // Static ITS generation from the stored P' of the row: x uniform in
    // [0, p'_{d-1}), then the smallest i with x < p'_i, by a lower-bound
    // search over the first d - 1 sums (p'_{d-1} > x bounds the answer).
    if (CHECK && !g.cdf) return kBroken;
    const unsigned long long* P = g.cdf + W.off;
    const unsigned long long S = __ldg(P + W.d - 1);
    if (S == 0ull) return kStop;                               // no positive weight
    const unsigned long long x = below64(B, S);
    int32_t lo = 0, n = W.d - 1;
    while (n > 0) {
      const int32_t half = n >> 1;
      if (__ldg(P + lo + half) <= x) {
        lo += half + 1;
        n -= half + 1;
      } else {
        n = half;
      }
    }
    const int64_t e = (int64_t)W.off + lo;
    if (g.rrec) {
      const int4 r = __ldg(&g.rrec[e].a);
      next = r.x;
      W.nxo = r.y;
      W.nxd = r.z;
      W.nxv = true;
    } else {
      next = ldg(g.col + e);
    }
    return kMoved;
  } else if (A == DW_REJ || A == DW_OREJ) {
    // REJ / O-REJ: dart (x, y), x uniform in [0, d_v); it hits when
    // y < floor(W_x * 2^32 / p*), i.e. when (y + 1) * p* <= W_x * 2^32.
    // p* is the row's stored bound (REJ) or the caller's (O-REJ, in T_stop).
    if (CHECK && !g.weights) return kBroken;
    unsigned long long ps = sp.T_stop;
    if (A == DW_REJ && sp.algo != DW_OREJ) {
      if (CHECK && ((uint32_t)W.cur >= (uint32_t)g.nv || !g.pmax)) return kBroken;
      ps = __ldg(g.pmax + W.cur);
      if (ps == 0ull) return kStop;                            // no positive weight
    }
    const int64_t e = (int64_t)W.off + below(B, (uint32_t)W.d);
    int4 rr;
    uint32_t wx;
    if (g.rrec) {
      rr = __ldg(&g.rrec[e].a);
      wx = (uint32_t)rr.w;
    } else {
      rr.x = ldg(g.col + e);
      wx = weight_fixed(__ldg(g.weights + e));
    }
    if (((unsigned long long)B.z + 1ull) * ps <= ((unsigned long long)wx << 32)) {
      next = rr.x;
      if (g.rrec) {
        W.nxo = rr.y;
        W.nxd = rr.z;
        W.nxv = true;
      }
      return kMoved;
    }
    return (W.att + 1 >= kRejectCap) ? kFail : kRetry;
  } else {  // NODE2VEC, N2V_W: O-REJ
    unsigned long long P = 0;
    if (A == N2V_W) {
      // the weight bound: the caller's, else the row's p*_v
      P = sp.T_stop;
      if (P == 0ull) {
        if (CHECK && ((uint32_t)W.cur >= (uint32_t)g.nv || !g.pmax)) return kBroken;
        P = __ldg(g.pmax + W.cur);
        if (P == 0ull) return kStop;                           // no positive weight
      }
      if (CHECK && !g.weights) return kBroken;
    }
    uint4 Bd = B;  // this dart's block
    uint32_t x = below(Bd, (uint32_t)W.d);
    if (A == NODE2VEC && RET && W.s > 0 && W.rev != -2) {
      // At or past both non-return thresholds only a return to prev can
      // accept, and prev's position in this row is known (-1: not in it): such
      // a dart is decided without reading its candidate.  When it is rejected
      // the next dart is drawn at once, within this unit of work, up to FOLD
      // darts; past them the unit ends with the retry.
      int folds = 0;
      while ((uint64_t)Bd.z >= sp.T_hi) {
        if ((int32_t)x == W.rev && (uint64_t)Bd.z < sp.T_ret) {
          next = W.prev;
          W.nxo = W.poff;
          W.nxd = W.pd;
          W.nxv = true;
          const int32_t t = W.rev;  // back along the edge just walked
          W.rev = W.px;
          W.px = t;
          return kMoved;
        }
        if (W.att + 1 >= kRejectCap) return kFail;
        if (FOLD == 0 || (FOLD < kFoldAll && ++folds >= FOLD)) return kRetry;
        W.att += 1;
        Bd = draw_block(sp, W.w, (uint32_t)W.s, W.att);
        x = below(Bd, (uint32_t)W.d);
      }
    }
    const int64_t e = (int64_t)W.off + x;
    int4 rr = make_int4(0, 0, 0, 0);
    int32_t rrev = -2;
    if (g.rrec) {
      rr = __ldg(&g.rrec[e].a);
      if (A == NODE2VEC && RET && g.rrec_rev) rrev = rr.w;  // the aux word holds rev_e
    }
    const int32_t c = g.rrec ? rr.x : ldg(g.col + e);
    if (A == N2V_W) {
      // weight word: (z + 1) * P <= W_x * 2^32, i.e. z < floor(W_x * 2^32 / P)
      const uint32_t wx = g.rrec ? (uint32_t)rr.w : weight_fixed(__ldg(g.weights + e));
      if (((unsigned long long)Bd.w + 1ull) * P > ((unsigned long long)wx << 32))
        return (W.att + 1 >= kRejectCap) ? kFail : kRetry;
    }
    bool accept;
    if (W.s == 0) accept = true;                               // Weight = MaxWeight on the first step
    else if (c == W.prev) accept = (uint64_t)Bd.z < sp.T_ret;
    else if ((uint64_t)Bd.z < sp.T_lo) accept = true;
    else if ((uint64_t)Bd.z >= sp.T_hi) accept = false;
    else if (W.pd >= coop.search && !g.nh.slots) {
      p.kind = 2;
      p.c = c;
      p.y = Bd.z;
      return kDefer;
    } else {
      accept = (uint64_t)Bd.z < (is_neighbor(g, W.prev, W.poff, W.pd, c) ? sp.T_nb : sp.T_far);
    }
    if (accept) {
      next = c;
      if (g.rrec) {
        W.nxo = rr.y;
        W.nxd = rr.z;
        W.nxv = true;
        if (A == NODE2VEC && RET) {  // positions for the next step's return-only darts
          W.rev = rrev;
          W.px = (int32_t)x;
        }
      }
      return kMoved;
    }
    return (W.att + 1 >= kRejectCap) ? kFail : kRetry;
  }
}

// The thread-serial step (no warp cooperation).
template <int A, bool CHECK = false, int FOLD = kFoldAll, bool RET = true>
__device__ __forceinline__ int step_serial(const DevGraph& g, const WalkSpec& sp, Walker& W, int32_t& next) {
  Pend p;
  return step_begin<A, CHECK, FOLD, RET>(g, sp, W, next, p, Coop{0x7fffffff, 0x7fffffff});
}

// Completes a deferred step once the warp has filled p.res.
__device__ __forceinline__ int step_finish(const DevGraph& g, const WalkSpec& sp, Walker& W, const Pend& p,
                                           int32_t& next) {
  if (p.kind == 1) {
    if (p.res < 0) return kStop;                               // no edge carries the label
    next = ldg(g.col + W.off + p.res);
    return kMoved;
  }
  if ((uint64_t)p.y < (p.res ? sp.T_nb : sp.T_far)) {
    next = p.c;
    W.rev = W.px = -2;  // the candidate's record was not read
    return kMoved;
  }
  return (W.att + 1 >= kRejectCap) ? kFail : kRetry;
}

// Bytes of the aligned word at wa that lie in [lo, hi), as a byte mask.
__device__ __forceinline__ uint32_t bytes_in(int64_t wa, int64_t lo, int64_t hi) {
  if (wa + 4 <= lo || wa >= hi) return 0u;
  uint32_t m = 0xffffffffu;
  if (wa < lo) m &= 0xffffffffu << (8 * (int)(lo - wa));
  if (wa + 4 > hi) m &= 0xffffffffu >> (8 * (int)(wa + 4 - hi));
  return m;
}

// Matching bytes (0xff each) of the 16 labels at p, limited to [lo, hi).
__device__ __forceinline__ uint4 match16(const uint8_t* __restrict__ labels, int64_t p, int64_t lo, int64_t hi,
                                         uint32_t hrep) {
  uint4 m = make_uint4(0u, 0u, 0u, 0u);
  if (p < hi) {
    const uint4 v = __ldg(reinterpret_cast<const uint4*>(labels + p));
    m.x = __vcmpeq4(v.x, hrep) & bytes_in(p, lo, hi);
    m.y = __vcmpeq4(v.y, hrep) & bytes_in(p + 4, lo, hi);
    m.z = __vcmpeq4(v.z, hrep) & bytes_in(p + 8, lo, hi);
    m.w = __vcmpeq4(v.w, hrep) & bytes_in(p + 12, lo, hi);
  }
  return m;
}

__device__ __forceinline__ uint32_t count16(uint4 m) {
  return (uint32_t)((__popc(m.x) + __popc(m.y) + __popc(m.z) + __popc(m.w)) >> 3);
}

// Index (relative to lo) of the k-th matching label among the 16 at pos.
__device__ __forceinline__ int32_t kth_in16(uint4 m, uint32_t k, int64_t pos, int64_t lo) {
  int32_t j = -1;
#pragma unroll
  for (int wi = 0; wi < 4; ++wi) {
    const uint32_t w = (wi == 0) ? m.x : (wi == 1) ? m.y : (wi == 2) ? m.z : m.w;
    const uint32_t cw = (uint32_t)__popc(w) >> 3;
    if (j < 0) {
      if (k < cw) {
        for (int b = 0; b < 4; ++b) {
          if ((w >> (8 * b)) & 0xffu) {
            if (k == 0) {
              j = (int32_t)(pos + 4 * wi + b - lo);
              break;
            }
            --k;
          }
        }
      } else {
        k -= cw;
      }
    }
  }
  return j;
}

// Within one 512-byte chunk whose per-lane match masks are m: the index of the
// r-th match of the chunk (r < the chunk's total), found with a warp prefix sum.
__device__ __forceinline__ int32_t select_in_chunk(uint4 m, uint32_t r, int64_t pos, int64_t lo, int lane) {
  const uint32_t c = count16(m);
  uint32_t incl = c;
#pragma unroll
  for (int o2 = 1; o2 < 32; o2 <<= 1) {
    const uint32_t t = __shfl_up_sync(kFull, incl, o2);
    if (lane >= o2) incl += t;
  }
  const bool mine = r >= incl - c && r < incl;
  const int32_t j = mine ? kth_in16(m, r - (incl - c), pos, lo) : -1;
  const unsigned owner = __ballot_sync(kFull, mine);
  return __shfl_sync(kFull, j, __ffs(owner) - 1);
}

// Warp-cooperative MetaPath Gather + ITS generation for the lanes in `who`:
// the warp counts the row's labels equal to the step's label 512 bytes at a
// time (16 per lane, byte compares and popcount, a warp sum), lane g keeping
// the total of chunk group g; it draws r in [0, cnt) from the owner's draw,
// finds the group holding the r-th match with a warp prefix sum, and rescans
// only that group (a one-chunk row is not rescanned).  Sets p.res of each owner.
__device__ __forceinline__ void warp_metapath(const uint8_t* __restrict__ labels, unsigned who, const Walker& W,
                                              Pend& p) {
  const int lane = threadIdx.x & 31;
  while (who) {
    const int o = __ffs(who) - 1;
    who &= who - 1;
    const int64_t lo = __shfl_sync(kFull, W.off, o);
    const int64_t hi = lo + __shfl_sync(kFull, W.d, o);
    const uint32_t hrep = __shfl_sync(kFull, p.hrep, o);
    const unsigned long long r64 = __shfl_sync(kFull, p.r64, o);
    const int64_t a0 = lo & ~int64_t(15);
    const int64_t nch = (hi - a0 + 511) >> 9;           // 512-byte chunks
    const int64_t gs = (nch + 31) >> 5;                  // chunks per group (32 groups at most)
    uint32_t cnt = 0, grp = 0;
    uint4 m0 = make_uint4(0u, 0u, 0u, 0u);
    for (int64_t k = 0; k < nch; ++k) {
      const uint4 m = match16(labels, a0 + (k << 9) + 16 * lane, lo, hi, hrep);
      if (k == 0) m0 = m;
      const uint32_t t = __reduce_add_sync(kFull, count16(m));
      cnt += t;
      if (lane == (int)(k / gs)) grp += t;
    }
    int32_t res = -1;
    if (cnt > 0) {
      uint32_t r = (uint32_t)__umul64hi(r64, (unsigned long long)cnt);
      if (nch == 1) {
        res = select_in_chunk(m0, r, a0 + 16 * lane, lo, lane);
      } else {
        // the group holding match r
        uint32_t incl = grp;
#pragma unroll
        for (int o2 = 1; o2 < 32; o2 <<= 1) {
          const uint32_t t = __shfl_up_sync(kFull, incl, o2);
          if (lane >= o2) incl += t;
        }
        const unsigned hit = __ballot_sync(kFull, r >= incl - grp && r < incl);
        const int tg = __ffs(hit) - 1;
        r -= __shfl_sync(kFull, incl - grp, tg);
        const int64_t k_end = min(nch, (int64_t)(tg + 1) * gs);
        for (int64_t k = (int64_t)tg * gs; k < k_end; ++k) {
          const int64_t pos = a0 + (k << 9) + 16 * lane;
          const uint4 m = match16(labels, pos, lo, hi, hrep);
          const uint32_t t = __reduce_add_sync(kFull, count16(m));
          if (r < t) {
            res = select_in_chunk(m, r, pos, lo, lane);
            break;
          }
          r -= t;
        }
      }
    }
    if (lane == o) p.res = res;
  }
}

// Warp-cooperative IsNeighbor(c, prev) for the lanes in `who`: a 32-way search
// of c in the sorted row of prev -- each round the lanes load the last element
// of 32 equal segments and keep the first segment whose last element is >= c --
// then one compare per lane over the final <= 32 elements.  Sets p.res (0/1).
__device__ __forceinline__ void warp_neighbor(const int32_t* __restrict__ col, unsigned who, const Walker& W, Pend& p) {
  const int lane = threadIdx.x & 31;
  while (who) {
    const int o = __ffs(who) - 1;
    who &= who - 1;
    const int32_t poff = __shfl_sync(kFull, W.poff, o);
    const int32_t c = __shfl_sync(kFull, p.c, o);
    int32_t lo = 0, n = __shfl_sync(kFull, W.pd, o);
    int found = -1;
    while (n > 32) {
      const int32_t last = lo + (int32_t)(((int64_t)(lane + 1) * n) >> 5) - 1;
      const int32_t x = ldg(col + poff + last);
      const unsigned ge = __ballot_sync(kFull, x >= c);
      if (ge == 0u) {
        found = 0;  // c is beyond the last element
        break;
      }
      const int t = __ffs(ge) - 1;
      if (__shfl_sync(kFull, x, t) == c) {
        found = 1;
        break;
      }
      const int32_t seg_lo = lo + (int32_t)(((int64_t)t * n) >> 5);
      const int32_t seg_hi = lo + (int32_t)(((int64_t)(t + 1) * n) >> 5);
      lo = seg_lo;
      n = seg_hi - seg_lo;
    }
    if (found < 0) found = __ballot_sync(kFull, lane < n && ldg(col + poff + lo + lane) == c) != 0u ? 1 : 0;
    if (lane == o) p.res = found;
  }
}

// Resolves the deferred work of a warp; every lane of the warp must call it.
__device__ __forceinline__ void warp_resolve(const DevGraph& g, int r, const Walker& W, Pend& p) {
  const unsigned meta = __ballot_sync(kFull, r == kDefer && p.kind == 1);
  if (meta) warp_metapath(g.labels, meta, W, p);
  const unsigned nb = __ballot_sync(kFull, r == kDefer && p.kind == 2);
  if (nb) warp_neighbor(g.col, nb, W, p);
}

__device__ __forceinline__ void advance(Walker& W, int32_t next) {
  W.prev = W.cur;
  W.poff = W.off;
  W.pd = W.d;
  W.cur = next;
  W.s += 1;
  W.att = 0;
  W.rowok = W.nxv;
  if (W.nxv) {
    W.off = W.nxo;
    W.d = W.nxd;
    W.nxv = false;
  }
}


// Weighted DeepWalk under ITS, REJ or O-REJ, and weighted Node2Vec, in the
// mixed kernels (batches and the server): one step run out of line, so that these samplers' registers do
// not weigh on every other algorithm of the dispatcher.  The walker goes in
// by value; the fields a step may change come back.
struct SamplerOut {
  int r;
  int32_t next, off, d, nxo, nxd;
  bool nxv;
};

template <bool CHECK>
__device__ __noinline__ SamplerOut sampler_step(const DevGraph& g, const WalkSpec& sp, Walker W) {
  SamplerOut o;
  Pend p;
  o.next = -1;
  const Coop none{0x7fffffff, 0x7fffffff};
  o.r = sp.algo == DW_ITS  ? step_begin<DW_ITS, CHECK>(g, sp, W, o.next, p, none)
        : sp.algo == N2V_W ? step_begin<N2V_W, CHECK>(g, sp, W, o.next, p, none)
                           : step_begin<DW_REJ, CHECK>(g, sp, W, o.next, p, none);
  o.off = W.off;
  o.d = W.d;
  o.nxo = W.nxo;
  o.nxd = W.nxd;
  o.nxv = W.nxv;
  return o;
}

template <bool CHECK>
__device__ __forceinline__ int sampler_step_apply(const DevGraph& g, const WalkSpec& sp, Walker& W, int32_t& next) {
  const SamplerOut o = sampler_step<CHECK>(g, sp, W);
  W.off = o.off;
  W.d = o.d;
  W.nxo = o.nxo;
  W.nxd = o.nxd;
  W.nxv = o.nxv;
  next = o.next;
  return o.r;
}

template <int A, bool CHECK = false, int FOLD = kFoldAll>
__device__ __forceinline__ int step_dispatch(const DevGraph& g, const WalkSpec& sp, Walker& W, int32_t& next) {
  if constexpr (A != MIXED) {
    return step_serial<A, CHECK, FOLD>(g, sp, W, next);
  } else {
    switch (sp.algo) {
      case DEEPWALK: return step_serial<DEEPWALK, CHECK, FOLD>(g, sp, W, next);
      case DEEPWALK_WEIGHTED: return step_serial<DEEPWALK_WEIGHTED, CHECK, FOLD>(g, sp, W, next);
      case PPR: return step_serial<PPR, CHECK, FOLD>(g, sp, W, next);
      case NODE2VEC: return step_serial<NODE2VEC, CHECK, FOLD, false>(g, sp, W, next);
      case METAPATH: return step_serial<METAPATH, CHECK, FOLD>(g, sp, W, next);
      case DW_ITS:
      case DW_REJ:
      case DW_OREJ:
      case N2V_W: return sampler_step_apply<CHECK>(g, sp, W, next);
      default: return kBroken;
    }
  }
}

// step_begin for a compile-time or per-request algorithm.
template <int A, bool CHECK = false, int FOLD = kFoldAll>
__device__ __forceinline__ int step_begin_dispatch(const DevGraph& g, const WalkSpec& sp, Walker& W, int32_t& next,
                                                   Pend& p, Coop coop) {
  if constexpr (A != MIXED) {
    return step_begin<A, CHECK, FOLD>(g, sp, W, next, p, coop);
  } else {
    switch (sp.algo) {
      case DEEPWALK: return step_begin<DEEPWALK, CHECK>(g, sp, W, next, p, coop);
      case DEEPWALK_WEIGHTED: return step_begin<DEEPWALK_WEIGHTED, CHECK>(g, sp, W, next, p, coop);
      case PPR: return step_begin<PPR, CHECK>(g, sp, W, next, p, coop);
      case NODE2VEC: return step_begin<NODE2VEC, CHECK, kFoldAll, false>(g, sp, W, next, p, coop);
      case METAPATH: return step_begin<METAPATH, CHECK>(g, sp, W, next, p, coop);
      case DW_ITS:
      case DW_REJ:
      case DW_OREJ:
      case N2V_W: p.kind = 0; return sampler_step_apply<CHECK>(g, sp, W, next);
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
