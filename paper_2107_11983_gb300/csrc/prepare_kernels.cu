// Preprocessing for static walks (Algorithm 3) and graph checks, on the device.
//
// ALIAS initialisation (Section 2.3) per vertex, by Vose's method on integer
// weights: W_j = round-half-even(w_j * 2^16); item j carries q_j = d * W_j
// against a bucket capacity S = sum_j W_j.  Items with q_j < S wait in a
// first-in first-out "small" list, the others in a "large" list; the front
// small item s fills its bucket from the front large item l:
//   H[s] = floor(q_s * 2^32 / S), first = s, second = l, q_l -= S - q_s,
// and l joins the back of the small list once q_l < S.  What remains forms
// one-element buckets (H = 2^32 - 1 and second = first, which picks the same
// edge for every 32-bit dart).  The sequence of list operations is fixed, so
// the tables are exactly reproducible.  Records hold the destination vertices
// directly, with their own CSR rows (see AliasRec).  A vertex whose integer
// weights sum to zero gets records with both destinations -1: a dead end.
//
// Parallel form of the same sequence: a warp (a block for rows of kBigRow
// edges or more) sums and classifies the row and lays the items out in queue
// order with ballots; only the pairing itself is sequential, and it runs as
// a lockstep warp loop over two register windows (pair_row); the records,
// with their divisions and destination-row lookups, are then built by all
// threads.  Large rows go first, largest first, since their pairings are the
// longest sequential chains.
#include <algorithm>
#include <cstdint>
#include <vector>

#include <cuda_runtime.h>

#include "trw_device.cuh"
#include "trw_internal.h"

namespace trw {

namespace {

// Integer weight of an fp32 weight; false for a negative or non-finite value.
__device__ __forceinline__ bool quantize(float w, uint32_t& out) {
  if (!(w >= 0.0f) || isinf(w)) return false;
  // w * 2^16 is exact in double; rint rounds half to even.
  double t = rint((double)w * 65536.0);
  if (t > 4294967295.0) t = 4294967295.0;
  out = (uint32_t)t;
  return true;
}

// floor(q * 2^32 / S) for q < S <= 2^63, by restoring long division over the
// 32 fractional bits (the quotient is below 2^32).
__device__ __forceinline__ uint32_t frac32(unsigned long long q, unsigned long long S) {
  if (S <= 0xffffffffull) return (uint32_t)((q << 32) / S);
  unsigned long long rem = q;
  uint32_t quo = 0;
#pragma unroll 4
  for (int i = 0; i < 32; ++i) {
    rem <<= 1;
    quo <<= 1;
    if (rem >= S) {
      rem -= S;
      quo |= 1u;
    }
  }
  return quo;
}

constexpr int kPrepThreads = 256;
constexpr int32_t kBigRow = 4096;  // rows this long are prepared by a whole block

__device__ __forceinline__ unsigned long long shfl64_xor(unsigned long long v, int m) {
  const uint32_t lo = __shfl_xor_sync(0xffffffffu, (uint32_t)v, m);
  const uint32_t hi = __shfl_xor_sync(0xffffffffu, (uint32_t)(v >> 32), m);
  return ((unsigned long long)hi << 32) | lo;
}

// Record of a bucket whose first element is destination u (taken with
// probability H / 2^32) and whose second is v.
__device__ __forceinline__ AliasRec make_rec(const int32_t* __restrict__ row_ptr, uint32_t H, int32_t u, int32_t v) {
  const int32_t ou = row_ptr[u], ov = row_ptr[v];
  AliasRec r;
  r.a = make_uint4(H, (uint32_t)u, (uint32_t)v, (uint32_t)ou);
  r.b = make_uint4((uint32_t)ov, (uint32_t)(row_ptr[u + 1] - ou), (uint32_t)(row_ptr[v + 1] - ov), 0u);
  return r;
}

constexpr unsigned kFull = 0xffffffffu;

__device__ __forceinline__ unsigned long long shfl64(unsigned long long v, int src) {
  const uint32_t lo = __shfl_sync(kFull, (uint32_t)v, src);
  const uint32_t hi = __shfl_sync(kFull, (uint32_t)(v >> 32), src);
  return ((unsigned long long)hi << 32) | lo;
}

__device__ __forceinline__ unsigned long long warp_sum64(unsigned long long v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += shfl64_xor(v, o);
  return v;
}

// Scratch of one row at offset off: idx[p] is the item at position p of the
// queue order (the small items 0..ns-1 first, then the large ones, each in
// ascending item order), qv[p] its q, and part[p] the large index it is
// paired with.
struct Scratch {
  unsigned long long* qv;
  int32_t* idx;
  int32_t* part;
};

// The FIFO pairing of one row, run by all 32 lanes of a warp in lockstep.
// The small queue is the small items followed by the large items in the
// order they turn small, which is their own order, so position p of idx is
// the p-th item popped; qv[ns + k] receives the q of large k when it turns
// small, before the loop can reach position ns + k.  The loop only moves
// two cursors forward, so each lane holds one element of a 32-position
// window per cursor: wI (the pop cursor i) and wL (the large cursor
// ns + lh, whose entries are overwritten as larges turn small).  When both
// cursors are in the same window the pop reads wL.  Returns the number of
// pops; part[p] is written for every p below it and qv[p] holds the popped q.
__device__ int32_t pair_row(int64_t off, int32_t d, int32_t ns, unsigned long long S, const Scratch& sc,
                            int lane) {
  const int32_t nl = d - ns;
  if (ns == 0 || nl == 0) return 0;
  unsigned long long* qv = sc.qv + off;
  int32_t* part = sc.part + off;
  int32_t i = 0, lh = 0, lpos = ns;
  const int32_t lb0 = lpos & ~31;
  unsigned long long wL = lb0 + lane < d ? qv[lb0 + lane] : 0ull;
  unsigned long long wI = (lpos >> 5) != 0 ? qv[lane] : 0ull;  // block 0 holds only small items then
  int32_t my_part = -1;
  unsigned long long rem = shfl64(wL, lpos & 31);
  while (i < ns + lh && lh < nl) {
    const bool same = (i >> 5) == (lpos >> 5);
    const unsigned long long qs = shfl64(same ? wL : wI, i & 31);
    if (lane == (i & 31)) my_part = lh;
    rem -= S - qs;
    ++i;
    if ((i & 31) == 0) {
      part[i - 32 + lane] = my_part;
      if ((i >> 5) != (lpos >> 5)) wI = i + lane < d ? qv[i + lane] : 0ull;
    }
    if (rem < S) {
      if (lane == (lpos & 31)) wL = rem;
      ++lh;
      ++lpos;
      if ((lpos & 31) == 0) {
        const int32_t b = lpos - 32;
        if (b + lane < d) qv[b + lane] = wL;
        if ((i >> 5) == (b >> 5)) wI = wL;
        wL = lpos + lane < d ? qv[lpos + lane] : 0ull;
      }
      if (lh < nl) rem = shfl64(wL, lpos & 31);
    }
  }
  {
    const int32_t b = i & ~31;
    if (b + lane < i) part[b + lane] = my_part;
  }
  {
    const int32_t b = lpos & ~31;
    if (b + lane < lpos && b + lane < d) qv[b + lane] = wL;
  }
  return i;
}

// The record of the item at queue position p.
__device__ __forceinline__ void emit(int64_t off, int32_t p, int32_t ns, int32_t npop, unsigned long long S,
                                     const int32_t* __restrict__ row_ptr, const int32_t* __restrict__ col,
                                     const Scratch& sc, AliasRec* __restrict__ alias) {
  const int32_t j = sc.idx[off + p];
  const int32_t u = col[off + j];
  if (p < npop) {
    const int32_t l = sc.idx[off + ns + sc.part[off + p]];
    alias[off + j] = make_rec(row_ptr, frac32(sc.qv[off + p], S), u, col[off + l]);
  } else {
    alias[off + j] = make_rec(row_ptr, 0xffffffffu, u, u);
  }
}

__device__ __forceinline__ AliasRec dead_rec() {
  AliasRec r;
  r.a = make_uint4(0u, 0xffffffffu, 0xffffffffu, 0u);
  r.b = make_uint4(0u, 0u, 0u, 0u);
  return r;
}

// One row of fewer than kBigRow edges, by one warp.
__device__ void warp_row(int64_t off, int32_t d, const int32_t* __restrict__ row_ptr,
                         const int32_t* __restrict__ col, const float* __restrict__ weights, const Scratch& sc,
                         AliasRec* __restrict__ alias, Ctrl* ctrl, int lane) {
  unsigned long long S = 0;
  bool ok = true;
  for (int32_t j = lane; j < d; j += 32) {
    uint32_t W;
    ok &= quantize(weights[off + j], W);
    S += W;
  }
  S = warp_sum64(S);
  if (!__all_sync(kFull, ok)) {
    if (lane == 0) atomicCAS(&ctrl->err, 0, kErrInvalid);
    return;
  }
  if (S == 0) {
    for (int32_t j = lane; j < d; j += 32) alias[off + j] = dead_rec();
    return;
  }
  const unsigned lt = (1u << lane) - 1u;
  int32_t ns = 0;
  for (int32_t b = 0; b < d; b += 32) {
    const int32_t j = b + lane;
    uint32_t W = 0;
    if (j < d) quantize(weights[off + j], W);
    ns += __popc(__ballot_sync(kFull, j < d && (unsigned long long)d * W < S));
  }
  int32_t cs = 0, cl = ns;
  for (int32_t b = 0; b < d; b += 32) {
    const int32_t j = b + lane;
    uint32_t W = 0;
    if (j < d) quantize(weights[off + j], W);
    const unsigned long long q = (unsigned long long)d * W;
    const bool small = j < d && q < S;
    const unsigned ms = __ballot_sync(kFull, small), ml = __ballot_sync(kFull, j < d && !small);
    if (j < d) {
      const int32_t p = small ? cs + __popc(ms & lt) : cl + __popc(ml & lt);
      sc.idx[off + p] = j;
      sc.qv[off + p] = q;
    }
    cs += __popc(ms);
    cl += __popc(ml);
  }
  __syncwarp();
  const int32_t npop = pair_row(off, d, ns, S, sc, lane);
  __syncwarp();
  for (int32_t p = lane; p < d; p += 32) emit(off, p, ns, npop, S, row_ptr, col, sc, alias);
}

// One row of kBigRow or more edges, by the whole block (kPrepThreads
// threads); warp 0 runs the pairing.
__device__ void block_row(int64_t off, int32_t d, const int32_t* __restrict__ row_ptr,
                          const int32_t* __restrict__ col, const float* __restrict__ weights, const Scratch& sc,
                          AliasRec* __restrict__ alias, Ctrl* ctrl) {
  constexpr int kWarps = kPrepThreads / 32;
  __shared__ unsigned long long s_sum[kWarps];
  __shared__ int32_t s_cnt[2][kWarps];
  __shared__ int32_t s_ok, s_npop;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  unsigned long long S = 0;
  bool ok = true;
  for (int32_t j = threadIdx.x; j < d; j += kPrepThreads) {
    uint32_t W;
    ok &= quantize(weights[off + j], W);
    S += W;
  }
  S = warp_sum64(S);
  ok = __all_sync(kFull, ok);
  if (threadIdx.x == 0) s_ok = 1;
  __syncthreads();
  if (lane == 0) {
    s_sum[warp] = S;
    if (!ok) s_ok = 0;
  }
  __syncthreads();
  S = 0;
#pragma unroll
  for (int k = 0; k < kWarps; ++k) S += s_sum[k];
  const bool all_ok = s_ok != 0;
  __syncthreads();
  if (!all_ok) {
    if (threadIdx.x == 0) atomicCAS(&ctrl->err, 0, kErrInvalid);
    return;
  }
  if (S == 0) {
    for (int32_t j = threadIdx.x; j < d; j += kPrepThreads) alias[off + j] = dead_rec();
    return;
  }
  // Small-item count.
  int32_t ns_part = 0;
  for (int32_t j = threadIdx.x; j < d; j += kPrepThreads) {
    uint32_t W;
    quantize(weights[off + j], W);
    ns_part += (unsigned long long)d * W < S ? 1 : 0;
  }
  ns_part = __reduce_add_sync(kFull, ns_part);
  if (lane == 0) s_cnt[0][warp] = ns_part;
  __syncthreads();
  int32_t ns = 0;
#pragma unroll
  for (int k = 0; k < kWarps; ++k) ns += s_cnt[0][k];
  __syncthreads();
  // Ordered compaction, kPrepThreads items per round.
  const unsigned lt = (1u << lane) - 1u;
  int32_t cs = 0, cl = ns;
  for (int32_t b = 0; b < d; b += kPrepThreads) {
    const int32_t j = b + threadIdx.x;
    uint32_t W = 0;
    if (j < d) quantize(weights[off + j], W);
    const unsigned long long q = (unsigned long long)d * W;
    const bool small = j < d && q < S;
    const unsigned ms = __ballot_sync(kFull, small), ml = __ballot_sync(kFull, j < d && !small);
    if (lane == 0) {
      s_cnt[0][warp] = __popc(ms);
      s_cnt[1][warp] = __popc(ml);
    }
    __syncthreads();
    int32_t bs = cs, bl = cl, ts = 0, tl = 0;
#pragma unroll
    for (int k = 0; k < kWarps; ++k) {
      if (k < warp) {
        bs += s_cnt[0][k];
        bl += s_cnt[1][k];
      }
      ts += s_cnt[0][k];
      tl += s_cnt[1][k];
    }
    if (j < d) {
      const int32_t p = small ? bs + __popc(ms & lt) : bl + __popc(ml & lt);
      sc.idx[off + p] = j;
      sc.qv[off + p] = q;
    }
    cs += ts;
    cl += tl;
    __syncthreads();
  }
  if (warp == 0) {
    const int32_t npop = pair_row(off, d, ns, S, sc, lane);
    if (lane == 0) s_npop = npop;
  }
  __syncthreads();
  const int32_t npop = s_npop;
  for (int32_t p = threadIdx.x; p < d; p += kPrepThreads) emit(off, p, ns, npop, S, row_ptr, col, sc, alias);
  __syncthreads();
}

// Rows of kBigRow edges or more first, one per block, largest first (the
// list is sorted by degree on the host); then every other row, one per warp,
// claimed 32 rows at a time.
__global__ void __launch_bounds__(kPrepThreads) prepare_alias_kernel(
    int32_t nv, const int32_t* __restrict__ row_ptr, const int32_t* __restrict__ col,
    const float* __restrict__ weights, AliasRec* __restrict__ alias, Scratch sc, const int32_t* __restrict__ big,
    int32_t nbig, unsigned int* counters, Ctrl* ctrl) {
  __shared__ int32_t s_r;
  for (;;) {
    if (threadIdx.x == 0) s_r = (int32_t)atomicAdd(&counters[0], 1u);
    __syncthreads();
    const int32_t r = s_r;
    __syncthreads();
    if (r >= nbig) break;
    const int32_t v = big[r];
    const int32_t off = row_ptr[v];
    block_row(off, row_ptr[v + 1] - off, row_ptr, col, weights, sc, alias, ctrl);
  }
  const int lane = threadIdx.x & 31;
  for (;;) {
    unsigned int base = 0;
    if (lane == 0) base = atomicAdd(&counters[1], 32u);
    base = __shfl_sync(kFull, base, 0);
    if (base >= (unsigned)nv) break;
    const int32_t end = min((int32_t)base + 32, nv);
    for (int32_t v = (int32_t)base; v < end; ++v) {
      const int32_t off = row_ptr[v];
      const int32_t d = row_ptr[v + 1] - off;
      if (d == 0 || d >= kBigRow) continue;
      warp_row(off, d, row_ptr, col, weights, sc, alias, ctrl, lane);
    }
  }
}

// Inserts neighbour v into the table of cap slots at tab: the first empty
// slot from slot_of(v, cap) on, wrapping; probe[0] flags a table found full
// (cannot happen at load 1/2).
__device__ __forceinline__ void row_hash_insert(int32_t* tab, uint32_t cap, int32_t v, unsigned int* probe) {
  uint32_t b = slot_of(v, cap);
  for (uint32_t n = 0; n < cap; ++n) {
    const int32_t old = atomicCAS(tab + b, kHashEmpty, v);
    if (old == kHashEmpty || old == v) return;
    b = b + 1 == cap ? 0u : b + 1;
  }
  atomicExch(probe, 1u);
}

// Same schedule as the alias preparation: rows of kBigRow edges or more by
// whole blocks, largest first, then the other rows one warp each.  Each row
// fills only its own table, which the warp or block has just cleared, so the
// compare-and-swaps stay in L2.
__global__ void __launch_bounds__(kPrepThreads) hash_insert_kernel(
    int32_t nv, const int32_t* __restrict__ row_ptr, const int32_t* __restrict__ col, int32_t min_degree,
    const int32_t* __restrict__ big, int32_t nbig, unsigned int* counters, int32_t* slots, unsigned int* probe) {
  __shared__ int32_t s_r;
  for (;;) {
    if (threadIdx.x == 0) s_r = (int32_t)atomicAdd(&counters[0], 1u);
    __syncthreads();
    const int32_t r = s_r;
    __syncthreads();
    if (r >= nbig) break;
    const int32_t v = big[r];
    const int32_t off = row_ptr[v], d = row_ptr[v + 1] - off;
    if (d < min_degree) continue;
    int32_t* tab = slots + 2 * (int64_t)off;
    for (int32_t j = threadIdx.x; j < 2 * d; j += kPrepThreads) tab[j] = kHashEmpty;
    __syncthreads();
    for (int32_t j = threadIdx.x; j < d; j += kPrepThreads) row_hash_insert(tab, 2u * (uint32_t)d, col[off + j], probe);
    __syncthreads();
  }
  const int lane = threadIdx.x & 31;
  for (;;) {
    unsigned int base = 0;
    if (lane == 0) base = atomicAdd(&counters[1], 32u);
    base = __shfl_sync(kFull, base, 0);
    if (base >= (unsigned)nv) break;
    const int32_t end = min((int32_t)base + 32, nv);
    for (int32_t v = (int32_t)base; v < end; ++v) {
      const int32_t off = row_ptr[v], d = row_ptr[v + 1] - off;
      if (d < min_degree || d >= kBigRow) continue;
      int32_t* tab = slots + 2 * (int64_t)off;
      for (int32_t j = lane; j < 2 * d; j += 32) tab[j] = kHashEmpty;
      __syncwarp();
      for (int32_t j = lane; j < d; j += 32) row_hash_insert(tab, 2u * (uint32_t)d, col[off + j], probe);
      __syncwarp();
    }
  }
}

// Rows of kBigRow edges or more, as (degree << 32 | vertex) keys.
__global__ void collect_big_rows(int32_t nv, const int32_t* __restrict__ row_ptr, unsigned long long* keys,
                                 unsigned int* count) {
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < nv; v += (int64_t)gridDim.x * blockDim.x) {
    const int32_t d = row_ptr[v + 1] - row_ptr[v];
    if (d >= kBigRow) keys[atomicAdd(count, 1u)] = ((unsigned long long)d << 32) | (unsigned long long)v;
  }
}

// ------------------------------------------------------ MetaPath label index
// (see LabelIndex).  One warp per row: labels are counted per value with
// __match_any_sync (the lowest lane of each equal-label group adds the
// group's size), the exclusive prefix over labels gives the group starts,
// and a second pass scatters the destinations in CSR order, each lane at its
// group's cursor plus its rank among the equal labels of lower lanes.

__global__ void label_max_kernel(const uint8_t* __restrict__ labels, int64_t ne, unsigned int* out) {
  unsigned int m = 0;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < ne; e += (int64_t)gridDim.x * blockDim.x)
    m = max(m, (unsigned int)labels[e]);
  m = __reduce_max_sync(kFull, m);
  if ((threadIdx.x & 31) == 0) atomicMax(out, m);
}

constexpr int kLabelWarps = 8;

__global__ void __launch_bounds__(kLabelWarps * 32) label_rows_kernel(
    int32_t nv, const int32_t* __restrict__ row_ptr, const int32_t* __restrict__ col,
    const uint8_t* __restrict__ labels, int32_t nl, int32_t stride, int32_t* __restrict__ vrec,
    int32_t* __restrict__ erec) {
  __shared__ int32_t s_cur[kLabelWarps][32];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  int32_t* cur = s_cur[wib];
  const unsigned lt = (1u << lane) - 1u;
  for (int64_t v = (int64_t)blockIdx.x * kLabelWarps + wib; v < nv; v += (int64_t)gridDim.x * kLabelWarps) {
    const int32_t off = row_ptr[v];
    const int32_t d = row_ptr[v + 1] - off;
    cur[lane] = 0;
    __syncwarp();
    for (int32_t b = 0; b < d; b += 32) {
      const int32_t j = b + lane;
      const bool valid = j < d;
      const uint32_t x = valid ? labels[off + j] : 0xffu;
      const unsigned m = __match_any_sync(kFull, x);
      if (valid && lane == __ffs(m) - 1) cur[x] += __popc(m);
      __syncwarp();
    }
    const int32_t cnt = lane < nl ? cur[lane] : 0;
    int32_t incl = cnt;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int32_t t = __shfl_up_sync(kFull, incl, o);
      if (lane >= o) incl += t;
    }
    const int32_t start = off + incl - cnt;  // g(v, lane) for lane < nl
    const int32_t prev_start = __shfl_up_sync(kFull, start, 1);
    __syncwarp();
    if (lane < nl) cur[lane] = start;
    // record word k: v, then g(v, 0..nl), then padding (the row end)
    if (lane < stride) {
      int32_t word;
      if (lane == 0) word = (int32_t)v;
      else if (lane - 1 < nl) word = prev_start;
      else word = off + d;
      vrec[v * stride + lane] = word;
    }
    __syncwarp();
    for (int32_t b = 0; b < d; b += 32) {
      const int32_t j = b + lane;
      const bool valid = j < d;
      const uint32_t x = valid ? labels[off + j] : 0xffu;
      const int32_t c = valid ? col[off + j] : 0;
      const unsigned m = __match_any_sync(kFull, x);
      if (valid) erec[(int64_t)(cur[x] + __popc(m & lt)) * stride] = c;
      __syncwarp();
      if (valid && lane == __ffs(m) - 1) cur[x] += __popc(m);
      __syncwarp();
    }
  }
}

// Edge record e = the vertex record of the destination stored in its word 0.
__global__ void label_gather_kernel(int64_t ne, int32_t stride, const int32_t* __restrict__ vrec,
                                    int32_t* __restrict__ erec) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < ne; e += (int64_t)gridDim.x * blockDim.x) {
    int4* dst = reinterpret_cast<int4*>(erec + e * stride);
    const int32_t v = erec[e * stride];
    const int4* src = reinterpret_cast<const int4*>(vrec + (int64_t)v * stride);
    for (int k = 0; k < stride / 4; ++k) dst[k] = __ldg(src + k);
  }
}

// ---------------------------------------------------------------- row records

// One thread per edge e = (v -> c): c's row and the aux word, the integer
// weight on a weighted graph, else the position of v in c's sorted row (a
// lower-bound search; -1 when absent or the rows are not sorted), where v is
// found from e by a search of the row offsets.
__global__ void row_records_kernel(int32_t nv, int64_t ne, const int32_t* __restrict__ row_ptr,
                                   const int32_t* __restrict__ col, const float* __restrict__ weights, bool sorted,
                                   RowRec* __restrict__ rec) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < ne; e += (int64_t)gridDim.x * blockDim.x) {
    const int32_t c = col[e];
    const int32_t o = row_ptr[c];
    const int32_t d = row_ptr[c + 1] - o;
    int32_t aux = -1;
    if (weights) {
      aux = (int32_t)weight_fixed(weights[e]);
    } else if (sorted) {
      // v: the last row whose offset is <= e
      int32_t lo = 0, n = nv;
      while (n > 0) {
        const int32_t half = n >> 1;
        if ((int64_t)row_ptr[lo + half + 1] <= e) {
          lo += half + 1;
          n -= half + 1;
        } else {
          n = half;
        }
      }
      const int32_t v = lo;
      // lower bound of v in c's row
      int32_t a = 0;
      n = d;
      while (n > 0) {
        const int32_t half = n >> 1;
        if (col[o + a + half] < v) {
          a += half + 1;
          n -= half + 1;
        } else {
          n = half;
        }
      }
      if (a < d && col[o + a] == v) aux = a;
    }
    RowRec r;
    r.a = make_int4(c, o, d, aux);
    rec[e] = r;
  }
}

// ITS and REJ initialisation (Section 2.3) for static weighted walks, one
// warp per row: the inclusive prefix sums P' of the row's integer weights
// (32 at a time: a warp scan plus the running total) and p*_v, the largest
// integer weight.  Either output may be null.
__global__ void sampler_tables_kernel(int32_t nv, const int32_t* __restrict__ row_ptr,
                                      const float* __restrict__ weights, unsigned long long* __restrict__ cdf,
                                      uint32_t* __restrict__ pmax) {
  const int lane = threadIdx.x & 31;
  const int64_t warps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t v = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; v < nv; v += warps) {
    const int32_t lo = row_ptr[v], hi = row_ptr[v + 1];
    unsigned long long run = 0;
    uint32_t mx = 0;
    for (int32_t base = lo; base < hi; base += 32) {
      const int32_t e = base + lane;
      const uint32_t w = e < hi ? weight_fixed(weights[e]) : 0u;
      mx = max(mx, w);
      if (cdf) {
        unsigned long long incl = w;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
          const unsigned long long t = __shfl_up_sync(0xffffffffu, incl, o);
          if (lane >= o) incl += t;
        }
        if (e < hi) cdf[e] = run + incl;
        run += __shfl_sync(0xffffffffu, incl, 31);
      }
    }
    if (pmax) {
      mx = __reduce_max_sync(0xffffffffu, mx);
      if (lane == 0) pmax[v] = mx;
    }
  }
}

// Every id in [0, nv); flags a row that is not strictly increasing.  One warp
// per row, so that a hub row does not hold a single thread for its length.
__global__ void check_graph_kernel(int32_t nv, const int32_t* __restrict__ row_ptr, const int32_t* __restrict__ col,
                                   Ctrl* ctrl, int* unsorted) {
  const int lane = threadIdx.x & 31;
  const int64_t warps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t v = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; v < nv; v += warps) {
    const int32_t lo = row_ptr[v], hi = row_ptr[v + 1];
    bool bad_id = false, bad_order = false;
    for (int32_t e = lo + lane; e < hi; e += 32) {
      const int32_t c = col[e];
      bad_id |= c < 0 || c >= nv;
      if (e > lo) bad_order |= col[e - 1] >= c;
    }
    if (__any_sync(0xffffffffu, bad_id) && lane == 0) atomicCAS(&ctrl->err, 0, kErrInvalid);
    if (__any_sync(0xffffffffu, bad_order) && lane == 0) atomicExch(unsorted, 1);
  }
}

// Every weight finite and non-negative.
__global__ void check_weights_kernel(int64_t ne, const float* __restrict__ w, Ctrl* ctrl) {
  bool bad = false;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < ne; e += (int64_t)gridDim.x * blockDim.x) {
    const float x = w[e];
    bad |= !(x >= 0.0f) || isinf(x);
  }
  if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) atomicCAS(&ctrl->err, 0, kErrInvalid);
}

// Rows of kBigRow edges or more, collected on the device and sorted by
// degree (largest first) on the host, so that the longest rows start first;
// plus zeroed claim counters ([0] big rows, [1] other rows).
struct BigRows {
  int32_t* list = nullptr;
  unsigned int n = 0;
  unsigned int* counters = nullptr;
  unsigned long long* keys = nullptr;
  ~BigRows() {
    cudaFree(list);
    cudaFree(counters);
    cudaFree(keys);
  }
};

cudaError_t collect_big(int32_t nv, int64_t ne, const int32_t* row_ptr, cudaStream_t st, BigRows& br) {
  const size_t max_big = (size_t)(ne / kBigRow) + 1;
  cudaError_t e = trw_dev_malloc((void**)&br.keys, sizeof(unsigned long long) * max_big);
  if (e == cudaSuccess) e = trw_dev_malloc((void**)&br.list, sizeof(int32_t) * max_big);
  if (e == cudaSuccess) e = trw_dev_malloc((void**)&br.counters, sizeof(unsigned int) * 4);
  if (e == cudaSuccess) e = cudaMemsetAsync(br.counters, 0, sizeof(unsigned int) * 4, st);
  int64_t blocks = ((int64_t)nv + 255) / 256;
  if (blocks > 65535) blocks = 65535;
  if (e == cudaSuccess) {
    collect_big_rows<<<(unsigned)blocks, 256, 0, st>>>(nv, row_ptr, br.keys, br.counters + 2);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(&br.n, br.counters + 2, sizeof(unsigned int), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e == cudaSuccess && br.n > max_big) e = cudaErrorUnknown;  // cannot happen: each big row holds kBigRow edges
  if (e == cudaSuccess && br.n > 0) {
    std::vector<unsigned long long> hk(br.n);
    std::vector<int32_t> hb(br.n);
    e = cudaMemcpy(hk.data(), br.keys, sizeof(unsigned long long) * br.n, cudaMemcpyDeviceToHost);
    std::sort(hk.begin(), hk.end(), [](unsigned long long a, unsigned long long b) { return a > b; });
    for (unsigned int k = 0; k < br.n; ++k) hb[k] = (int32_t)(hk[k] & 0xffffffffu);
    if (e == cudaSuccess) e = cudaMemcpy(br.list, hb.data(), sizeof(int32_t) * br.n, cudaMemcpyHostToDevice);
  }
  return e;
}

template <typename K>
cudaError_t persistent_grid(K kernel, int threads, unsigned* grid) {
  int dev = 0, sms = 1, occ = 1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kernel, threads, 0);
  *grid = (unsigned)(sms * (occ > 0 ? occ : 1));
  return e;
}

}  // namespace

cudaError_t launch_prepare_alias(int32_t nv, int64_t ne, const int32_t* row_ptr, const int32_t* col,
                                 const float* weights, AliasRec* alias, unsigned long long* q_scratch,
                                 int32_t* idx_scratch, int32_t* part_scratch, Ctrl* ctrl, cudaStream_t st) {
  if (nv <= 0) return cudaSuccess;
  BigRows br;
  cudaError_t e = collect_big(nv, ne, row_ptr, st, br);
  unsigned grid = 1;
  if (e == cudaSuccess) e = persistent_grid(prepare_alias_kernel, kPrepThreads, &grid);
  if (e == cudaSuccess) {
    const Scratch sc{q_scratch, idx_scratch, part_scratch};
    prepare_alias_kernel<<<grid, kPrepThreads, 0, st>>>(nv, row_ptr, col, weights, alias, sc, br.list,
                                                        (int32_t)br.n, br.counters, ctrl);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  return e;
}

cudaError_t launch_neighbor_hash(int32_t nv, int64_t ne, const int32_t* row_ptr, const int32_t* col,
                                 int32_t min_degree, int32_t* slots, cudaStream_t st) {
  if (nv <= 0 || ne <= 0) return cudaSuccess;
  unsigned int* d_probe = nullptr;
  cudaError_t e = trw_dev_malloc((void**)&d_probe, sizeof(unsigned int));
  if (e == cudaSuccess) e = cudaMemsetAsync(d_probe, 0, sizeof(unsigned int), st);
  BigRows br;
  if (e == cudaSuccess) e = collect_big(nv, ne, row_ptr, st, br);
  unsigned grid = 1;
  if (e == cudaSuccess) e = persistent_grid(hash_insert_kernel, kPrepThreads, &grid);
  if (e == cudaSuccess) {
    hash_insert_kernel<<<grid, kPrepThreads, 0, st>>>(nv, row_ptr, col, min_degree, br.list, (int32_t)br.n,
                                                      br.counters, slots, d_probe);
    e = cudaGetLastError();
  }
  unsigned int full = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&full, d_probe, sizeof(full), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  cudaFree(d_probe);
  if (e == cudaSuccess && full != 0) e = cudaErrorUnknown;  // a table found full: cannot happen at load 1/2
  return e;
}

cudaError_t launch_label_max(const uint8_t* labels, int64_t ne, unsigned int* d_out, cudaStream_t st) {
  if (ne <= 0) return cudaSuccess;
  int64_t blocks = (ne + 255) / 256;
  if (blocks > 4096) blocks = 4096;
  label_max_kernel<<<(unsigned)blocks, 256, 0, st>>>(labels, ne, d_out);
  return cudaGetLastError();
}

cudaError_t launch_prepare_labels(int32_t nv, int64_t ne, const int32_t* row_ptr, const int32_t* col,
                                  const uint8_t* labels, int32_t nl, int32_t stride, int32_t* vrec, int32_t* erec,
                                  cudaStream_t st) {
  if (nv <= 0) return cudaSuccess;
  int64_t blocks = ((int64_t)nv + kLabelWarps - 1) / kLabelWarps;
  if (blocks > 65535) blocks = 65535;
  label_rows_kernel<<<(unsigned)blocks, kLabelWarps * 32, 0, st>>>(nv, row_ptr, col, labels, nl, stride, vrec, erec);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess && ne > 0) {
    int64_t eb = (ne + 255) / 256;
    if (eb > 65535) eb = 65535;
    label_gather_kernel<<<(unsigned)eb, 256, 0, st>>>(ne, stride, vrec, erec);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  return e;
}

cudaError_t launch_row_records(int32_t nv, int64_t ne, const int32_t* row_ptr, const int32_t* col,
                               const float* weights, bool sorted, RowRec* rec, cudaStream_t st) {
  if (ne <= 0) return cudaSuccess;
  int64_t blocks = (ne + 255) / 256;
  if (blocks > 65535) blocks = 65535;
  row_records_kernel<<<(unsigned)blocks, 256, 0, st>>>(nv, ne, row_ptr, col, weights, sorted, rec);
  return cudaGetLastError();
}

// Guided ITS records (ItsRec), one warp per row.  Pass 1: the row's prefix
// sums P'_j by warp scans, with each edge's destination and its row.  Pass 2:
// U_j = floor((P'_j * 2^64 - 1) / S) in place (0 where P'_j = 0).  Pass 3: the
// guide.  Cell k holds the draws r with floor(r * d / 2^64) = k, and its first
// candidate is the answer at its smallest draw (at least 1); the answer at r
// is the smallest j with r <= U_j, so edge j is the first candidate exactly of
// the cells from the one after U_{j-1}'s cell to U_j's cell (from cell 0 for
// the first positive edge): each edge writes its own cells, O(d) per row.  The
// last candidate of cell k is the first of cell k + 1 (d - 1 for the last).
__global__ void its_records_kernel(int32_t nv, const int32_t* __restrict__ row_ptr, const int32_t* __restrict__ col,
                                   const float* __restrict__ weights, ItsRec* __restrict__ rec) {
  const int lane = threadIdx.x & 31;
  const int64_t warps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  uint32_t* words = reinterpret_cast<uint32_t*>(rec);
  for (int64_t v = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; v < nv; v += warps) {
    const int32_t lo = row_ptr[v], hi = row_ptr[v + 1];
    const int32_t d = hi - lo;
    unsigned long long run = 0;
    for (int32_t base = lo; base < hi; base += 32) {
      const int32_t e = base + lane;
      const uint32_t w = e < hi ? weight_fixed(weights[e]) : 0u;
      unsigned long long incl = w;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const unsigned long long t = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += t;
      }
      if (e < hi) {
        const unsigned long long P = run + incl;
        const int32_t c = col[e];
        const int32_t co = row_ptr[c];
        rec[e].a = make_uint4((uint32_t)P, (uint32_t)(P >> 32), (uint32_t)c, (uint32_t)co);
        rec[e].b = make_uint4((uint32_t)(row_ptr[c + 1] - co), 0xffffffffu, 0xffffffffu, 0u);
      }
      run += __shfl_sync(0xffffffffu, incl, 31);
    }
    const unsigned long long S = run;
    if (S == 0) continue;  // no positive weight: every first candidate stays -1
    __syncwarp();
    for (int32_t e = lo + lane; e < hi; e += 32) {
      const unsigned long long P = ((unsigned long long)rec[e].a.y << 32) | rec[e].a.x;
      const unsigned long long U =
          P == 0 ? 0ull : (unsigned long long)((((unsigned __int128)P << 64) - 1u) / (unsigned __int128)S);
      rec[e].a.x = (uint32_t)U;
      rec[e].a.y = (uint32_t)(U >> 32);
    }
    __syncwarp();
    for (int32_t j = lane; j < d; j += 32) {
      const unsigned long long U = ((unsigned long long)rec[lo + j].a.y << 32) | rec[lo + j].a.x;
      if (U == 0) continue;  // zero prefix: never an answer
      const unsigned long long Up = j == 0 ? 0ull : ((unsigned long long)rec[lo + j - 1].a.y << 32) | rec[lo + j - 1].a.x;
      const int64_t k0 = Up == 0 ? 0 : (int64_t)__umul64hi(Up, (unsigned long long)d) + 1;
      const int64_t k1 = (int64_t)__umul64hi(U, (unsigned long long)d);
      for (int64_t k = k0; k <= k1; ++k) {
        words[8 * (int64_t)(lo + k) + 5] = (uint32_t)j;               // b.y of cell k
        if (k >= 1) words[8 * (int64_t)(lo + k - 1) + 6] = (uint32_t)j;  // b.z of cell k - 1
      }
    }
    if (lane == 0) words[8 * (int64_t)(hi - 1) + 6] = (uint32_t)(d - 1);
  }
}

cudaError_t launch_its_records(int32_t nv, const int32_t* row_ptr, const int32_t* col, const float* weights,
                               ItsRec* rec, cudaStream_t st) {
  if (nv <= 0) return cudaSuccess;
  int64_t blocks = ((int64_t)nv * 32 + 255) / 256;
  if (blocks > 65535) blocks = 65535;
  its_records_kernel<<<(unsigned)blocks, 256, 0, st>>>(nv, row_ptr, col, weights, rec);
  return cudaGetLastError();
}

cudaError_t launch_sampler_tables(int32_t nv, const int32_t* row_ptr, const float* weights, unsigned long long* cdf,
                                  uint32_t* pmax, cudaStream_t st) {
  if (nv <= 0) return cudaSuccess;
  int64_t blocks = ((int64_t)nv * 32 + 255) / 256;
  if (blocks > 65535) blocks = 65535;
  sampler_tables_kernel<<<(unsigned)blocks, 256, 0, st>>>(nv, row_ptr, weights, cdf, pmax);
  return cudaGetLastError();
}

cudaError_t launch_check_graph(int32_t nv, const int32_t* row_ptr, const int32_t* col, Ctrl* ctrl, int* d_unsorted,
                               cudaStream_t st) {
  if (nv <= 0) return cudaSuccess;
  int64_t blocks = ((int64_t)nv * 32 + 255) / 256;
  if (blocks > 65535) blocks = 65535;
  check_graph_kernel<<<(unsigned)blocks, 256, 0, st>>>(nv, row_ptr, col, ctrl, d_unsorted);
  return cudaGetLastError();
}

cudaError_t launch_check_weights(int64_t ne, const float* weights, Ctrl* ctrl, cudaStream_t st) {
  if (ne <= 0) return cudaSuccess;
  int64_t blocks = (ne + 255) / 256;
  if (blocks > 65535) blocks = 65535;
  check_weights_kernel<<<(unsigned)blocks, 256, 0, st>>>(ne, weights, ctrl);
  return cudaGetLastError();
}

}  // namespace trw
