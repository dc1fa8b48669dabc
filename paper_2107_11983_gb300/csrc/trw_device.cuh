// Device-side building blocks of the walk kernels: the Philox4x32-10 block
// function, fixed-point sampling helpers, and the structs that describe a
// loaded graph and one walk request to a kernel.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/trw_draws.cuh"

namespace trw {

// Device algorithm ids: the public ones, the mixed-batch dispatcher, and
// weighted DeepWalk under the other samplers of Section 2.3.
enum Algo : int {
  DEEPWALK = 0, DEEPWALK_WEIGHTED = 1, PPR = 2, NODE2VEC = 3, METAPATH = 4, MIXED = 5,
  DW_ITS = 6,    // weighted DeepWalk, static ITS over the stored prefix sums
  DW_REJ = 7,    // weighted DeepWalk, REJ with the stored per-vertex bound p*_v
  DW_OREJ = 8,   // weighted DeepWalk, O-REJ with the caller's bound
  N2V_W = 9      // weighted Node2Vec: O-REJ darts pass Eq. 1's class word and a weight word
};

// Node2Vec, unweighted or weighted (the same second-order step).
__host__ __device__ constexpr bool is_n2v(int a) { return a == NODE2VEC || a == N2V_W; }

constexpr int kMaxSchema = 16;
constexpr uint32_t kRejectCap = 65536;

// Status words a kernel may leave in the control block.
constexpr int kErrInvalid = -1;
constexpr int kErrRejectCap = -6;
constexpr int kErrInternal = -9;

// ALIAS record of one edge slot, one 32-byte sector: the bucket's threshold
// H and both destinations, each with its own CSR row, so that an ALIAS move
// needs one random read and the next step no row-offset lookup.
//   a = {H, first dst, second dst, row offset of first dst}
//   b = {row offset of second dst, degree of first dst, degree of second dst, 0}
// A vertex with no positive weight has first = second = -1 in every record.
struct __align__(32) AliasRec {
  uint4 a;
  uint4 b;
};

// Row record of one edge slot e = (v -> dst), 16 bytes (an optional
// preparation; walks are identical with and without it):
//   a = {dst, row offset of dst, degree of dst, aux}
// On a weighted graph aux is W_e, the integer weight, which a REJ dart or a
// weighted O-REJ candidate reads.  On a graph without weights it is rev_e, the
// position in dst's row of the edge back to v (-1 when dst has none or the rows
// are not sorted): Node2Vec keeps it for the next step, where it decides a
// return-only dart without reading its candidate.  Two records share a 32-byte
// sector, so neighbouring edge slots of a row cost one DRAM sector.
struct __align__(16) RowRec {
  int4 a;
};

// Guided ITS records (an optional preparation; walks are identical with and
// without it).  ITS picks the smallest i with x < p'_i, x = floor(r64 * S / 2^64)
// and S = p'_{d-1}; since x < p'_i exactly when max(r64, 1) <= U_i with
//   U_i = floor((p'_i * 2^64 - 1) / S) for p'_i > 0, and U_i = 0 for p'_i = 0,
// the search runs on r64 itself and needs no S.  The draw's cell
// k = floor(r64 * d / 2^64) (one of d equal cells of the 64-bit draw space)
// bounds the answer: it lies between the answers at the smallest draws of
// cells k and k + 1, the guide entries of cell k (Chen and Asau's guide
// table, 1974).  One 32-byte record per edge slot j of a row:
//   a = {U_j low, U_j high, dst_j, row offset of dst_j}
//   b = {degree of dst_j, first candidate of cell j, last candidate of cell j, 0}
// A row without positive weight has first candidate -1 in every record.
struct __align__(32) ItsRec {
  uint4 a;
  uint4 b;
};

// MetaPath label index (an optional preparation; walks are identical with
// and without it).  Each row is stably partitioned by label, so the group of
// label l in row v, [g(v, l), g(v, l + 1)), lists the edges labelled l in CSR
// order and its r-th entry is the r-th matching edge of the row.  A vertex
// record is lstride int32 words {v, g(v, 0), ..., g(v, NL)} (NL labels,
// g(v, 0) = row_ptr[v], g(v, NL) = row_ptr[v + 1]); the edge record at
// partitioned slot e is the vertex record of that edge's destination, so a
// MetaPath move reads one record and learns both the next vertex and the
// bounds of its label groups for the next step.
struct LabelIndex {
  const int32_t* __restrict__ vrec;      // [nv * stride], or null when not prepared
  const int32_t* __restrict__ erec;      // [ne * stride]
  int32_t stride;                        // words per record: 8, 16 or 32 (NL + 2 rounded up)
  int32_t nl;                            // NL; a schema label >= NL has an empty group everywhere
};

// Neighbour hash (an optional preparation; walks are identical with and
// without it).  Every row u of at least min_degree entries owns an
// open-addressing table of 2 d(u) int32 slots at offset 2 row_ptr[u] of one
// array (so a lookup needs only the row it already holds): each neighbour v
// sits in the first empty slot at or after slot_of(v, 2 d(u)), wrapping
// within the row's table; empty slots hold -1, and the load factor is 1/2.
struct NeighborHash {
  const int32_t* __restrict__ slots;     // [2 ne], or null when not prepared
  int32_t min_degree;                    // rows shorter than this are searched in place
};

constexpr int32_t kHashEmpty = -1;

// MurmurHash3's 32-bit finaliser (Appleby): a bijective mix of the key bits.
__host__ __device__ __forceinline__ uint32_t mix32(uint32_t k) {
  k ^= k >> 16;
  k *= 0x85ebca6bu;
  k ^= k >> 13;
  k *= 0xc2b2ae35u;
  k ^= k >> 16;
  return k;
}

// First probe of key v in a table of cap slots: the mixed key scaled to
// [0, cap) by a 32x32-bit high product.
__host__ __device__ __forceinline__ uint32_t slot_of(int32_t v, uint32_t cap) {
  return (uint32_t)(((uint64_t)mix32((uint32_t)v) * cap) >> 32);
}

// A CSR graph resident in HBM.  Offsets and ids are int32 (nv, ne < 2^31).
struct DevGraph {
  const int32_t* __restrict__ row_ptr;   // [nv + 1]
  const int32_t* __restrict__ col;       // [ne], rows sorted ascending when sorted != 0
  const AliasRec* __restrict__ alias;    // [ne] after ALIAS preparation, or null
  const uint8_t* __restrict__ labels;    // [ne + 16] (padded for word loads), or null
  const float* __restrict__ weights;     // [ne] edge weights, or null
  const unsigned long long* __restrict__ cdf;  // [ne] ITS: inclusive prefix sums of the row's integer weights, or null
  const uint32_t* __restrict__ pmax;     // [nv] REJ: largest integer weight of the row (0: none positive), or null
  const ItsRec* __restrict__ its_rec;    // [ne] guided ITS records, or null
  const RowRec* __restrict__ rrec;       // [ne] row records, or null
  LabelIndex lidx;
  NeighborHash nh;
  int32_t nv;
  int32_t ne;
  int32_t rrec_rev;                     // 1: the records' aux word is rev_e (no weights), 0: W_e
};

// One walk request as a kernel sees it.  Thresholds are fixed-point
// probabilities in [0, 2^32]: a 32-bit word y succeeds when y < T.
struct WalkSpec {
  int32_t algo;
  int32_t max_len;            // moves
  uint32_t wps;               // walks per source
  uint32_t endpoints;         // 1: one output vertex per walk
  uint32_t key0, key1;        // Philox key (seed)
  uint32_t walk_offset;       // Philox counter word 0 of walk 0
  uint32_t schema_len;
  uint64_t T_stop;            // PPR stop threshold; DW_OREJ, N2V_W: the caller's bound P on the integer
                              // weights (>= 1; N2V_W: 0 for the row's p*_v)
  uint64_t T_ret, T_nb, T_far;// Node2Vec O-REJ thresholds (Eq. 1 over p*)
  uint64_t T_lo, T_hi;        // min / max of T_nb, T_far (skip IsNeighbor outside [T_lo, T_hi))
  const int32_t* sources;
  int32_t* out_paths;
  int32_t* out_lengths;
  int64_t nwalks;
  uint64_t schema_lo;         // MetaPath labels H[0..7], byte k = H[k]
  uint64_t schema_hi;         // H[8..15]
};

// MetaPath label H[k] of a packed schema (no dynamic indexing into local memory).
__device__ __forceinline__ uint32_t schema_label(const WalkSpec& sp, uint32_t k) {
  const uint64_t w = k < 8 ? sp.schema_lo : sp.schema_hi;
  return (uint32_t)(w >> (8 * (k & 7))) & 0xffu;
}

// Control block shared by the launches of one call (device memory).
struct Ctrl {
  unsigned long long head;    // next unclaimed walk of the work queue
  unsigned long long moves;   // total moves taken
  int err;                    // first error status (0 = none)
  int pad;
};

// -------------------------------------------------------------------- draws
// Philox4x32-10 and the uniform-integer rule, as every walk defines them
// (include/trw_draws.cuh, shared with user-defined walks).

__device__ __forceinline__ uint4 philox10(uint4 c, uint32_t k0, uint32_t k1) {
  return trw_draws::philox4x32_10(c, k0, k1);
}

// Draw `draw` of step `step` of walk `w`.
__device__ __forceinline__ uint4 draw_block(const WalkSpec& sp, uint32_t w, uint32_t step, uint32_t draw) {
  return philox10(make_uint4(w, step, draw, 0u), sp.key0, sp.key1);
}

using trw_draws::below;
using trw_draws::below64;

// Integer weight of a finite non-negative fp32 weight: round-half-even(w * 2^16),
// clamped to 2^32 - 1.  w * 2^16 is exact in fp32 (a power-of-two scale), and
// an fp32 value below 2^32 is at most 2^32 - 256, so the clamp is one compare.
__device__ __forceinline__ uint32_t weight_fixed(float w) {
  const float t = w * 65536.0f;
  return t >= 4294967296.0f ? 0xffffffffu : __float2uint_rn(t);
}

// Read-only loads through the non-coherent path.
__device__ __forceinline__ int32_t ldg(const int32_t* p) { return __ldg(p); }
__device__ __forceinline__ uint4 ldg(const uint4* p) { return __ldg(p); }
// A 32-byte record (32-byte aligned) in one load: one L1 request for its one
// sector, so its second half never depends on the line staying in L1 after
// the first half's fill.  Read-only data (non-coherent path).
__device__ __forceinline__ void ldg32(const void* p, uint4& a, uint4& b) {
  asm("ld.global.nc.v8.u32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
      : "=r"(a.x), "=r"(a.y), "=r"(a.z), "=r"(a.w), "=r"(b.x), "=r"(b.y), "=r"(b.z), "=r"(b.w)
      : "l"(p));
}

}  // namespace trw
