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
#include <cstdint>
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

// Record of a bucket whose first element is destination u (taken with
// probability H / 2^32) and whose second is v.
__device__ __forceinline__ AliasRec make_rec(const int32_t* __restrict__ row_ptr, uint32_t H, int32_t u, int32_t v) {
  const int32_t ou = row_ptr[u], ov = row_ptr[v];
  AliasRec r;
  r.a = make_uint4(H, (uint32_t)u, (uint32_t)v, (uint32_t)ou);
  r.b = make_uint4((uint32_t)ov, (uint32_t)(row_ptr[u + 1] - ou), (uint32_t)(row_ptr[v + 1] - ov), 0u);
  return r;
}

__global__ void prepare_alias_kernel(int32_t nv, const int32_t* __restrict__ row_ptr,
                                     const int32_t* __restrict__ col, const float* __restrict__ weights,
                                     AliasRec* __restrict__ alias, unsigned long long* __restrict__ q,
                                     int32_t* __restrict__ small, int32_t* __restrict__ large, Ctrl* ctrl) {
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < nv; v += (int64_t)gridDim.x * blockDim.x) {
    const int32_t off = row_ptr[v];
    const int32_t d = row_ptr[v + 1] - off;
    if (d == 0) continue;
    unsigned long long S = 0;
    bool ok = true;
    for (int32_t j = 0; j < d; ++j) {
      uint32_t W;
      ok &= quantize(weights[off + j], W);
      S += W;
    }
    if (!ok) {
      atomicCAS(&ctrl->err, 0, kErrInvalid);
      continue;
    }
    if (S == 0) {
      AliasRec dead;
      dead.a = make_uint4(0u, 0xffffffffu, 0xffffffffu, 0u);
      dead.b = make_uint4(0u, 0u, 0u, 0u);
      for (int32_t j = 0; j < d; ++j) alias[off + j] = dead;
      continue;
    }
    int32_t ns = 0, nl = 0;
    for (int32_t j = 0; j < d; ++j) {
      uint32_t W;
      quantize(weights[off + j], W);
      const unsigned long long qj = (unsigned long long)d * W;
      q[off + j] = qj;
      if (qj < S) small[off + ns++] = j;
      else large[off + nl++] = j;
    }
    int32_t sh = 0, st = ns, lh = 0;
    while (sh < st && lh < nl) {
      const int32_t s = small[off + sh++];
      const int32_t l = large[off + lh];
      const unsigned long long qs = q[off + s];
      alias[off + s] = make_rec(row_ptr, frac32(qs, S), col[off + s], col[off + l]);
      const unsigned long long ql = q[off + l] - (S - qs);
      q[off + l] = ql;
      if (ql < S) {
        ++lh;
        small[off + st++] = l;
      }
    }
    for (; lh < nl; ++lh) {
      const int32_t j = large[off + lh];
      alias[off + j] = make_rec(row_ptr, 0xffffffffu, col[off + j], col[off + j]);
    }
    for (; sh < st; ++sh) {
      const int32_t j = small[off + sh];
      alias[off + j] = make_rec(row_ptr, 0xffffffffu, col[off + j], col[off + j]);
    }
  }
}

// Every id in [0, nv); flags a row that is not strictly increasing.
__global__ void check_graph_kernel(int32_t nv, const int32_t* __restrict__ row_ptr, const int32_t* __restrict__ col,
                                   Ctrl* ctrl, int* unsorted) {
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < nv; v += (int64_t)gridDim.x * blockDim.x) {
    const int32_t lo = row_ptr[v], hi = row_ptr[v + 1];
    int32_t last = -1;
    bool bad_order = false;
    for (int32_t e = lo; e < hi; ++e) {
      const int32_t c = col[e];
      if (c < 0 || c >= nv) {
        atomicCAS(&ctrl->err, 0, kErrInvalid);
        break;
      }
      if (c <= last) bad_order = true;
      last = c;
    }
    if (bad_order) atomicExch(unsorted, 1);
  }
}

}  // namespace

cudaError_t launch_prepare_alias(int32_t nv, const int32_t* row_ptr, const int32_t* col, const float* weights,
                                 AliasRec* alias, unsigned long long* q_scratch, int32_t* small_scratch,
                                 int32_t* large_scratch, Ctrl* ctrl, cudaStream_t st) {
  if (nv <= 0) return cudaSuccess;
  int64_t blocks = ((int64_t)nv + 127) / 128;
  if (blocks > 65535) blocks = 65535;
  prepare_alias_kernel<<<(unsigned)blocks, 128, 0, st>>>(nv, row_ptr, col, weights, alias, q_scratch, small_scratch,
                                                         large_scratch, ctrl);
  return cudaGetLastError();
}

cudaError_t launch_check_graph(int32_t nv, const int32_t* row_ptr, const int32_t* col, Ctrl* ctrl, int* d_unsorted,
                               cudaStream_t st) {
  if (nv <= 0) return cudaSuccess;
  int64_t blocks = ((int64_t)nv + 255) / 256;
  if (blocks > 65535) blocks = 65535;
  check_graph_kernel<<<(unsigned)blocks, 256, 0, st>>>(nv, row_ptr, col, ctrl, d_unsorted);
  return cudaGetLastError();
}

}  // namespace trw
