// Random-gather ceiling: dependent random loads of 4-, 8- or 16-byte records
// from a table in HBM, one chain of hops per thread (or several interleaved
// chains), with the occupancy of the walk kernels.  Each hop reads the record
// at the current index and derives the next index from it, as a walk step
// reads the record of its current vertex.  It measures the rate HBM serves
// such loads, the practical ceiling for the walk kernels.
#include <cstdint>
#include <cuda_runtime.h>

#include "trw_api_internal.h"

namespace {

// splitmix-style mix for the table contents and the chain starts
__device__ __forceinline__ uint64_t mix(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
  z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
  return z ^ (z >> 31);
}

template <int RB>
struct Rec;
template <>
struct Rec<4> { using T = uint32_t; };
template <>
struct Rec<8> { using T = uint2; };
template <>
struct Rec<16> { using T = uint4; };

__device__ __forceinline__ uint32_t first_word(uint32_t v) { return v; }
__device__ __forceinline__ uint32_t first_word(uint2 v) { return v.x ^ v.y; }
__device__ __forceinline__ uint32_t first_word(uint4 v) { return v.x ^ v.y ^ v.z ^ v.w; }

template <int RB>
__global__ void fill_table(typename Rec<RB>::T* t, uint64_t n) {
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x) {
    const uint64_t r = mix(i + 1);
    typename Rec<RB>::T v;
    uint32_t* w = reinterpret_cast<uint32_t*>(&v);
    for (int k = 0; k < RB / 4; ++k) w[k] = (uint32_t)(mix(r + k) >> 16);
    t[i] = v;
  }
}

template <int RB, int CH>
__global__ void __launch_bounds__(256) chase(const typename Rec<RB>::T* __restrict__ t, uint64_t n, int hops,
                                             unsigned long long* sink) {
  const uint64_t tid = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  uint32_t idx[CH];
#pragma unroll
  for (int c = 0; c < CH; ++c) idx[c] = (uint32_t)(mix(tid * CH + c + 7) % n);
  uint32_t acc = 0;
  for (int h = 0; h < hops; ++h) {
#pragma unroll
    for (int c = 0; c < CH; ++c) {
      const uint32_t x = first_word(__ldg(t + idx[c]));
      acc += x;
      idx[c] = (uint32_t)(((uint64_t)(x * 2654435761u + idx[c]) * n) >> 32);
    }
  }
  if (acc == 0x12345678u) atomicAdd(sink, 1ull);
}

template <int RB>
cudaError_t run(uint64_t table_bytes, int hops, int chains, double* lps, double* ms_out, int num_sms) {
  using T = typename Rec<RB>::T;
  const uint64_t n = table_bytes / RB;
  T* t = nullptr;
  unsigned long long* sink = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t e = trw_dev_malloc((void**)&t, n * RB);
  if (e == cudaSuccess) e = trw_dev_malloc((void**)&sink, sizeof(unsigned long long));
  if (e == cudaSuccess) fill_table<RB><<<num_sms * 8, 256>>>(t, n), e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  int bps = 0;
  if (e == cudaSuccess) {
    if (chains == 1) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, chase<RB, 1>, 256, 0);
    else if (chains == 2) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, chase<RB, 2>, 256, 0);
    else e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, chase<RB, 4>, 256, 0);
  }
  const int blocks = num_sms * (bps > 0 ? bps : 1);
  float best = 1e30f;
  for (int rep = 0; rep < 4 && e == cudaSuccess; ++rep) {
    e = cudaEventRecord(e0);
    if (chains == 1) chase<RB, 1><<<blocks, 256>>>(t, n, hops, sink);
    else if (chains == 2) chase<RB, 2><<<blocks, 256>>>(t, n, hops, sink);
    else chase<RB, 4><<<blocks, 256>>>(t, n, hops, sink);
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaEventRecord(e1);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    float ms = 0;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (rep > 0 && ms < best) best = ms;
  }
  if (e == cudaSuccess) {
    const double loads = (double)blocks * 256.0 * chains * hops;
    *lps = loads / (best / 1000.0);
    *ms_out = best;
  }
  cudaFree(t);
  cudaFree(sink);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  return e;
}

}  // namespace

extern "C" trw_status trw_gather_ceiling(int64_t table_bytes, int32_t record_bytes, int32_t hops_per_chain,
                                         int32_t chains_per_thread, double* loads_per_s, double* kernel_ms) {
  if (!loads_per_s || !kernel_ms) return trw_fail(TRW_ERR_INVALID, "NULL output");
  if (record_bytes != 4 && record_bytes != 8 && record_bytes != 16) return trw_fail(TRW_ERR_INVALID, "record_bytes 4, 8 or 16");
  if (table_bytes < 4096 || table_bytes / record_bytes > 0xffffffffLL) return trw_fail(TRW_ERR_INVALID, "table size");
  if (hops_per_chain < 1 || hops_per_chain > 100000) return trw_fail(TRW_ERR_INVALID, "hops_per_chain in [1, 1e5]");
  if (chains_per_thread != 1 && chains_per_thread != 2 && chains_per_thread != 4)
    return trw_fail(TRW_ERR_INVALID, "chains_per_thread 1, 2 or 4");
  int dev = 0, sms = 1;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaError_t e;
  if (record_bytes == 4) e = run<4>((uint64_t)table_bytes, hops_per_chain, chains_per_thread, loads_per_s, kernel_ms, sms);
  else if (record_bytes == 8) e = run<8>((uint64_t)table_bytes, hops_per_chain, chains_per_thread, loads_per_s, kernel_ms, sms);
  else e = run<16>((uint64_t)table_bytes, hops_per_chain, chains_per_thread, loads_per_s, kernel_ms, sms);
  if (e != cudaSuccess) return trw_cuda_fail(e, "gather ceiling");
  return TRW_OK;
}
