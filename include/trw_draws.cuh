/*
 * trw_draws.cuh -- the random draws of every walk of libtrw.so, for device
 * code (the library's kernels and user-defined walks, trw_custom.cuh).
 *
 * Draw `attempt` of step `step` of walk `walk` under a 64-bit seed is the
 * Philox4x32-10 block of counter (walk, step, attempt, 0) and key
 * (seed low, seed high) (Salmon, Moraes, Dror and Shaw, "Parallel Random
 * Numbers: As Easy as 1, 2, 3", SC 2011).  A uniform integer in [0, n) is the
 * high 64 bits of r64 * n with r64 = word 1 : word 0; words 2 and 3 are
 * 32-bit uniforms for acceptance tests.
 */
#ifndef TRW_DRAWS_CUH
#define TRW_DRAWS_CUH

#include <cstdint>
#include <cuda_runtime.h>

namespace trw_draws {

// Ten rounds of two 32x32->64 multiplies with a word swap and a round key;
// the key advances by the Weyl constants after every round.
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint32_t lo0 = 0xD2511F53u * c.x;
    const uint32_t hi0 = __umulhi(0xD2511F53u, c.x);
    const uint32_t lo1 = 0xCD9E8D57u * c.z;
    const uint32_t hi1 = __umulhi(0xCD9E8D57u, c.z);
    c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
  return c;
}

// The block of draw `attempt` of step `step` of walk `walk`.
__device__ __forceinline__ uint4 draw(uint64_t seed, uint32_t walk, uint32_t step, uint32_t attempt) {
  return philox4x32_10(make_uint4(walk, step, attempt, 0u), (uint32_t)seed, (uint32_t)(seed >> 32));
}

// Uniform integer in [0, n): high 64 bits of r64 * n, r64 = (B.y:B.x).
__device__ __forceinline__ uint32_t below(uint4 B, uint32_t n) {
  const unsigned long long r64 = ((unsigned long long)B.y << 32) | B.x;
  return (uint32_t)__umul64hi(r64, (unsigned long long)n);
}

// The same for a 64-bit n.
__device__ __forceinline__ unsigned long long below64(uint4 B, unsigned long long n) {
  const unsigned long long r64 = ((unsigned long long)B.y << 32) | B.x;
  return __umul64hi(r64, n);
}

}  // namespace trw_draws

#endif  // TRW_DRAWS_CUH
