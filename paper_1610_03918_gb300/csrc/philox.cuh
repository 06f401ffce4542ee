// Counter-based random numbers for the device: Philox4x32-10 (Salmon,
// Moraes, Dror and Shaw, "Parallel random numbers: as easy as 1, 2, 3",
// SC 2011), written from its published definition.  Ten rounds mix a
// 128-bit counter with a 64-bit key; a round forms the 64-bit products of
// counter words 0 and 2 with two fixed odd constants and recombines their
// halves with the other two words and the key, and the key is advanced by
// two fixed increments between rounds.  A draw is a pure function of its
// counter and key, so results do not depend on thread or particle order.
//
// Uses: the seeded He initialisation of the warm-start network and the
// thermal ions that replace absorbed ions (ion recycling), keyed by
// (seed, step, particle id).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace picgb {

constexpr uint32_t kPhiloxM0 = 0xD2511F53u;
constexpr uint32_t kPhiloxM1 = 0xCD9E8D57u;
constexpr uint32_t kPhiloxW0 = 0x9E3779B9u;
constexpr uint32_t kPhiloxW1 = 0xBB67AE85u;

__host__ __device__ inline uint32_t mulhi32(uint32_t a, uint32_t b) {
#ifdef __CUDA_ARCH__
  return __umulhi(a, b);
#else
  return uint32_t((uint64_t(a) * b) >> 32);
#endif
}

__host__ __device__ inline uint4 philox4x32_10(uint4 c, uint2 k) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r) {
      k.x += kPhiloxW0;
      k.y += kPhiloxW1;
    }
    const uint32_t hi0 = mulhi32(kPhiloxM0, c.x), lo0 = kPhiloxM0 * c.x;
    const uint32_t hi1 = mulhi32(kPhiloxM1, c.z), lo1 = kPhiloxM1 * c.z;
    c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
  }
  return c;
}

// The top 24 bits of a word as a float in [0, 1) (exact), and in (0, 1].
__host__ __device__ inline float unit24(uint32_t w) { return float(w >> 8) * 0x1p-24f; }
__host__ __device__ inline float unit24_open(uint32_t w) { return float((w >> 8) + 1u) * 0x1p-24f; }
// floor(w n / 2^32): a uniform integer in [0, n)
__host__ __device__ inline uint32_t below(uint32_t w, uint32_t n) { return mulhi32(w, n); }

// Counter tags of the draws (third counter word)
constexpr uint32_t kTagRecycle = 1u;
constexpr uint32_t kTagInit = 2u;

}  // namespace picgb
