// Philox4x32-10 counter-based generator (Salmon, Moraes, Dror, Shaw, SC'11,
// Sec. 3), the hash that recreates B, Pi, G and C from a seed. Written from
// the published round function: both 32x32->64 products of counter words 0
// and 2 with the multipliers M0, M1, high halves mixed with words 1, 3 and
// the key, key bumped by the Weyl constants W0, W1 between rounds.
#pragma once
#include <cstdint>

namespace mck {

struct U32x4 {
  uint32_t x, y, z, w;
};

__host__ __device__ __forceinline__ uint32_t mulhi_u32(uint32_t a, uint32_t b) {
#ifdef __CUDA_ARCH__
  return __umulhi(a, b);
#else
  return static_cast<uint32_t>((static_cast<uint64_t>(a) * b) >> 32);
#endif
}

__host__ __device__ __forceinline__ U32x4 philox4x32_10(uint32_t c0, uint32_t c1, uint32_t c2,
                                                        uint32_t c3, uint32_t k0, uint32_t k1) {
  constexpr uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
  constexpr uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r) {
      k0 += W0;
      k1 += W1;
    }
    const uint32_t hi0 = mulhi_u32(M0, c0), lo0 = M0 * c0;
    const uint32_t hi1 = mulhi_u32(M1, c2), lo1 = M1 * c2;
    const uint32_t n0 = hi1 ^ c1 ^ k0;
    const uint32_t n2 = hi0 ^ c3 ^ k1;
    c0 = n0;
    c1 = lo1;
    c2 = n2;
    c3 = lo0;
  }
  return {c0, c1, c2, c3};
}

// Counter tags (word c2) of the draws of one plan.
enum : uint32_t {
  kTagB = 1,           // B_e[k] sign: bit 0 of word 0 at (k, e, 1, 0)
  kTagPerm = 2,        // Fisher-Yates draw of step i at (i, e, 2, 0)
  kTagG = 3,           // G_e[k] at (k, e, 3, 0)
  kTagRbf = 4,         // Marsaglia-Tsang trial j of radius k at (k, e, 4, j)
  kTagBall = 5,        // Matern ball point j, coords 2p, 2p+1 at (p, e, 5 + 16 k, j)
  kTagBallRadius = 6,  // Matern ball point j radius draw at (k, e, 6, j)
  kTagLaplace = 7,     // normal divisor of Laplacian radius k at (k, e, 7, 0)
};

}  // namespace mck
