// Philox4x32-10 counter-based generator on the device.
//
// Written from the published definition (Salmon, Moraes, Dror, Shaw, "Parallel random
// numbers: as easy as 1, 2, 3", SC'11): ten rounds, each multiplying counter words 0 and
// 2 by two fixed odd constants, exchanging the 64-bit product halves with words 1 and 3
// and the key, and bumping the key by two Weyl constants between rounds.
#pragma once
#include <cstdint>

namespace pim {

struct PhiloxOut {
  uint32_t x0, x1, x2, x3;
};

__device__ __forceinline__ PhiloxOut philox4x32_10(uint32_t c0, uint32_t c1, uint32_t c2,
                                                   uint32_t c3, uint32_t k0, uint32_t k1) {
  constexpr uint32_t kMulA = 0xD2511F53u;
  constexpr uint32_t kMulB = 0xCD9E8D57u;
  constexpr uint32_t kWeylA = 0x9E3779B9u;
  constexpr uint32_t kWeylB = 0xBB67AE85u;
#pragma unroll
  for (int round = 0; round < 10; ++round) {
    const uint32_t hiA = __umulhi(kMulA, c0);
    const uint32_t loA = kMulA * c0;
    const uint32_t hiB = __umulhi(kMulB, c2);
    const uint32_t loB = kMulB * c2;
    const uint32_t n0 = hiB ^ c1 ^ k0;
    const uint32_t n2 = hiA ^ c3 ^ k1;
    c0 = n0;
    c1 = loB;
    c2 = n2;
    c3 = loA;
    k0 += kWeylA;
    k1 += kWeylB;
  }
  return PhiloxOut{c0, c1, c2, c3};
}

// Same generator with the ten round keys given explicitly: rk[2r] = k0 + r * 0x9E3779B9,
// rk[2r+1] = k1 + r * 0xBB67AE85.  Passing them from the kernel parameter space lets every
// XOR read its key straight from the constant bank.
__device__ __forceinline__ PhiloxOut philox4x32_10_rk(uint32_t c0, uint32_t c1, uint32_t c2,
                                                      uint32_t c3, const uint32_t* rk) {
  constexpr uint32_t kMulA = 0xD2511F53u;
  constexpr uint32_t kMulB = 0xCD9E8D57u;
#pragma unroll
  for (int round = 0; round < 10; ++round) {
    const uint32_t hiA = __umulhi(kMulA, c0);
    const uint32_t loA = kMulA * c0;
    const uint32_t hiB = __umulhi(kMulB, c2);
    const uint32_t loB = kMulB * c2;
    const uint32_t n0 = hiB ^ c1 ^ rk[2 * round];
    const uint32_t n2 = hiA ^ c3 ^ rk[2 * round + 1];
    c0 = n0;
    c1 = loB;
    c2 = n2;
    c3 = loA;
  }
  return PhiloxOut{c0, c1, c2, c3};
}

// 16-bit draw for spin i from the block of i>>3: word (i&7)>>1, low half for even i.
__device__ __forceinline__ uint32_t philox_half(const PhiloxOut& o, int k) {
  const uint32_t w = (k >> 1) == 0 ? o.x0 : (k >> 1) == 1 ? o.x1 : (k >> 1) == 2 ? o.x2 : o.x3;
  return (k & 1) ? (w >> 16) : (w & 0xFFFFu);
}

}  // namespace pim
