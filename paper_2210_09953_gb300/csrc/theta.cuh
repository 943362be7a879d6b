// Device-side realisation of the sketching matrix Theta (Sec. 2: a seeded
// Gaussian OSE that is generated, never stored).
//
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): ten rounds of
//   (c0,c1,c2,c3) -> (hi(M1 c2) ^ c1 ^ k0, lo(M1 c2), hi(M0 c0) ^ c3 ^ k1, lo(M0 c0))
// with the key bumped by the Weyl constants between rounds.  One call yields
// 16 bytes: Theta's row i at the 16 consecutive global rows 16q .. 16q+15 of X.
#pragma once
#include <stdint.h>

namespace rcqr {

__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int round = 0; round < 10; ++round) {
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

// The same ten rounds with the round keys given: rk[2r] = k0 + r W0 and
// rk[2r+1] = k1 + r W1 (mod 2^32), r = 0..9, e.g. as kernel parameters, so that
// no key arithmetic runs per call.
__device__ __forceinline__ uint4 philox4x32_10_keys(uint4 c, const uint32_t (&rk)[20]) {
#pragma unroll
  for (int round = 0; round < 10; ++round) {
    const uint32_t lo0 = 0xD2511F53u * c.x;
    const uint32_t hi0 = __umulhi(0xD2511F53u, c.x);
    const uint32_t lo1 = 0xCD9E8D57u * c.z;
    const uint32_t hi1 = __umulhi(0xCD9E8D57u, c.z);
    c = make_uint4(hi1 ^ c.y ^ rk[2 * round], lo1, hi0 ^ c.w ^ rk[2 * round + 1], lo0);
  }
  return c;
}

// The 16 bytes of Theta's row i for the 16-row block q (global rows 16q..16q+15).
__device__ __forceinline__ uint4 theta_block(uint64_t q, uint32_t i, uint32_t stream, uint64_t seed) {
  return philox4x32_10(make_uint4((uint32_t)q, (uint32_t)(q >> 32), i, stream), (uint32_t)seed,
                       (uint32_t)(seed >> 32));
}

__device__ __forceinline__ uint32_t word_of(const uint4 &w, int j) {
  return j == 0 ? w.x : (j == 1 ? w.y : (j == 2 ? w.z : w.w));
}

// Byte b (0..15) of the block: bits 8*(b%4) .. of word b/4.
__device__ __forceinline__ uint32_t byte_of(const uint4 &w, int b) {
  return (word_of(w, b >> 2) >> (8 * (b & 3))) & 0xFFu;
}

}  // namespace rcqr
