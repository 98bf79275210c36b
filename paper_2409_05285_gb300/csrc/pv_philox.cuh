// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11), written from the published round
// function: 64-bit products of counter words 0 and 2 with two multipliers, a xor of
// the high halves with the other counter words and the key, and a Weyl key schedule.
#pragma once

#include <cstdint>

#if defined(__CUDACC__)
#define PX_HD __host__ __device__ __forceinline__
#else
#define PX_HD inline
#endif

namespace pv {

struct U4 {
  uint32_t x[4];
};

PX_HD U4 philox4x32_10(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3, uint32_t k0,
                       uint32_t k1) {
  const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
  const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
  for (int r = 0; r < 10; ++r) {
    uint64_t p0 = (uint64_t)M0 * c0;
    uint64_t p1 = (uint64_t)M1 * c2;
    uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    uint32_t n0 = hi1 ^ c1 ^ k0, n2 = hi0 ^ c3 ^ k1;
    c0 = n0;
    c1 = lo1;
    c2 = n2;
    c3 = lo0;
    k0 += W0;
    k1 += W1;
  }
  U4 o;
  o.x[0] = c0;
  o.x[1] = c1;
  o.x[2] = c2;
  o.x[3] = c3;
  return o;
}

// Uniform double in [0, 1) from the first two output words: 53 bits (x0 << 21 | x1 >> 11).
PX_HD double philox_uniform(uint64_t seed, uint32_t c0, uint32_t c1, uint32_t c2, uint32_t tag) {
  U4 o = philox4x32_10(c0, c1, c2, tag, (uint32_t)seed, (uint32_t)(seed >> 32));
  uint64_t u53 = ((uint64_t)o.x[0] << 21) | (uint64_t)(o.x[1] >> 11);
  return (double)u53 * (1.0 / 9007199254740992.0);
}

PX_HD uint32_t philox_bits(uint64_t seed, uint32_t c0, uint32_t c1, uint32_t c2, uint32_t tag) {
  return philox4x32_10(c0, c1, c2, tag, (uint32_t)seed, (uint32_t)(seed >> 32)).x[0];
}

// Stream tags (fourth counter word).
constexpr uint32_t TAG_INIT = 0x494E4954u;
constexpr uint32_t TAG_CFG = 0x43464731u;
constexpr uint32_t TAG_MC = 0x4D435357u;
constexpr uint32_t TAG_DIRECT = 0x44495231u;
constexpr uint32_t TAG_FINIT = 0x46494E54u;   // perturbation of the fermionic beta = 0 state
constexpr uint32_t TAG_FMC = 0x464D4331u;     // fermionic Metropolis acceptance uniforms

}  // namespace pv
