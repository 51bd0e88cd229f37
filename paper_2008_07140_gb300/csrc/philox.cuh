// Philox4x32-10 counter-based generator (Salmon, Moraes, Dror, Shaw, SC'11): ten rounds
// of the 4x32 S-box; round multipliers 0xD2511F53 and 0xCD9E8D57, key schedule bumped by
// 0x9E3779B9 and 0xBB67AE85 between rounds. Usable from host and device code.
#pragma once
#include <cstdint>

#if defined(__CUDACC__)
#define QS_HD __host__ __device__ __forceinline__
#else
#define QS_HD inline
#endif

namespace qsim {

struct Philox4 {
  uint32_t v[4];
};

QS_HD void mulhilo32(uint32_t a, uint32_t b, uint32_t &hi, uint32_t &lo) {
#if defined(__CUDA_ARCH__)
  lo = a * b;
  hi = __umulhi(a, b);
#else
  const uint64_t p = (uint64_t)a * (uint64_t)b;
  lo = (uint32_t)p;
  hi = (uint32_t)(p >> 32);
#endif
}

QS_HD Philox4 philox4x32_10(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3, uint32_t k0,
                            uint32_t k1) {
#pragma unroll
  for (int round = 0; round < 10; ++round) {
    uint32_t hi0, lo0, hi1, lo1;
    mulhilo32(0xD2511F53u, c0, hi0, lo0);
    mulhilo32(0xCD9E8D57u, c2, hi1, lo1);
    const uint32_t n0 = hi1 ^ c1 ^ k0;
    const uint32_t n2 = hi0 ^ c3 ^ k1;
    c0 = n0;
    c1 = lo1;
    c2 = n2;
    c3 = lo0;
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
  Philox4 r;
  r.v[0] = c0;
  r.v[1] = c1;
  r.v[2] = c2;
  r.v[3] = c3;
  return r;
}

// 53-bit uniform double in [0, 1) from two words: ((x0 << 32 | x1) >> 11) * 2^-53.
QS_HD double u01_from(uint32_t x0, uint32_t x1) {
  const uint64_t w = ((uint64_t)x0 << 32) | (uint64_t)x1;
  return (double)(w >> 11) * (1.0 / 9007199254740992.0);
}

constexpr uint32_t kSampleTag = 0x53414D50u;  // counter word 3 of sampling draws

}  // namespace qsim
