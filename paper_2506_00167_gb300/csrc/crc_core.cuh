// GF(2) helpers of the TB CRC-24 check, shared by the batch CRC kernel
// (crc.cu) and the serving loop (serve.cu).
#pragma once

#include "internal.cuh"

namespace ldpcgb {
namespace crccore {

constexpr uint32_t kPolyFull = 0x1864CFBu;

// a(x) * b(x) mod g(x), deg a, b < 24.
__device__ __forceinline__ uint32_t gf2_mulmod(uint32_t a, uint32_t b) {
  uint64_t p = 0;
#pragma unroll
  for (int i = 0; i < 24; ++i)
    if ((b >> i) & 1u) p ^= static_cast<uint64_t>(a) << i;
#pragma unroll
  for (int i = 46; i >= 24; --i)
    if ((p >> i) & 1u) p ^= static_cast<uint64_t>(kPolyFull) << (i - 24);
  return static_cast<uint32_t>(p);
}

}  // namespace crccore
}  // namespace ldpcgb
