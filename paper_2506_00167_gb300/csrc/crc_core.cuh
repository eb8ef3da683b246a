// GF(2) helpers of the TB CRC-24 check, shared by the batch CRC kernel
// (crc.cu) and the serving loop (serve.cu).
#pragma once

#include "internal.cuh"

namespace ldpcgb {
namespace crccore {

constexpr uint32_t kPolyFull = 0x1864CFBu;   // g(x), one per transport block
constexpr uint32_t kPolyFullB = 0x1800063u;  // g_B(x), one per code block of a segmented TB

// a(x) * b(x) mod g(x), deg a, b < 24; `poly` = g(x) with its x^24 term.
__device__ __forceinline__ uint32_t gf2_mulmod(uint32_t a, uint32_t b, uint32_t poly = kPolyFull) {
  uint64_t p = 0;
#pragma unroll
  for (int i = 0; i < 24; ++i)
    if ((b >> i) & 1u) p ^= static_cast<uint64_t>(a) << i;
#pragma unroll
  for (int i = 46; i >= 24; --i)
    if ((p >> i) & 1u) p ^= static_cast<uint64_t>(poly) << (i - 24);
  return static_cast<uint32_t>(p);
}

// One table step of an MSB-first CRC-24 register: eight more message bits.
__device__ __forceinline__ uint32_t crc_byte_step(uint32_t state, uint32_t byte, const uint32_t* table) {
  return ((state << 8) & 0xFFFFFFu) ^ table[((state >> 16) ^ byte) & 0xFFu];
}

// Byte j of a block's bit-packed bits (bit i at bit i % 32 of word i / 32),
// with its first bit in time as the most significant bit.
__device__ __forceinline__ uint32_t msb_first_byte(uint32_t word, int j) {
  return __brev((word >> (8 * (j & 3))) & 0xFFu) >> 24;
}

}  // namespace crccore
}  // namespace ldpcgb
