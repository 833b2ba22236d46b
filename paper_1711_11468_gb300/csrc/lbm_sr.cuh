// Stochastic rounding of scaled FP16-shifted storage. Round-to-nearest FP16
// storage stagnates when the per-step change of a deviation d_i = f_i - w_i is
// below half its FP16 spacing (a slow body-force flow: 3 w_i c_i.F ~ 2e-8
// against a spacing of 6e-8 near 1e-4). Rounding up with the probability of
// the remainder keeps every stored value unbiased, so the small increments
// survive on average.
//
// The format stores d_i 2^14 (kSrScaleLog2): FP16's normal range then covers
// |d| from 2^-28 to 4, and for a number in that range stochastic rounding of an
// FP32 value is one integer addition: add 13 random bits to its bit pattern
// (the 13 bits FP32 keeps below the FP16 spacing) and truncate to FP16. The
// result is the FP16 neighbour away from zero exactly when the 13 dropped bits
// plus the draw carry, i.e. with probability (remainder / spacing), without
// bias. Below 2^-14 (scaled) the addition covers less than one FP16 spacing and
// the rounding leans towards zero; those values are below 2^-28 unscaled.
//
// Random bits: splitmix64 (Steele, Lea and Flood, "Fast splittable
// pseudorandom number generators", OOPSLA 2014) used as a counter-based
// generator. Node `node` at sweep t draws its key, output number
// (t << 32) | node of the stream seeded with the lattice's seed, and four more
// words, outputs 0..3 of the stream the key seeds; direction j reads the 32-bit
// half (j mod 4) div 2 of word j div 4 and takes its bits 0..12 (even j) or
// 19..31 (odd j).
#pragma once

#include <cuda_fp16.h>
#include <cstdint>

namespace lbm {

constexpr unsigned long long kSplitmixGamma = 0x9E3779B97F4A7C15ull;

// splitmix64's output function ("mix64").
__device__ __forceinline__ unsigned long long splitmix_mix(unsigned long long z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

// The five words of a node: w[0] = key = mix(base + node * gamma), where
// base = seed + gamma (1 + (t << 32)) folds in the sweep; w[m] = mix(key + m gamma).
__device__ __forceinline__ void sr_words(unsigned long long base, uint32_t node, unsigned long long (&w)[5]) {
  w[0] = splitmix_mix(base + (unsigned long long)node * kSplitmixGamma);
#pragma unroll
  for (int m = 1; m < 5; ++m) w[m] = splitmix_mix(w[0] + (unsigned long long)m * kSplitmixGamma);
}

constexpr int kSrScaleLog2 = 14;

// The 13 random bits of direction j.
__device__ __forceinline__ unsigned sr_bits(const unsigned long long (&w)[5], int j) {
  const unsigned half = (j % 4) < 2 ? (unsigned)w[j / 4] : (unsigned)(w[j / 4] >> 32);
  return (j % 2) == 0 ? (half & 0x1FFFu) : (half >> 19);
}

// FP32 -> FP16 bits, stochastically: the draw is added to the magnitude bits
// (a carry out of the mantissa moves to the next binade, which is the value
// the rounding goes up to), then the conversion truncates. Infinities may turn
// into NaN; finite values beyond the FP16 range saturate at 65504.
__device__ __forceinline__ unsigned short round_half_stochastic(float x, unsigned r13) {
  return __half_as_ushort(__float2half_rz(__uint_as_float(__float_as_uint(x) + r13)));
}

}  // namespace lbm
