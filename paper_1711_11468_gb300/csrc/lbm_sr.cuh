// Stochastic rounding of scaled FP16-shifted storage. Round-to-nearest FP16
// storage stagnates when the per-step change of a deviation d_i = f_i - w_i is
// below half its FP16 spacing (a slow body-force flow: 3 w_i c_i.F ~ 2e-8
// against a spacing of 6e-8 near 1e-4). Rounding up with the probability of
// the remainder keeps every stored value unbiased, so the small increments
// survive on average.
//
// The format stores d_i 2^14 (kSrScaleLog2): FP16's normal range then covers
// |d| from 2^-28 to 4. The rule: with q the remainder of |x| in FP16 spacings
// and r a 13-bit draw, |x| rounds to the FP16 neighbour away from zero iff
// q + r / 2^13 >= 1, in every binade. For an FP32 value in FP16's normal range
// that is one integer addition: FP32 keeps exactly 13 bits below the FP16
// spacing there, so adding r to the bit pattern carries into the FP16 bits iff
// the rule says "away", and truncation to FP16 finishes the rounding. Below
// 2^-14 FP16's spacing is fixed (2^-24) and FP32 keeps more than 13 bits below
// it, so there the value is first cut to a fixed-point count of 2^-37 units
// (the truncation cannot change the decision: r is an integer), then the draw
// is added and the carry taken.
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

constexpr float kSrNormalMin = 6.103515625e-05f;   // 2^-14, FP16's smallest normal number

// FP32 -> FP16 bits, stochastically, for |x| >= 2^-14 (or x = 0): the draw is
// added to the magnitude bits (a carry out of the mantissa moves to the next
// binade, which is the value the rounding goes up to), then the conversion
// truncates. Finite values beyond the FP16 range saturate at 65504; non-finite
// values are outside the format.
__device__ __forceinline__ unsigned short round_half_stochastic_normal(float x, unsigned r13) {
  return __half_as_ushort(__float2half_rz(__uint_as_float(__float_as_uint(x) + r13)));
}

// The same rule for any finite x, by integer arithmetic on the bit pattern.
// Exponent field E >= 113 (|x| >= 2^-14): re-biasing the exponent (127 -> 15)
// and dropping the 13 low bits after adding the draw gives the FP16 pattern,
// saturated at 65504. E < 113: |x| = M 2^(E-150) with M the 24-bit significand,
// so M >> (113 - E) = floor(|x| 2^37), a count of 1/2^13 FP16 subnormal
// spacings; adding the draw and dropping 13 bits gives the subnormal count (a
// count of 1024 is the pattern of 2^-14, the next value up). FP32 subnormals
// and zero lie below 2^-37 and give 0.
__device__ __forceinline__ unsigned short round_half_stochastic_any(float x, unsigned r13) {
  const unsigned b = __float_as_uint(x);
  const unsigned ab = b & 0x7FFFFFFFu;
  const unsigned e = ab >> 23;
  unsigned h;
  if (e >= 113u) {
    h = min((ab + r13 - (112u << 23)) >> 13, 0x7BFFu);
  } else {
    const unsigned m = (ab & 0x7FFFFFu) | 0x800000u;
    h = ((m >> min(113u - e, 31u)) + r13) >> 13;
  }
  return (unsigned short)(h | ((b >> 16) & 0x8000u));
}

}  // namespace lbm
