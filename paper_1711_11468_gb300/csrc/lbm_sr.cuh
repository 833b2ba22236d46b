// Stochastic rounding of FP16-shifted storage. Round-to-nearest FP16 storage
// stagnates when the per-step change of a deviation d_i = f_i - w_i is below
// half its FP16 spacing (a slow body-force flow: 3 w_i c_i.F ~ 2e-8 against a
// spacing of 6e-8 near 1e-4). Rounding up with the probability of the
// remainder keeps every stored value unbiased, so the small increments survive
// on average.
//
// Random bits: splitmix64 (Steele, Lea and Flood, "Fast splittable
// pseudorandom number generators", OOPSLA 2014) used as a counter-based
// generator. Node `node` at sweep t draws its key, output number
// (t << 32) | node of the stream seeded with the lattice's seed, and four more
// words, outputs 0..3 of the stream the key seeds; direction j takes bits
// 16 (j mod 4) .. +15 of word j div 4.
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

// r / 2^16 as an FP32 value, for the 16 random bits of direction j.
__device__ __forceinline__ float sr_fraction(const unsigned long long (&w)[5], int j) {
  const unsigned word = (j % 4) < 2 ? (unsigned)w[j / 4] : (unsigned)(w[j / 4] >> 32);
  const unsigned bits = (j % 2) == 0 ? (word << 7) & 0x007FFF80u : (word >> 9) & 0x007FFF80u;
  return __uint_as_float(0x3F800000u | bits) - 1.0f;   // 1 + r 2^-16 is exact, and so is the subtraction
}

// FP32 -> FP16 bits with stochastic rounding: with u the FP16 spacing at |x|,
// the result is the FP16 neighbour of x away from zero if the remainder of |x|
// past the one towards zero plus r u reaches u, else that one. The fused
// multiply-add rounds towards zero, so |x| + r u stays below the next FP16 value
// exactly when the exact sum does: the decision is exact for the FP32 input.
// Finite values beyond the FP16 range saturate at 65504.
__device__ __forceinline__ unsigned short round_half_stochastic(float x, float r) {
  const unsigned e = __float_as_uint(x) & 0x7F800000u;
  const float u = __uint_as_float(max(e, 0x38800000u) - (10u << 23));   // 2^(max(e, -14) - 10)
  const float y = __fmaf_rz(r, u, fabsf(x));
  return __half_as_ushort(__float2half_rz(copysignf(y, x)));
}

}  // namespace lbm
