// Double-float arithmetic: a value is the unevaluated sum hi + lo of two FP32
// numbers with |lo| <= ulp(hi)/2, about 48 significant bits. GB300 executes
// FP32 fused multiply-adds 58 times faster than FP64 ones, so the collision of
// the FP64-storage sweep can run here instead of on the FP64 pipe.
//
// Algorithms: Knuth's TwoSum and Dekker's FastTwoSum for error-free addition,
// the FMA-based TwoProduct, and the "sloppy" double-word addition and
// double-word multiplication analysed by Joldes, Muller and Popescu, "Tight and
// rigorous error bounds for basic building blocks of double-word arithmetic",
// ACM TOMS 44(2), 2017. The sloppy addition's error is bounded relative to the
// operands, which is what the sweep needs: it keeps absolute errors near 2^-48
// of the PDF magnitudes.
//
// Conversions to and from FP64 are integer bit manipulations, because FP64 <->
// FP32 conversion instructions run at the FP64 pipe's rate on this GPU.
#pragma once

#include <cstdint>

namespace lbm {

struct df32 {
  float hi, lo;
  df32() = default;
  __host__ __device__ constexpr df32(float h, float l) : hi(h), lo(l) {}
  __host__ __device__ constexpr explicit df32(float h) : hi(h), lo(0.f) {}
  __host__ __device__ constexpr explicit df32(int h) : hi((float)h), lo(0.f) {}
  __host__ __device__ constexpr explicit df32(double h) : hi((float)h), lo((float)(h - (double)(float)h)) {}
};

__device__ __forceinline__ df32 two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return df32(s, e);
}

// requires |a| >= |b| (or a == 0)
__device__ __forceinline__ df32 fast_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  return df32(s, __fsub_rn(b, __fsub_rn(s, a)));
}

__device__ __forceinline__ df32 operator+(df32 x, df32 y) {
  const df32 s = two_sum(x.hi, y.hi);
  const float e = __fadd_rn(s.lo, __fadd_rn(x.lo, y.lo));
  return fast_two_sum(s.hi, e);
}
__device__ __forceinline__ df32 operator-(df32 x) { return df32(-x.hi, -x.lo); }
__device__ __forceinline__ df32 operator-(df32 x, df32 y) { return x + (-y); }

__device__ __forceinline__ df32 operator*(df32 x, df32 y) {
  const float p = __fmul_rn(x.hi, y.hi);
  float e = __fmaf_rn(x.hi, y.hi, -p);
  e = __fmaf_rn(x.hi, y.lo, e);
  e = __fmaf_rn(x.lo, y.hi, e);
  return fast_two_sum(p, e);
}

// x / y: quotient of the high parts, one correction from the exact residual.
__device__ __forceinline__ df32 operator/(df32 x, df32 y) {
  const float r = __frcp_rn(y.hi);
  const float q1 = __fmul_rn(x.hi, r);
  const df32 res = x - y * df32(q1);
  const float q2 = __fmul_rn(res.hi, r);
  const df32 q = fast_two_sum(q1, q2);
  // second correction: brings the quotient to the double-float precision
  const df32 res2 = x - y * q;
  return q + df32(__fmul_rn(res2.hi, r));
}

// FP64 -> double-float. hi takes the leading 24 significant bits (truncated),
// lo the remaining 29 bits rounded to 24. Exact to 2^-48 relative for
// |d| in [2^-74, 2^127]; `out_of_range` is set for other values (zero, tiny,
// huge), which the caller converts again with split_f64_slow.
__device__ __forceinline__ df32 split_f64_fast(double d, bool& out_of_range) {
  const unsigned long long bits = (unsigned long long)__double_as_longlong(d);
  const unsigned hw = (unsigned)(bits >> 32), lw = (unsigned)bits;
  const unsigned e = (hw >> 20) & 0x7FFu;
  out_of_range |= (e - 949u) > (1150u - 949u);   // unsigned: e < 949 wraps around
  const unsigned sign = hw & 0x80000000u;
  const unsigned mag = (hw & 0x7FFFFFFFu) - (896u << 20);   // rebias the exponent to FP32
  const unsigned hb = __funnelshift_l(lw, mag, 3) | sign;   // exponent, 23 leading mantissa bits
  const unsigned rem = lw & 0x1FFFFFFFu;                    // the 29 bits hi dropped
  const unsigned scale = sign | ((e - 948u) << 23);         // +-2^(e - 1075)
  return df32(__uint_as_float(hb), __fmul_rn(__uint2float_rn(rem), __uint_as_float(scale)));
}

// Any FP64 value, through the conversion instructions (FP64 pipe).
__device__ __forceinline__ df32 split_f64_slow(double d) {
  const float h = __double2float_rz(d);
  return df32(h, __double2float_rn(d - (double)h));
}

// FP32 -> FP64 exactly (normal numbers and zero; FP32 subnormals, below
// 1.2e-38, become zero).
__device__ __forceinline__ double f32_to_f64(float f) {
  const unsigned b = __float_as_uint(f);
  const unsigned ex = b & 0x7F800000u;
  const unsigned hw = (b & 0x80000000u) | (((b & 0x7FFFFFFFu) >> 3) + (896u << 20));
  const unsigned lw = b << 29;
  const unsigned long long bits = ex ? (((unsigned long long)hw << 32) | lw) : 0ull;
  return __longlong_as_double((long long)bits);
}

// c_k . (x, y, z) for the D3Q19 directions k = 1..9, without multiplications.
template <typename A>
__device__ __forceinline__ A cdot(int k, A x, A y, A z) {
  switch (k) {
    case 1: return x;
    case 2: return y;
    case 3: return z;
    case 4: return x + y;
    case 5: return x - y;
    case 6: return x + z;
    case 7: return x - z;
    case 8: return y + z;
    default: return y - z;
  }
}

}  // namespace lbm
