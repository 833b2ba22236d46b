// TRT collision of FP64-stored PDFs in FP32 arithmetic, for nodes near
// equilibrium: the "grid" double-float form. GB300 runs FP32 58 times faster
// than FP64; the general double-float collision (collide<df32>) spends most
// of its instructions renormalising sums. Here the work is arranged so that
// almost every addition is exact in FP32:
//
//  1. Split. Each PDF f_i (FP64) gives the exact fixed-point deviation
//     D_i = (f_i - w_i) 2^60 (a 64-bit integer: the significand shifted, minus
//     w_i 2^60 rounded), split at a grid 2^-(28+k) into an FP32 high part H_i
//     (the multiple of the grid, exact) and an FP32 low part L_i (the bits
//     below it, rounded to 24 bits: error below 2^-(52+k)). k (0..8) is chosen
//     per node from sum |D_i|: the finest grid on which the sums in step 2 stay
//     exact, so small deviations (slow flows) keep FP64-class resolution.
//  2. Moments. Every sum of H values (pair sums and differences, density,
//     momentum, c.j of the edges) lies on the grid and, by the choice of k,
//     below 2^24 grid units, so FP32 adds it exactly. The L parts are summed in
//     FP32 (errors near 2^-(52+k)).
//  3. Products with the TRT constants and the quadratic equilibrium terms use
//     unnormalised double-float pairs (hi, lo): an FMA-exact product of the
//     high parts plus first-order cross terms, and Knuth's TwoSum for sums of
//     terms that are not on a common grid. Relative error about 2^-46 of the
//     terms, i.e. below 1e-17 absolute for the non-equilibrium parts (<= 1e-3)
//     these produce.
//  4. Join. The increment f*_i - f_i (a double-float) is added to the exact
//     stored f_i in FP64: either as two FP64 additions of its exactly
//     converted parts, or as one FP64 addition of the part pair assembled
//     exactly into one FP64 value by integer operations (fewer FP64-pipe
//     instructions, more integer ones); kJoin1 selects per direction.
//
// Range of the path: every f_i in [2^-8, 1) and 2 sum |f_i - w_i| + 2 |F / w-|_1
// below 2^-4 (about |u| < 0.02 on the lattice's typical flows); other nodes
// take collide<df32>. The decision depends on the node's own values only, so
// results do not depend on launch shapes.
//
// Algorithms: TwoSum (Knuth), FastTwoSum (Dekker), FMA TwoProduct, as in
// lbm_df32.cuh.
#pragma once

#include <cstdint>

#include "lbm_df32.cuh"

namespace lbm {
namespace dfg {

// ---------------------------------------------------------------- constants
// w_c 2^60 rounded to an integer (rest, face, edge)
__host__ __device__ constexpr unsigned long long wfix(int c) {
  return c == 0 ? ((1ull << 60) + 1ull) / 3ull : (c == 1 ? ((1ull << 60) + 9ull) / 18ull : ((1ull << 60) + 18ull) / 36ull);
}

// ---------------------------------------------------------------- pairs
struct dd {
  float h, l;
};

__device__ __forceinline__ dd two_sum_dd(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return {s, e};
}
// (x.h + y.h) exactly, plus the low parts: 8 instructions, unnormalised.
__device__ __forceinline__ dd add(dd x, dd y) {
  const dd s = two_sum_dd(x.h, y.h);
  return {s.h, __fadd_rn(s.l, __fadd_rn(x.l, y.l))};
}
__device__ __forceinline__ dd neg(dd x) { return {-x.h, -x.l}; }
// constant c (c.h + c.l) times x: the product of the high parts exactly (FMA),
// plus the two cross terms.
__device__ __forceinline__ dd mul(df32 c, dd x) {
  const float p = __fmul_rn(c.hi, x.h);
  float e = __fmaf_rn(c.hi, x.h, -p);
  e = __fmaf_rn(c.hi, x.l, e);
  e = __fmaf_rn(c.lo, x.h, e);
  return {p, e};
}
__device__ __forceinline__ dd mul(dd c, dd x) { return mul(df32(c.h, c.l), x); }
// x^2: exact square of the high part plus the cross term.
__device__ __forceinline__ dd sqr(dd x) {
  const float p = __fmul_rn(x.h, x.h);
  float e = __fmaf_rn(x.h, x.h, -p);
  e = __fmaf_rn(__fadd_rn(x.h, x.h), x.l, e);
  return {p, e};
}
// scaling by a power of two (exact)
__device__ __forceinline__ dd scale(dd x, float s) { return {x.h * s, x.l * s}; }

// ---------------------------------------------------------------- join
// FP32 -> FP64 by integer operations for a value added to f >= 2^-8 (all PDFs
// on this path): normal numbers convert exactly; zero and FP32 subnormals come
// out as magnitudes below 2^-125, which the addition to f absorbs exactly, so
// the conversion needs no test for them.
__device__ __forceinline__ double f32_to_f64_added(float v) {
  const uint32_t b = __float_as_uint(v);
  const uint32_t hw = (((b & 0x7FFFFFFFu) >> 3) + (896u << 20)) | (b & 0x80000000u);
  return __hiloint2double((int)hw, (int)(b << 29));
}
// f + (h + l) with two FP64 additions of the converted parts.
__device__ __forceinline__ double join2(double f, dd x) {
  return (f + f32_to_f64_added(x.h)) + f32_to_f64_added(x.l);
}

// h + l as one FP64 value, by integer operations, for |l| <= ulp(h)/2 (a
// FastTwoSum result) and h normal. h's FP64 pattern has 29 zero bits below its
// FP32 mantissa; l, at most half a unit of h's last FP32 bit, lies within
// them: its 24-bit significand shifted to h's FP64 spacing (bits below that
// spacing are dropped, an error below 2^-52 |h|) is added to or, for opposite
// signs, subtracted from the 64-bit pattern. A subtraction borrows across the
// binade boundary only when h is a power of two, where the spacing below is
// half as large: the amount is doubled there. The value is only ever added to
// a PDF of at least 2^-8, so zero or subnormal parts need no test: they yield
// magnitudes below 2^-66 (h zero: about 2^-127; l zero: nothing, or an amount
// below h's last bit when |h| < 2^-66), which that addition absorbs exactly.
__device__ __forceinline__ double pair_to_f64(dd x) {
  const uint32_t hb = __float_as_uint(x.h), lb = __float_as_uint(x.l);
  const uint32_t ah = hb & 0x7FFFFFFFu;
  const uint32_t hw = ((ah >> 3) + (896u << 20)) | (hb & 0x80000000u);
  const uint32_t lw = hb << 29;
  const int sh = (int)((lb << 1) >> 24) - (int)(ah >> 23) + 29;
  const uint32_t ml = (lb & 0x7FFFFFu) | 0x800000u;
  uint32_t t;
  // clamped shifts: amounts of 32 or more give 0
  asm("shl.b32 %0, %1, %2;" : "=r"(t) : "r"(ml), "r"((uint32_t)max(sh, 0)));
  asm("shr.b32 %0, %0, %1;" : "+r"(t) : "r"((uint32_t)max(-sh, 0)));
  const bool opposite = (int32_t)(hb ^ lb) < 0;
  if (opposite && (hb & 0x7FFFFFu) == 0u) t <<= 1;
  unsigned long long p = ((unsigned long long)hw << 32) | lw;
  p = opposite ? p - t : p + t;
  return __longlong_as_double((long long)p);
}
__device__ __forceinline__ dd fast_two_sum_dd(float a, float b) {
  const float s = __fadd_rn(a, b);
  return {s, __fsub_rn(b, __fsub_rn(s, a))};
}
// f + (h + l) with one FP64 addition: renormalise (|l| may exceed half a
// unit of h after unnormalised sums), assemble, add.
__device__ __forceinline__ double join1(double f, dd x) {
  return f + pair_to_f64(fast_two_sum_dd(x.h, x.l));
}

// c_k . (x, y, z) for k = 1..9 on pairs whose high parts lie on a common grid
// (exact high sums, rounded low sums).
__device__ __forceinline__ dd cdot_dd(int k, dd x, dd y, dd z) {
  switch (k) {
    case 1: return x;
    case 2: return y;
    case 3: return z;
    case 4: return {x.h + y.h, x.l + y.l};
    case 5: return {x.h - y.h, x.l - y.l};
    case 6: return {x.h + z.h, x.l + z.l};
    case 7: return {x.h - z.h, x.l - z.l};
    case 8: return {y.h + z.h, y.l + z.l};
    default: return {y.h - z.h, y.l - z.l};
  }
}

// ---------------------------------------------------------------- collision
// The TRT increment f*_i - f_i of one node, written per pair (k, k+9) as
//   -U = a s + G_c + (C4_c / rho) (c.j)^2,   -V = b (f_k - f_k+9) + C3_c (c.j) + S_k,
//   f*_k - f_k = -U - V,  f*_k+9 - f_k+9 = -U + V,
// with s = d_k + d_k+9, a = -w+/2, b = -w-/2 (the increment constants of
// Trt<df32>), G_c = w+ w_c (drho - 3/2 |j|^2 / rho), C4_c = 9/2 w+ w_c,
// C3_c = 3 w- w_c, S_k = 3 w_k (c_k . F), here computed as
// C3_c (c.j) + S_k = C3_c c.(j + F / w-); and for the rest direction
// -w+ d_0 + (w+ / 3)(drho - 3/2 |j|^2 / rho). This is collide<A, true> with the
// increment constants, term for term.
//
// Returns false, leaving f untouched, when the node is outside the path's
// range (see the top of the file). kJoin1 has bit i set for the directions
// whose increment is joined with one FP64 addition (join1), clear for two (join2).
// The grid collision's core: from the fixed-point deviations D_i = Dh:Dl
// (units of 2^-60) and the bound dabs on sum |D_i| (units of 2^-28), the
// increment f*_i - f_i of every direction as a pair, handed to join(i, x) as
// soon as it is known. a_inc = -w+/2, b_inc = -w-/2 and rest_inc = -w+ are the
// increment constants. Returns false, calling no join, if the deviations are too
// large for an exact grid.
template <typename P, typename Join>
__device__ __forceinline__ bool grid_increments(const uint32_t (&Dh)[19], const uint32_t (&Dl)[19], uint32_t dabs,
                                                const P& p, df32 a_inc, df32 b_inc, df32 rest_inc, Join&& join) {
  // The grid of the high parts: 2^-(28 + k) with the largest k <= 8 for which
  // every partial sum of high parts (edges count one pair twice; the folded
  // force adds 2 |F / w-|_1) stays below 2^24 grid units, i.e. is exact in FP32.
  const uint32_t t = 2u * (dabs + 20u) + p.fw_abs28;
  const int k = min(24 - (32 - __clz((int)t)), 8);
  if (k < 0 || dabs >= (1u << 24)) return false;
  const float hscale = __uint_as_float((uint32_t)(127 - 28 - k) << 23);   // 2^-(28 + k)
  const uint32_t lmask = 0xFFFFFFFFu >> k;                               // bits below the grid
  float H[19], L[19];
#pragma unroll
  for (int i = 0; i < 19; ++i) {
    // high part: D >> (32 - k), at most 23 bits by the choice of k, exact in FP32
    H[i] = (float)(int32_t)__funnelshift_rc(Dl[i], Dh[i], 32 - k) * hscale;
    // low part: the bits below the grid (non-negative), rounded to 24 bits
    L[i] = __uint2float_rn(Dl[i] & lmask) * 8.6736173798840355e-19f;   // 2^-60
  }

  // moments: H sums exact, L sums rounded
  float sH[10], sL[10], aH[10], aL[10];
#pragma unroll
  for (int k = 1; k <= 9; ++k) {
    sH[k] = H[k] + H[k + 9];
    sL[k] = L[k] + L[k + 9];
    aH[k] = H[k] - H[k + 9];
    aL[k] = L[k] - L[k + 9];
  }
  const dd drho = {H[0] + (((sH[1] + sH[2]) + (sH[3] + sH[4])) + ((sH[5] + sH[6]) + (sH[7] + sH[8])) + sH[9]),
                   L[0] + (((sL[1] + sL[2]) + (sL[3] + sL[4])) + ((sL[5] + sL[6]) + (sL[7] + sL[8])) + sL[9])};
  const dd jx = {(aH[1] + aH[4]) + (aH[5] + aH[6]) + aH[7], (aL[1] + aL[4]) + (aL[5] + aL[6]) + aL[7]};
  const dd jy = {(aH[2] + aH[4]) - aH[5] + (aH[8] + aH[9]), (aL[2] + aL[4]) - aL[5] + (aL[8] + aL[9])};
  const dd jz = {(aH[3] + aH[6]) - aH[7] + (aH[8] - aH[9]), (aL[3] + aL[6]) - aL[7] + (aL[8] - aL[9])};

  // 1 / rho: reciprocal of the high part, one correction from the residual
  const dd rho = add({1.0f, 0.0f}, drho);
  float r0;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r0) : "f"(rho.h));
  const float res = __fmaf_rn(-rho.l, r0, __fmaf_rn(-rho.h, r0, 1.0f));   // 1 - rho r0
  const dd rinv = {r0, r0 * res};
  const dd jsq = add(add(sqr(jx), sqr(jy)), sqr(jz));
  const dd base = add(drho, mul(df32(-1.5f), mul(rinv, jsq)));   // drho - 3/2 |j|^2 / rho
  dd G[2], R4[2];
  G[0] = mul(p.wp_w[0], base);
  G[1] = scale(G[0], 0.5f);           // w_edge = w_face / 2: the edge constants are exactly half
  R4[0] = mul(p.c4[0], rinv);
  R4[1] = scale(R4[0], 0.5f);
  const df32 c3[2] = {p.c3[0], p.c3[1]};
  // j + F / w-: the force source folded into the antisymmetric part, F / w-
  // split on the node's grid like the deviations (exact high parts)
  dd fwk[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const uint32_t fh = (uint32_t)((unsigned long long)p.fw60[a] >> 32), fl = (uint32_t)p.fw60[a];
    fwk[a] = {(float)(int32_t)__funnelshift_rc(fl, fh, 32 - k) * hscale,
              __uint2float_rn(fl & lmask) * 8.6736173798840355e-19f};
  }
  const dd gx = {jx.h + fwk[0].h, jx.l + fwk[0].l}, gy = {jy.h + fwk[1].h, jy.l + fwk[1].l},
           gz = {jz.h + fwk[2].h, jz.l + fwk[2].l};

  {
    join(0, add(mul(rest_inc, {H[0], L[0]}), mul(p.wp_w0, base)));
  }
#pragma unroll
  for (int k = 1; k <= 9; ++k) {
    const int c = k <= 3 ? 0 : 1;
    const dd cj = cdot_dd(k, jx, jy, jz), cg = cdot_dd(k, gx, gy, gz);
    const dd mU = add(add(mul(a_inc, {sH[k], sL[k]}), G[c]), mul(R4[c], sqr(cj)));
    const dd mV = add(mul(b_inc, {aH[k], aL[k]}), mul(c3[c], cg));
    join(k, add(mU, mV));
    join(k + 9, add(mU, neg(mV)));
  }
  return true;
}

template <uint32_t kJoin1, typename P>
__device__ __forceinline__ bool collide_grid(double (&f)[19], const P& p) {
  // Deviations in fixed point: D_i = (f_i - w_i) 2^60 as a 64-bit integer. For
  // f_i in [2^-8, 1) (FP64 exponent field 1015..1022) this is the 53-bit
  // significand shifted left by e - 1015 <= 7 bits, minus w_i 2^60 rounded:
  // exact up to that rounding (2^-61).
  uint32_t Dh[19], Dl[19];
  bool ok = true;
  uint32_t dabs = 0;   // sum |D_i| in units of 2^-28 (rounded down)
#pragma unroll
  for (int i = 0; i < 19; ++i) {
    const uint32_t hw = (uint32_t)__double2hiint(f[i]), lw = (uint32_t)__double2loint(f[i]);
    const uint32_t sh = (hw >> 20) - 1015u;
    ok &= sh < 8u;   // positive, exponent field 1015..1022
    const uint32_t mh = (hw & 0xFFFFFu) | 0x100000u;
    const uint32_t fh = __funnelshift_l(lw, mh, sh), fl = lw << sh;
    const int c = i == 0 ? 0 : (((i - 1) % 9) < 3 ? 1 : 2);
    const unsigned long long W = wfix(c);
    const unsigned long long Dv = (((unsigned long long)fh << 32) | fl) - W;
    Dh[i] = (uint32_t)(Dv >> 32);
    Dl[i] = (uint32_t)Dv;
    dabs += min((uint32_t)abs((int32_t)Dh[i]), 1u << 24);   // saturated: no overflow
  }
  if (!ok) return false;
  return grid_increments(Dh, Dl, dabs, p, p.a, p.b, p.rest, [&](int i, dd x) {
    f[i] = (kJoin1 >> i & 1u) ? join1(f[i], x) : join2(f[i], x);
  });
}

}  // namespace dfg
}  // namespace lbm
