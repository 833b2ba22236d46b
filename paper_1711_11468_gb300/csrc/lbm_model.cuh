// D3Q19 TRT model on the device: direction table, storage formats and the
// fused collision (Sec. 2 of Wittmann et al., arXiv 1711.11468: D3Q19, TRT,
// constant body force for verification).
//
// Direction order is the ABI's: 0 rest; k = 1..9 the "positive" directions
// (1,0,0) (0,1,0) (0,0,1) (1,1,0) (1,-1,0) (1,0,1) (1,0,-1) (0,1,1) (0,1,-1);
// k + 9 the opposite of k. The collision works on the nine opposite pairs,
// which is how TRT is defined (symmetric / antisymmetric parts per pair).
#pragma once

#include <cuda_fp16.h>
#include <cstdint>
#include <type_traits>

#include "lbm_df32.cuh"
#include "lbm_df64.cuh"
#include "lbm_sr.cuh"

namespace lbm {

constexpr int Q = 19;

// Velocity components by direction, written out per axis.
__host__ __device__ constexpr int cx(int i) {
  return (i == 1 || i == 4 || i == 5 || i == 6 || i == 7) ? 1
       : (i == 10 || i == 13 || i == 14 || i == 15 || i == 16) ? -1 : 0;
}
__host__ __device__ constexpr int cy(int i) {
  return (i == 2 || i == 4 || i == 8 || i == 9 || i == 14) ? 1
       : (i == 5 || i == 11 || i == 13 || i == 17 || i == 18) ? -1 : 0;
}
__host__ __device__ constexpr int cz(int i) {
  return (i == 3 || i == 6 || i == 8 || i == 16 || i == 18) ? 1
       : (i == 7 || i == 9 || i == 12 || i == 15 || i == 17) ? -1 : 0;
}
__host__ __device__ constexpr int opp(int i) { return i == 0 ? 0 : (i <= 9 ? i + 9 : i - 9); }
// 1/3 at rest, 1/18 on the faces (k = 1..3 and their opposites), 1/36 on the edges.
__host__ __device__ constexpr double weight(int i) {
  return i == 0 ? 1.0 / 3.0 : (((i - 1) % 9) < 3 ? 1.0 / 18.0 : 1.0 / 36.0);
}

// Compile-time checks of the table against the listed vectors and the pairing.
constexpr bool table_ok() {
  constexpr int v[10][3] = {{0, 0, 0}, {1, 0, 0}, {0, 1, 0}, {0, 0, 1}, {1, 1, 0},
                            {1, -1, 0}, {1, 0, 1}, {1, 0, -1}, {0, 1, 1}, {0, 1, -1}};
  for (int k = 0; k <= 9; ++k) {
    if (cx(k) != v[k][0] || cy(k) != v[k][1] || cz(k) != v[k][2]) return false;
    if (k > 0 && (cx(k + 9) != -v[k][0] || cy(k + 9) != -v[k][1] || cz(k + 9) != -v[k][2])) return false;
    if (k > 0 && (opp(opp(k)) != k || opp(k) != k + 9)) return false;
    const int c2 = v[k][0] * v[k][0] + v[k][1] * v[k][1] + v[k][2] * v[k][2];
    if (k > 0 && weight(k) != (c2 == 1 ? 1.0 / 18.0 : 1.0 / 36.0)) return false;
  }
  return true;
}
static_assert(table_ok(), "D3Q19 direction table does not match the ABI order");

enum Flag : uint8_t { kFluid = 0, kSolidFullway = 1, kSolidHalfway = 2 };

// TRT parameters in the arithmetic type A, folded for the pair update below:
//   a = (1 - w+)/2, b = (1 - w-)/2, wp_w[c] = w+ * w_c, c4[c] = 9/2 w+ w_c,
//   c3[c] = 3 w- w_c for the weight classes c = 0 (faces), 1 (edges),
//   fk[k-1] = 3 w_k (c_k . F) the body-force source of direction k (its
//   opposite gets -fk), rest = 1 - w+, wp_w0 = w+ / 3;
//   fw60[a] = F_a / w- times 2^60 rounded to an integer and fw_abs28 =
//   2 (|F_x| + |F_y| + |F_z|) / w- in units of 2^-28 (rounded up), used by the
//   grid double-float collision of FP64 storage (lbm_df64.cuh), which folds the
//   force source into the momentum: 3 w- w_c (c.j) + 3 w_c (c.F) =
//   c3[c] (c.(j + F / w-)), splitting F / w- on the node's grid like the PDFs.
template <typename A>
struct Trt {
  A a, b, rest, wp_w0;
  A wp_w[2], c4[2], c3[2];
  A fk[9];
  long long fw60[3];
  uint32_t fw_abs28;
};

// TRT parameters of the stochastically rounded FP16 format plus its random
// stream: the lattice's seed, the device word pair that numbers the sweeps
// (ctr[parity] holds this sweep's number t; the sweep writes t + 1 into
// ctr[parity ^ 1], which the next sweep, of the other parity, reads) and the
// per-sweep base seed + gamma (1 + (t << 32)), set on the device.
struct TrtSr : Trt<float> {
  unsigned long long seed;
  unsigned long long base;
  unsigned long long* ctr;
  int parity;
};

// 1/rho for the collision. In FP64 the IEEE division costs 5 FP64 fused
// multiply-adds on the pipe that bounds the FP64 sweep; here an FP32 reciprocal
// of rho's leading 24 bits (relative error below 2^-22) is refined by one Newton
// step in FP64, e = 1 - rho r0, r = r0 + r0 e, to a relative error of about 2^-44
// in 2 FP64 instructions (the conversions are integer bit operations). 1/rho only
// scales the quadratic terms of the equilibrium, (c.j)^2 / rho and |j|^2 / rho,
// whose magnitude is below 1e-3 for |u| <= 0.03, so this error stays below 1e-16
// absolute. Densities outside the normal FP32 range take the division.
template <typename A>
__device__ __forceinline__ A reciprocal(A rho) {
  return A(1.0f) / rho;
}
template <>
__device__ __forceinline__ double reciprocal<double>(double rho) {
  bool out_of_range = false;
  const float lead = split_f64_fast(rho, out_of_range).hi;
  if (out_of_range) return 1.0 / rho;
  const double r0 = f32_to_f64(__frcp_rn(lead));
  const double e = fma(-rho, r0, 1.0);
  return fma(r0, e, r0);
}

// x / 2 without the FP64 pipe, by one less in the exponent field: exact for
// normal x of magnitude at least 2^-1021, and x / 2 = x for zero, infinities and
// NaN; only the lowest normal binade and subnormals (below 4.5e-308) would come
// out wrong, and the collision never halves such values. No branch, so no FP64
// instruction is issued. The edge constants are half the face constants
// (w_edge = w_face / 2, so the host's w+ w_c and 9/2 w+ w_c are exactly halved
// too), which lets the FP64 collision derive the two edge products from the face
// products bit for bit.
__device__ __forceinline__ double half_exact(double x) {
  const int hi = __double2hiint(x);
  const unsigned e = ((unsigned)hi >> 20) & 0x7FFu;
  return __hiloint2double((e - 2u) < 0x7FDu ? hi - (1 << 20) : hi, __double2loint(x));
}

// ---------------------------------------------------------------- collision
// TRT collision plus body force on one node, in place on f[19].
//   rho = sum f_i, j = sum c_i f_i, u = j / rho,
//   e_i = w_i rho (1 + 3 c.u + 9/2 (c.u)^2 - 3/2 u.u),
//   per pair (k, k+9): f+ = (f_k + f_k+9)/2, f- = (f_k - f_k+9)/2 (same for e),
//   f*_k = f_k - w+ (f+ - e+) - w- (f- - e-) + 3 w_k c_k.F, f*_k+9 mirrored.
// Written per pair with s = f_k + f_k+9 and d = f_k - f_k+9 as
//   P = (1 - w+) s/2 + w+ e+,  M = (1 - w-) d/2 + w- e- + 3 w_k c_k.F,
//   f*_k = P + M,  f*_k+9 = P - M,
// with e+ = w (rho - 3/2 rho u.u) + 9/2 w (c.u)(c.j) and e- = 3 w (c.j): the same
// algebra, arranged so that each step is a fused multiply-add. The velocity
// itself is never formed: rho u.u = |j|^2 / rho and (c.u)(c.j) = (c.j)^2 / rho,
// so one reciprocal of rho scales the two quadratic terms (on the FP64 pipe,
// which bounds the FP64 sweep, 131 -> 124 instructions per fluid cell, ncu; 121
// with reciprocal<double> above, 119 with half_exact).
// With kShifted, f holds d_i = f_i - w_i: then rho = 1 + sum d_i, j = sum c_i d_i
// (sum c_i w_i = 0), and e_i - w_i = w_i (drho - 3/2 rho u.u + 3 c.j + 9/2 (c.u)(c.j)),
// the same pairwise algebra with rho replaced by drho in the constant term.
// With the increment constants (a - 1/2, b - 1/2, rest - 1) the same code
// returns f*_i - f_i instead of f*_i.
// With kScaled, f holds 2^14 d_i (the scaled stochastic FP16 format): the
// collision of scaled values is the same code with rho = 1 + 2^-14 rho0, the
// 3/2 of the u.u term and c4 divided by 2^14 and the force terms multiplied by
// 2^14 (the constants in p carry the latter two). Powers of two scale exactly,
// so this computes 2^14 times what the unscaled FP32 collision computes.
template <typename A, bool kShifted, bool kScaled = false>
__device__ __forceinline__ void collide(A (&f)[Q], const Trt<A>& p) {
  A s[10], d[10];
#pragma unroll
  for (int k = 1; k <= 9; ++k) {
    s[k] = f[k] + f[k + 9];
    d[k] = f[k] - f[k + 9];
  }
  const A rho0 = f[0] + (((s[1] + s[2]) + (s[3] + s[4])) + ((s[5] + s[6]) + (s[7] + s[8])) + s[9]);
  constexpr float kInvScale = 1.0f / (float)(1 << kSrScaleLog2);
  const A rho = kShifted ? (kScaled ? rho0 * A(kInvScale) + A(1.0f) : A(1.0f) + rho0) : rho0;
  const A jx = (d[1] + d[4]) + (d[5] + d[6]) + d[7];
  const A jy = (d[2] + d[4]) - d[5] + (d[8] + d[9]);
  const A jz = (d[3] + d[6]) - d[7] + (d[8] - d[9]);
  const A inv_rho = reciprocal<A>(rho);
  const A jsq = jx * jx + jy * jy + jz * jz;
  // constant part of e+ per unit weight: rho0 - 3/2 rho u.u = rho0 - 3/2 |j|^2 / rho
  const A base = rho0 - (A(kScaled ? 1.5f * kInvScale : 1.5f) * inv_rho) * jsq;
  A bw[2], c4r[2];   // w+ w_c base and 9/2 w+ w_c / rho for the faces (c = 0) and the edges
  bw[0] = p.wp_w[0] * base;
  c4r[0] = p.c4[0] * inv_rho;
  if constexpr (std::is_same<A, double>::value) {
    bw[1] = half_exact(bw[0]);
    c4r[1] = half_exact(c4r[0]);
  } else {
    bw[1] = p.wp_w[1] * base;
    c4r[1] = p.c4[1] * inv_rho;
  }

  f[0] = p.rest * f[0] + p.wp_w0 * base;

#pragma unroll
  for (int k = 1; k <= 9; ++k) {
    const int c = k <= 3 ? 0 : 1;
    const A cj = cdot<A>(k, jx, jy, jz);
    const A P = (c4r[c] * cj) * cj + (p.a * s[k] + bw[c]);
    const A M = p.b * d[k] + (p.c3[c] * cj + p.fk[k - 1]);
    f[k] = P + M;
    f[k + 9] = P - M;
  }
}

// ---------------------------------------------------------------- storage
// Each storage format defines the register type of a loaded PDF (Raw), the
// arithmetic type of the collision (A) and relax(), which turns the 19 loaded
// values of a node into its 19 post-collision values.
//   double : f_i in FP64, collided in FP64.
//   float  : d_i = f_i - w_i in FP32, collided in FP32.
//   __half : d_i = f_i - w_i in FP16, collided in FP32.
//   f64df  : f_i in FP64; the collision runs in double-float on the deviations
//            d_i = f_i - w_i and returns the increments f*_i - f_i, which are
//            added to the exact stored values in FP64.
//   f32df  : d_i = f_i - w_i in FP32, collided in double-float and rounded
//            once on store. FP32 collision arithmetic makes correlated
//            rounding errors that accumulate over steps; rounding a precisely
//            collided value only at the store does not.
//   h16sr  : 2^14 d_i in FP16, collided in FP32 (scaled), rounded to FP16
//            stochastically (lbm_sr.cuh) with the random bits of the node.
//            Raw values are the FP16 bit patterns, so that moving them (and
//            reversing them at full-way solids) needs no conversion.
// relax(f, p, node) is the entry point of the sweeps; node numbers the node's
// random stream and only h16sr uses it. unpack / pack convert between a stored
// element and its raw register value exactly as load / store do, for copies
// kept in shared memory.
// The shift keeps the collided magnitudes near the small departures that carry
// the flow instead of near w_i.
struct f64df {
  double v;
};
struct f32df {
  float v;
};
struct h16sr {
  __half v;
};

template <typename S>
struct Storage;

template <>
struct Storage<double> {
  using Params = Trt<double>;
  using Raw = double;
  using A = double;
  static constexpr bool kShifted = false, kIncrement = false;
  __device__ __forceinline__ static Raw load(const double* p) { return __ldcs(p); }
  __device__ __forceinline__ static void store(double* p, Raw v) { __stcs(p, v); }
  __device__ __forceinline__ static void relax(Raw (&f)[Q], const Params& p, uint32_t = 0) {
    collide<A, false>(f, p);
  }
  __device__ __forceinline__ static Raw unpack(double v) { return v; }
  __device__ __forceinline__ static double pack(Raw v) { return v; }
  __device__ __forceinline__ static double to_f64(double v, int) { return v; }
  __device__ __forceinline__ static double from_f64(double f, int) { return f; }
};

template <>
struct Storage<float> {
  using Params = Trt<float>;
  using Raw = float;
  using A = float;
  static constexpr bool kShifted = true, kIncrement = false;
  __device__ __forceinline__ static Raw load(const float* p) { return __ldcs(p); }
  __device__ __forceinline__ static void store(float* p, Raw v) { __stcs(p, v); }
  __device__ __forceinline__ static void relax(Raw (&f)[Q], const Params& p, uint32_t = 0) {
    collide<A, true>(f, p);
  }
  __device__ __forceinline__ static Raw unpack(float v) { return v; }
  __device__ __forceinline__ static float pack(Raw v) { return v; }
  __device__ __forceinline__ static double to_f64(float v, int i) { return weight(i) + (double)v; }
  __device__ __forceinline__ static float from_f64(double f, int i) { return __double2float_rn(f - weight(i)); }
};

template <>
struct Storage<__half> {
  using Params = Trt<float>;
  using Raw = float;
  using A = float;
  static constexpr bool kShifted = true, kIncrement = false;
  __device__ __forceinline__ static Raw load(const __half* p) {
    return __half2float(__ushort_as_half(__ldcs(reinterpret_cast<const unsigned short*>(p))));
  }
  __device__ __forceinline__ static void store(__half* p, Raw v) {
    __stcs(reinterpret_cast<unsigned short*>(p), __half_as_ushort(__float2half_rn(v)));
  }
  __device__ __forceinline__ static void relax(Raw (&f)[Q], const Params& p, uint32_t = 0) {
    collide<A, true>(f, p);
  }
  __device__ __forceinline__ static Raw unpack(__half v) { return __half2float(v); }
  __device__ __forceinline__ static __half pack(Raw v) { return __float2half_rn(v); }
  __device__ __forceinline__ static double to_f64(__half v, int i) { return weight(i) + (double)__half2float(v); }
  __device__ __forceinline__ static __half from_f64(double f, int i) {
    // FP64 -> FP16 in one rounding (a detour through FP32 could double-round).
    return __double2half(f - weight(i));
  }
};

#ifndef LBM_F64DF_JOIN1
#define LBM_F64DF_JOIN1 0x7FE7Eu
#endif

template <>
struct Storage<f64df> {
  using Params = Trt<df32>;
  using Raw = double;
  using A = df32;
  static constexpr bool kShifted = true, kIncrement = true;
  __device__ __forceinline__ static Raw load(const f64df* p) { return __ldcs(reinterpret_cast<const double*>(p)); }
  __device__ __forceinline__ static void store(f64df* p, Raw v) { __stcs(reinterpret_cast<double*>(p), v); }
  // Directions whose increment is joined with one FP64 addition (the rest with
  // two): balances the FP64 pipe against integer instructions.
  static constexpr uint32_t kJoin1 = LBM_F64DF_JOIN1;
  __device__ __forceinline__ static void relax(Raw (&f)[Q], const Params& p, uint32_t = 0) {
    if (dfg::collide_grid<kJoin1>(f, p)) return;   // nodes near equilibrium (lbm_df64.cuh)
    df32 d[Q];
    bool out_of_range = false;
#pragma unroll
    for (int i = 0; i < Q; ++i) d[i] = split_f64_fast(f[i], out_of_range) - df32(weight(i));
    if (out_of_range) {   // a zero or extreme PDF somewhere in the node: convert all 19 exactly
#pragma unroll
      for (int i = 0; i < Q; ++i) d[i] = split_f64_slow(f[i]) - df32(weight(i));
    }
    collide<A, true>(d, p);
#pragma unroll
    for (int i = 0; i < Q; ++i) f[i] = (f[i] + f32_to_f64(d[i].hi)) + f32_to_f64(d[i].lo);
  }
  __device__ __forceinline__ static Raw unpack(f64df v) { return v.v; }
  __device__ __forceinline__ static f64df pack(Raw v) { return f64df{v}; }
  __device__ __forceinline__ static double to_f64(f64df v, int) { return v.v; }
  __device__ __forceinline__ static f64df from_f64(double f, int) { return f64df{f}; }
};

template <>
struct Storage<f32df> {
  using Params = Trt<df32>;
  using Raw = float;
  using A = df32;
  static constexpr bool kShifted = true, kIncrement = false;
  __device__ __forceinline__ static Raw load(const f32df* p) { return __ldcs(reinterpret_cast<const float*>(p)); }
  __device__ __forceinline__ static void store(f32df* p, Raw v) { __stcs(reinterpret_cast<float*>(p), v); }
  __device__ __forceinline__ static void relax(Raw (&f)[Q], const Params& p, uint32_t = 0) {
    df32 d[Q];
#pragma unroll
    for (int i = 0; i < Q; ++i) d[i] = df32(f[i]);
    collide<A, true>(d, p);
#pragma unroll
    for (int i = 0; i < Q; ++i) f[i] = __fadd_rn(d[i].hi, d[i].lo);
  }
  __device__ __forceinline__ static Raw unpack(f32df v) { return v.v; }
  __device__ __forceinline__ static f32df pack(Raw v) { return f32df{v}; }
  __device__ __forceinline__ static double to_f64(f32df v, int i) { return weight(i) + (double)v.v; }
  __device__ __forceinline__ static f32df from_f64(double f, int i) { return f32df{__double2float_rn(f - weight(i))}; }
};

template <>
struct Storage<h16sr> {
  using Raw = uint32_t;   // the FP16 bit pattern in the low half; the high half is ignored
  using A = float;
  using Params = TrtSr;
  static constexpr bool kShifted = true, kIncrement = false;
  __device__ __forceinline__ static Raw load(const h16sr* p) {
    return __ldcs(reinterpret_cast<const unsigned short*>(p));
  }
  __device__ __forceinline__ static void store(h16sr* p, Raw v) {
    __stcs(reinterpret_cast<unsigned short*>(p), (unsigned short)v);
  }
  __device__ __forceinline__ static void relax(Raw (&f)[Q], const Params& p, uint32_t node) {
    float d[Q];
#pragma unroll
    for (int i = 0; i < Q; ++i) d[i] = __half2float(__ushort_as_half((unsigned short)f[i]));
    collide<float, true, true>(d, p);
    unsigned long long w[5];
    sr_words(p.base, node, w);
    // The one-addition form is exact when every value is at least 2^-14 in
    // magnitude (or 0); the general form is exact for all and gives the same
    // bits wherever the first one is exact. The choice is made per warp (a
    // vote), so that it is a uniform branch: a warp takes the general form only
    // if one of its nodes has a value below 2^-14 (zeros included, which only
    // the rest state has), which is rare in a flow.
    float small = fabsf(d[0]);
#pragma unroll
    for (int i = 1; i < Q; ++i) small = fminf(small, fabsf(d[i]));
    if (!__any_sync(__activemask(), small < kSrNormalMin)) {
#pragma unroll
      for (int i = 0; i < Q; ++i) f[i] = round_half_stochastic_normal(d[i], sr_bits(w, i));
    } else {
#pragma unroll
      for (int i = 0; i < Q; ++i) f[i] = round_half_stochastic_any(d[i], sr_bits(w, i));
    }
  }
  __device__ __forceinline__ static Raw unpack(h16sr v) { return __half_as_ushort(v.v); }
  __device__ __forceinline__ static h16sr pack(Raw v) { return h16sr{__ushort_as_half((unsigned short)v)}; }
  __device__ __forceinline__ static double to_f64(h16sr v, int i) {
    return weight(i) + ldexp((double)__half2float(v.v), -kSrScaleLog2);
  }
  __device__ __forceinline__ static h16sr from_f64(double f, int i) {
    return h16sr{__double2half(ldexp(f - weight(i), kSrScaleLog2))};
  }
};

// Per-sweep set-up of the launch parameters. Every thread of the launch calls
// it first; for the stochastic format it reads the sweep number and the launch's
// first thread advances the counter of the other parity.
template <typename S>
__device__ __forceinline__ typename Storage<S>::Params begin_sweep(const typename Storage<S>::Params& p) {
  return p;
}
template <>
__device__ __forceinline__ TrtSr begin_sweep<h16sr>(const TrtSr& p) {
  TrtSr q = p;
  const unsigned long long t = p.ctr[p.parity];
  if (blockIdx.x == 0 && blockIdx.y == 0 && threadIdx.x == 0) p.ctr[p.parity ^ 1] = t + 1;
  q.base = p.seed + kSplitmixGamma * (1ull + (t << 32));
  return q;
}

// The same for a launch that performs two sweeps (temporal blocking): pa for
// sweep t, pb for sweep t + 1; the counter of the other parity receives t + 2.
template <typename S>
__device__ __forceinline__ void begin_two_sweeps(const typename Storage<S>::Params& p, typename Storage<S>::Params& pa,
                                                 typename Storage<S>::Params& pb) {
  pa = p;
  pb = p;
}
template <>
__device__ __forceinline__ void begin_two_sweeps<h16sr>(const TrtSr& p, TrtSr& pa, TrtSr& pb) {
  pa = p;
  pb = p;
  const unsigned long long t = p.ctr[p.parity];
  if (blockIdx.x == 0 && blockIdx.y == 0 && blockIdx.z == 0 && threadIdx.x == 0 && threadIdx.y == 0)
    p.ctr[p.parity ^ 1] = t + 2;
  pa.base = p.seed + kSplitmixGamma * (1ull + (t << 32));
  pb.base = p.seed + kSplitmixGamma * (1ull + ((t + 1) << 32));
}

// The 19 FP64 equilibria of one cell (initialisation), by opposite pairs: f_k
// and f_k+9 (c_k+9 = -c_k) share w rho (1 - 3/2 |u|^2 + 9/2 (c.u)^2) and
// differ in the sign of 3 w rho (c.u), so a pair costs about as much as one
// direction of the per-direction form below.
__device__ __forceinline__ void equilibria_f64(double rho, double ux, double uy, double uz, double (&feq)[19]) {
  const double base = rho * fma(-1.5, fma(ux, ux, fma(uy, uy, uz * uz)), 1.0);
  feq[0] = (1.0 / 3.0) * base;
#pragma unroll
  for (int k = 1; k <= 9; ++k) {
    const int a = cx(k), b = cy(k), c = cz(k);
    const double tx = a > 0 ? ux : -ux, ty = b > 0 ? uy : -uy, tz = c > 0 ? uz : -uz;
    // c_k.u as the signed sum of the components c_k selects: the dot product's
    // value (products by +-1 and 0 are exact) without the multiplications by 0
    // and additions of 0 that the compiler must keep (signed zeros)
    double cu = 0.0;
    if (a != 0 && b != 0) cu = tx + ty;
    else if (a != 0 && c != 0) cu = tx + tz;
    else if (b != 0 && c != 0) cu = ty + tz;
    else if (a != 0) cu = tx;
    else if (b != 0) cu = ty;
    else cu = tz;
    const double w = weight(k);
    const double t = rho * cu;
    const double sym = w * fma(4.5 * t, cu, base);
    const double anti = (3.0 * w) * t;
    feq[k] = sym + anti;
    feq[k + 9] = sym - anti;
  }
}

}  // namespace lbm
