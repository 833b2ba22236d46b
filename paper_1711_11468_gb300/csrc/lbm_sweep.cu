// Single-lattice sweep kernels: one thread per cell of the full array (rows of
// x on a 2-D grid) or per node of the fluid list. The per-node bodies live in
// lbm_sweep.cuh and are shared with the batched kernel.
#include <cmath>
#include <mutex>
#include <type_traits>

#include "lbm_async.cuh"
#include "lbm_internal.h"
#include "lbm_sweep.cuh"

namespace lbm {

template <typename S>
Trt<Arith<S>> trt_as(const TrtParams& p) {
  using A = Arith<S>;
  Trt<A> t;
  const double w[2] = {1.0 / 18.0, 1.0 / 36.0};
  t.a = (A)((1.0 - p.omega_p) * 0.5);
  t.b = (A)((1.0 - p.omega_m) * 0.5);
  t.rest = (A)(1.0 - p.omega_p);
  t.wp_w0 = (A)(p.omega_p / 3.0);
  for (int c = 0; c < 2; ++c) {
    t.wp_w[c] = (A)(p.omega_p * w[c]);
    t.c4[c] = (A)(4.5 * p.omega_p * w[c]);
    t.c3[c] = (A)(3.0 * p.omega_m * w[c]);
  }
  // w[1] = w[0] / 2 exactly, so the edge constants are exactly half the face
  // constants; the FP64 collision relies on it (half_exact)
  for (int k = 0; k < 9; ++k) t.fk[k] = (A)p.fk[k];
  // F / w- in fixed point for the grid collision of FP64 storage; a force too
  // large for it (|F / w-| >= 2^-5) gets a budget that keeps that path off
  double fw_abs = 0.0;
  for (int a = 0; a < 3; ++a) {
    const double fw = p.force[a] / p.omega_m;
    fw_abs += 2.0 * std::fabs(fw);
    t.fw60[a] = std::fabs(fw) < 0.03125 ? std::llround(fw * 1152921504606846976.0) : 0;   // 2^60
  }
  t.fw_abs28 = fw_abs < 0.0625 ? (uint32_t)std::ceil(fw_abs * 268435456.0) : (1u << 30);   // 2^28
  if (Storage<S>::kIncrement) {
    // return f*_i - f_i: the rest direction and the pair terms lose the f_i itself
    t.a = (A)((1.0 - p.omega_p) * 0.5 - 0.5);
    t.b = (A)((1.0 - p.omega_m) * 0.5 - 0.5);
    t.rest = (A)(-p.omega_p);
  }
  return t;
}
template Trt<double> trt_as<double>(const TrtParams&);
template Trt<float> trt_as<float>(const TrtParams&);
template Trt<float> trt_as<__half>(const TrtParams&);
template Trt<df32> trt_as<f64df>(const TrtParams&);
template Trt<df32> trt_as<f32df>(const TrtParams&);
template Trt<float> trt_as<h16sr>(const TrtParams&);

namespace {

// ------------------------------------------------------------- full array
// Grid: blockIdx.x = row (y + ny*z), blockIdx.y * blockDim.x + threadIdx.x = x.
template <typename S, bool kHW>
__global__ void __launch_bounds__(512) k_dense_pull(const S* __restrict__ src, S* __restrict__ dst,
                                                    const uint8_t* __restrict__ flags, int nx, int ny, int nz,
                                                    int64_t stride, ParamsT<S> lp) {
  const ParamsT<S> p = begin_sweep<S>(lp);
  const int x = blockIdx.y * blockDim.x + threadIdx.x;
  if (x >= nx) return;
  const int row = blockIdx.x;
  const int z = row / ny, y = row - z * ny;
  pull_dense_node<S, kHW>(src, dst, flags, x, y, z, x + nx * row, nx, ny, nz, stride, p);
}

template <typename S>
__global__ void __launch_bounds__(512) k_dense_aa_even(S* __restrict__ pdf, const uint8_t* __restrict__ flags,
                                                       int nx, int64_t stride, ParamsT<S> lp) {
  const ParamsT<S> p = begin_sweep<S>(lp);
  const int x = blockIdx.y * blockDim.x + threadIdx.x;
  if (x >= nx) return;
  const int n = x + nx * (int)blockIdx.x;
  if (flags[n] != kFluid) return;
  aa_even_node<S>(pdf, n, stride, p);
}

template <typename S, bool kHW>
__global__ void __launch_bounds__(512) k_dense_aa_odd(S* __restrict__ pdf, const uint8_t* __restrict__ flags,
                                                      int nx, int ny, int nz, int64_t stride, ParamsT<S> lp) {
  const ParamsT<S> p = begin_sweep<S>(lp);
  const int x = blockIdx.y * blockDim.x + threadIdx.x;
  if (x >= nx) return;
  const int row = blockIdx.x;
  const int z = row / ny, y = row - z * ny;
  const int n = x + nx * row;
  if (flags[n] != kFluid) return;
  aa_odd_dense_node<S, kHW>(pdf, flags, x, y, z, n, nx, ny, nz, stride, p);
}

// Two cells per thread: x and x + blockDim.x of the same row (grid.y covers
// x-blocks of 2 * blockDim.x).
template <typename S, bool kHW>
__global__ void __launch_bounds__(512) k_dense_pull2(const S* __restrict__ src, S* __restrict__ dst,
                                                     const uint8_t* __restrict__ flags, int nx, int ny, int nz,
                                                     int64_t stride, ParamsT<S> lp) {
  const ParamsT<S> p = begin_sweep<S>(lp);
  const int xa = blockIdx.y * 2 * blockDim.x + threadIdx.x, xb = xa + blockDim.x;
  if (xa >= nx) return;
  const int row = blockIdx.x;
  const int z = row / ny, y = row - z * ny;
  const int na = xa + nx * row, nb_ = xb + nx * row;
  const bool hb = xb < nx;
  const uint8_t fa = flags[na], fb = hb ? flags[nb_] : (uint8_t)kSolidHalfway;
  RawT<S> f[Q], g[Q];
  if (fa != kSolidHalfway) pull_dense_gather<S, kHW>(src, flags, Nbr(xa, y, z, nx, ny, nz), na, stride, f);
  if (fb != kSolidHalfway) pull_dense_gather<S, kHW>(src, flags, Nbr(xb, y, z, nx, ny, nz), nb_, stride, g);
  if (fa != kSolidHalfway) {
    if (fa == kSolidFullway) reverse(f); else Storage<S>::relax(f, p, (uint32_t)na);
#pragma unroll
    for (int i = 0; i < Q; ++i) Storage<S>::store(dir(dst, i, stride) + na, f[i]);
  }
  if (fb != kSolidHalfway) {
    if (fb == kSolidFullway) reverse(g); else Storage<S>::relax(g, p, (uint32_t)nb_);
#pragma unroll
    for (int i = 0; i < Q; ++i) Storage<S>::store(dir(dst, i, stride) + nb_, g[i]);
  }
}

template <typename S>
__global__ void __launch_bounds__(512) k_dense_aa_even2(S* __restrict__ pdf, const uint8_t* __restrict__ flags,
                                                        int nx, int64_t stride, ParamsT<S> lp) {
  const ParamsT<S> p = begin_sweep<S>(lp);
  const int xa = blockIdx.y * 2 * blockDim.x + threadIdx.x, xb = xa + blockDim.x;
  if (xa >= nx) return;
  const int na = xa + nx * (int)blockIdx.x, nb_ = xb + nx * (int)blockIdx.x;
  const bool ua = flags[na] == kFluid, ub = xb < nx && flags[nb_] == kFluid;
  RawT<S> f[Q], g[Q];
  if (ua)
#pragma unroll
    for (int i = 0; i < Q; ++i) f[i] = Storage<S>::load(dir(pdf, i, stride) + na);
  if (ub)
#pragma unroll
    for (int i = 0; i < Q; ++i) g[i] = Storage<S>::load(dir(pdf, i, stride) + nb_);
  if (ua) {
    Storage<S>::relax(f, p, (uint32_t)na);
#pragma unroll
    for (int i = 0; i < Q; ++i) Storage<S>::store(dir(pdf, opp(i), stride) + na, f[i]);
  }
  if (ub) {
    Storage<S>::relax(g, p, (uint32_t)nb_);
#pragma unroll
    for (int i = 0; i < Q; ++i) Storage<S>::store(dir(pdf, opp(i), stride) + nb_, g[i]);
  }
}

template <typename S, bool kHW>
__global__ void __launch_bounds__(512) k_dense_aa_odd2(S* __restrict__ pdf, const uint8_t* __restrict__ flags,
                                                       int nx, int ny, int nz, int64_t stride, ParamsT<S> lp) {
  const ParamsT<S> p = begin_sweep<S>(lp);
  const int xa = blockIdx.y * 2 * blockDim.x + threadIdx.x, xb = xa + blockDim.x;
  if (xa >= nx) return;
  const int row = blockIdx.x;
  const int z = row / ny, y = row - z * ny;
  const int na = xa + nx * row, nb_ = xb + nx * row;
  const bool ua = flags[na] == kFluid, ub = xb < nx && flags[nb_] == kFluid;
  const Nbr ba(xa, y, z, nx, ny, nz), bb(xb < nx ? xb : xa, y, z, nx, ny, nz);
  RawT<S> f[Q], g[Q];
  if (ua) aa_odd_dense_gather<S, kHW>(pdf, flags, ba, na, stride, f);
  if (ub) aa_odd_dense_gather<S, kHW>(pdf, flags, bb, nb_, stride, g);
  if (ua) {
    Storage<S>::relax(f, p, (uint32_t)na);
    aa_odd_dense_scatter<S, kHW>(pdf, flags, ba, na, stride, f);
  }
  if (ub) {
    Storage<S>::relax(g, p, (uint32_t)nb_);
    aa_odd_dense_scatter<S, kHW>(pdf, flags, bb, nb_, stride, g);
  }
}

// Even AA step on two adjacent cells (x, x+1) per thread, x even, moving both
// cells of a direction with one vector access (2 x FP16 in 4 bytes, 2 x FP32
// in 8). Half the memory requests of the scalar kernel. Needs nx even, so that
// every pair starts on an even element. A solid cell of a pair is reversed
// instead of collided, which makes its swapped store leave it unchanged.
template <typename S>
struct PairIO;
template <>
struct PairIO<__half> {
  __device__ __forceinline__ static void load(const __half* p, float& a, float& b) {
    const unsigned u = __ldcs(reinterpret_cast<const unsigned*>(p));
    a = __half2float(__ushort_as_half((unsigned short)(u & 0xFFFFu)));
    b = __half2float(__ushort_as_half((unsigned short)(u >> 16)));
  }
  __device__ __forceinline__ static void store(__half* p, float a, float b) {
    const unsigned u = (unsigned)__half_as_ushort(__float2half_rn(a)) |
                       ((unsigned)__half_as_ushort(__float2half_rn(b)) << 16);
    __stcs(reinterpret_cast<unsigned*>(p), u);
  }
};
template <>
struct PairIO<float> {
  __device__ __forceinline__ static void load(const float* p, float& a, float& b) {
    const float2 v = __ldcs(reinterpret_cast<const float2*>(p));
    a = v.x;
    b = v.y;
  }
  __device__ __forceinline__ static void store(float* p, float a, float b) {
    __stcs(reinterpret_cast<float2*>(p), make_float2(a, b));
  }
};
template <>
struct PairIO<h16sr> {   // raw values are the bit patterns in the low halves: no conversion, no masking
  __device__ __forceinline__ static void load(const h16sr* p, uint32_t& a, uint32_t& b) {
    const unsigned u = __ldcs(reinterpret_cast<const unsigned*>(p));
    a = u;
    b = u >> 16;
  }
  __device__ __forceinline__ static void store(h16sr* p, uint32_t a, uint32_t b) {
    __stcs(reinterpret_cast<unsigned*>(p), __byte_perm(a, b, 0x5410u));
  }
};
template <>
struct PairIO<f32df> {
  __device__ __forceinline__ static void load(const f32df* p, float& a, float& b) {
    PairIO<float>::load(reinterpret_cast<const float*>(p), a, b);
  }
  __device__ __forceinline__ static void store(f32df* p, float a, float b) {
    PairIO<float>::store(reinterpret_cast<float*>(p), a, b);
  }
};

template <typename S>
__global__ void __launch_bounds__(512) k_dense_aa_even_pair(S* __restrict__ pdf, const uint8_t* __restrict__ flags,
                                                            int nx, int64_t stride, ParamsT<S> lp) {
  const ParamsT<S> p = begin_sweep<S>(lp);
  const int x = 2 * (blockIdx.y * blockDim.x + threadIdx.x);
  if (x >= nx) return;
  const int n = x + nx * (int)blockIdx.x;
  const bool ua = flags[n] == kFluid, ub = flags[n + 1] == kFluid;
  if (!ua && !ub) return;
  RawT<S> f[Q], g[Q];
#pragma unroll
  for (int i = 0; i < Q; ++i) PairIO<S>::load(dir(pdf, i, stride) + n, f[i], g[i]);
  if (ua) Storage<S>::relax(f, p, (uint32_t)n); else reverse(f);
  if (ub) Storage<S>::relax(g, p, (uint32_t)(n + 1)); else reverse(g);
#pragma unroll
  for (int i = 0; i < Q; ++i) PairIO<S>::store(dir(pdf, opp(i), stride) + n, f[i], g[i]);
}

// Odd AA step and pull on the same (x, x+1) pairs: the 9 directions without an
// x component read and write both cells' slots with one vector access (the y and
// z offsets are multiples of nx, so the pair stays aligned); the 10 directions
// with one are two scalar accesses. A pair with a solid cell falls back to the
// per-cell bodies. Full arrays without half-way solids only.
template <typename S>
__global__ void __launch_bounds__(512) k_dense_aa_odd_pair(S* __restrict__ pdf, const uint8_t* __restrict__ flags,
                                                           int nx, int ny, int nz, int64_t stride, ParamsT<S> lp) {
  const ParamsT<S> p = begin_sweep<S>(lp);
  const int x = 2 * (blockIdx.y * blockDim.x + threadIdx.x);
  if (x >= nx) return;
  const int row = blockIdx.x;
  const int z = row / ny, y = row - z * ny;
  int n = x + nx * row;
  const bool ua = flags[n] == kFluid, ub = flags[n + 1] == kFluid;
  if (!ua && !ub) return;
  Nbr na(x, y, z, nx, ny, nz), nb(x + 1, y, z, nx, ny, nz);
  RawT<S> f[Q], g[Q];
  if (!(ua && ub)) {
    if (ua) {
      aa_odd_dense_gather<S, false>(pdf, flags, na, n, stride, f);
      Storage<S>::relax(f, p, (uint32_t)n);
      aa_odd_dense_scatter<S, false>(pdf, flags, na, n, stride, f);
    }
    if (ub) {
      aa_odd_dense_gather<S, false>(pdf, flags, nb, n + 1, stride, g);
      Storage<S>::relax(g, p, (uint32_t)(n + 1));
      aa_odd_dense_scatter<S, false>(pdf, flags, nb, n + 1, stride, g);
    }
    return;
  }
#pragma unroll
  for (int i = 0; i < Q; ++i) {
    if (cx(i) == 0) {
      PairIO<S>::load(dir(pdf, opp(i), stride) + n + na.up(i), f[i], g[i]);
    } else {
      f[i] = Storage<S>::load(dir(pdf, opp(i), stride) + n + na.up(i));
      g[i] = Storage<S>::load(dir(pdf, opp(i), stride) + n + 1 + nb.up(i));
    }
  }
  Storage<S>::relax(f, p, (uint32_t)n);
  Storage<S>::relax(g, p, (uint32_t)(n + 1));
  opaque<S, false>(na, n);
  opaque<S, false>(nb, n);
#pragma unroll
  for (int i = 0; i < Q; ++i) {
    if (cx(i) == 0) {
      PairIO<S>::store(dir(pdf, i, stride) + n + na.down(i), f[i], g[i]);
    } else {
      Storage<S>::store(dir(pdf, i, stride) + n + na.down(i), f[i]);
      Storage<S>::store(dir(pdf, i, stride) + n + 1 + nb.down(i), g[i]);
    }
  }
}

template <typename S>
__global__ void __launch_bounds__(512) k_dense_pull_pair(const S* __restrict__ src, S* __restrict__ dst,
                                                         const uint8_t* __restrict__ flags, int nx, int ny, int nz,
                                                         int64_t stride, ParamsT<S> lp) {
  const ParamsT<S> p = begin_sweep<S>(lp);
  const int x = 2 * (blockIdx.y * blockDim.x + threadIdx.x);
  if (x >= nx) return;
  const int row = blockIdx.x;
  const int z = row / ny, y = row - z * ny;
  const int n = x + nx * row;
  const uint8_t fa = flags[n], fb = flags[n + 1];
  const Nbr na(x, y, z, nx, ny, nz), nb(x + 1, y, z, nx, ny, nz);
  RawT<S> f[Q], g[Q];
#pragma unroll
  for (int i = 0; i < Q; ++i) {
    if (cx(i) == 0) {
      PairIO<S>::load(dir(src, i, stride) + n + na.up(i), f[i], g[i]);
    } else {
      f[i] = Storage<S>::load(dir(src, i, stride) + n + na.up(i));
      g[i] = Storage<S>::load(dir(src, i, stride) + n + 1 + nb.up(i));
    }
  }
  // full arrays without half-way solids: every cell holds PDFs (fluid collides, solid reverses)
  if (fa == kSolidFullway) reverse(f); else Storage<S>::relax(f, p, (uint32_t)n);
  if (fb == kSolidFullway) reverse(g); else Storage<S>::relax(g, p, (uint32_t)(n + 1));
#pragma unroll
  for (int i = 0; i < Q; ++i) PairIO<S>::store(dir(dst, i, stride) + n, f[i], g[i]);
}

template <typename S>
constexpr bool kHasPairIO = std::is_same<S, __half>::value || std::is_same<S, float>::value ||
                            std::is_same<S, f32df>::value || std::is_same<S, h16sr>::value;

// ------------------------------------------------------------ fluid list
template <typename S>
__global__ void __launch_bounds__(512) k_list_pull(const S* __restrict__ src, S* __restrict__ dst,
                                                   const uint32_t* __restrict__ link, int64_t nf, int64_t stride,
                                                   ParamsT<S> lp) {
  const ParamsT<S> p = begin_sweep<S>(lp);
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= nf) return;
  pull_list_node<S>(src, dst, link, k, stride, p);
}

template <typename S>
__global__ void __launch_bounds__(512) k_list_aa_even(S* __restrict__ pdf, int64_t nf, int64_t stride,
                                                      ParamsT<S> lp) {
  const ParamsT<S> p = begin_sweep<S>(lp);
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= nf) return;
  aa_even_node<S>(pdf, k, stride, p);
}

template <typename S>
__global__ void __launch_bounds__(512) k_list_aa_odd(S* __restrict__ pdf, const uint32_t* __restrict__ link,
                                                     int64_t nf, int64_t stride, ParamsT<S> lp) {
  const ParamsT<S> p = begin_sweep<S>(lp);
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= nf) return;
  aa_odd_list_node<S>(pdf, link, k, stride, p);
}

// Fluid-list sweeps with the links staged in shared memory. A persistent grid
// strides over tiles of T = blockDim.x nodes; while a CTA works on one tile,
// one elected thread has the next tile's 18 link rows already on their way
// into the other shared-memory buffer by bulk copy. The gathers then depend on
// a shared-memory read instead of a global load, and the 18 offsets need no
// registers between the gather and the scatter. The odd AA step works in place
// on dst; its callers pass no src.
constexpr int kStagedMaxThreads = 512;
constexpr size_t staged_smem_bytes(int threads) { return (size_t)2 * 18 * threads * sizeof(uint32_t); }

template <typename S, int KIND>
__global__ void __launch_bounds__(kStagedMaxThreads) k_list_staged(const S* __restrict__ src, S* __restrict__ dst,
                                                                   const uint32_t* __restrict__ link, int64_t nf,
                                                                   int64_t stride, ParamsT<S> lp, int* status) {
  const ParamsT<S> p = begin_sweep<S>(lp);
  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ uint64_t bar[2];
  __shared__ int abort_flag;
  const int T = blockDim.x;
  const int j = threadIdx.x;
  // buffer b at buf0 + b * 18 T (no arrays indexed by b: they would live in local memory)
  uint32_t* const buf0 = reinterpret_cast<uint32_t*>(smem);
  const int64_t ntiles = (nf + T - 1) / T;
  if (j == 0) {
    mbar_init(&bar[0], 1);
    mbar_init(&bar[1], 1);
    fence_mbar_init();
    abort_flag = 0;
  }
  __syncthreads();
  // rows of `count` int32 rounded up to 16 bytes: stays inside the padded stride
  auto issue = [&](int64_t tile, int b) {
    const int64_t first = tile * T;
    const int64_t count = nf - first < T ? nf - first : T;
    const uint32_t row = (uint32_t)((count * 4 + 15) & ~(int64_t)15);
    uint32_t* buf = buf0 + b * 18 * T;
    mbar_arrive_expect_tx(&bar[b], 18u * row);
    for (int i = 0; i < 18; ++i) bulk_copy_g2s(buf + i * T, link + (int64_t)i * stride + first, row, &bar[b]);
  };
  int64_t t = blockIdx.x;
  if (j == 0 && t < ntiles) issue(t, 0);
  // pass `it` uses buffer it & 1 in its ((it >> 1) + 1)-th fill: phase parity (it >> 1) & 1
  for (int it = 0; t < ntiles; t += gridDim.x, ++it) {
    const int b = it & 1;
    const int64_t tn = t + gridDim.x;
    if (j == 0 && tn < ntiles) {
      fence_proxy_async_smem();   // the reads of buffer b^1 (previous tile) are ordered before its refill
      issue(tn, b ^ 1);
    }
    if (!mbar_wait_bounded(&bar[b], (uint32_t)(it >> 1) & 1u)) {
      atomicOr(status, kStatusWaitTimeout);
      abort_flag = 1;
    } else {
      const int64_t k = t * T + j;
      if (k < nf) {
        if (KIND == kPull)
          pull_list_node_staged<S>(src, dst, buf0 + b * 18 * T, T, j, k, stride, p);
        else
          aa_odd_list_node_staged<S>(dst, buf0 + b * 18 * T, T, j, k, p);
      }
    }
    __syncthreads();
    if (abort_flag) {
      // never leave a copy in flight into shared memory that is about to be
      // released: this tile's and, when issued, the next one's
      if (j == 0) {
        mbar_wait_bounded(&bar[b], (uint32_t)(it >> 1) & 1u);
        if (tn < ntiles) mbar_wait_bounded(&bar[b ^ 1], (uint32_t)((it + 1) >> 1) & 1u);
      }
      return;
    }
  }
}

// One node of a run-indexed list sweep: lane `lane` of a 32-node chunk decodes
// its 18 links from the chunk's headers `hd` and pool slice `pl` (pool index
// `pb` at pl[0]; le = the mask of lanes 0..lane), then gathers, collides and
// stores (pull: into dst's own slots; odd AA step: scattered in place).
template <typename S, int KIND>
__device__ __forceinline__ void ria_node(const S* __restrict__ src, S* __restrict__ dst, const uint2* hd,
                                         const uint32_t* pl, uint32_t pb, unsigned le, int lane, int64_t k,
                                         int64_t stride, const ParamsT<S>& p) {
  uint32_t off[Q];
#pragma unroll
  for (int i = 1; i < Q; ++i) {
    const uint2 h = hd[i - 1];
    const unsigned below = h.x & le;
    off[i] = pl[h.y - pb + (uint32_t)__popc(below) - 1u] + (uint32_t)(lane - 31 + __clz(below));
  }
  RawT<S> f[Q];
  if (KIND == kPull) {
    f[0] = Storage<S>::load(src + k);
#pragma unroll
    for (int i = 1; i < Q; ++i) f[i] = Storage<S>::load(src + off[i]);
    Storage<S>::relax(f, p, (uint32_t)k);
#pragma unroll
    for (int i = 0; i < Q; ++i) Storage<S>::store(dir(dst, i, stride) + k, f[i]);
  } else {
    f[0] = Storage<S>::load(dst + k);
#pragma unroll
    for (int i = 1; i < Q; ++i) f[i] = Storage<S>::load(dst + off[i]);
    Storage<S>::relax(f, p, (uint32_t)k);
    // Hiding the base pointer from the compiler makes the scatter rebuild its
    // addresses from the 32-bit offsets instead of keeping the gather's 18
    // 64-bit addresses live across the collision (64 instead of 80 registers,
    // and no spills for the FP64-storage double-float collision). It pays for
    // that format (+8% on the porous 256^3 medium) and for stochastic FP16
    // (+2%); for the others it was equal or slower.
    S* out = dst;
    if constexpr (std::is_same<S, f64df>::value || std::is_same<S, h16sr>::value) asm volatile("" : "+l"(out));
    Storage<S>::store(out + k, f[0]);
#pragma unroll
    for (int i = 1; i < Q; ++i) Storage<S>::store(out + off[opp(i)], f[i]);
  }
}

// The same persistent, double-buffered sweep reading the run-indexed code of
// the links (lbm_ria.cu) instead of the table: per tile of T nodes (T/32
// chunks) one bulk copy brings the chunks' headers (144 bytes each) and one the
// chunks' slice of the run pool, rounded out to 16-byte boundaries. Each lane
// decodes its 18 links from shared memory. Results are those of the table
// kernel, bit for bit: only the way the offsets are found differs.
constexpr size_t staged_ria_smem_bytes(int threads) {
  return (size_t)2 * ((size_t)(threads / 32) * (Q - 1) * sizeof(uint2) + ((size_t)(Q - 1) * threads + 8) * sizeof(uint32_t));
}

template <typename S, int KIND>
__global__ void __launch_bounds__(kStagedMaxThreads) k_list_staged_ria(const S* __restrict__ src, S* __restrict__ dst,
                                                                       const uint2* __restrict__ head,
                                                                       const uint32_t* __restrict__ pool,
                                                                       const uint32_t* __restrict__ chunk_start,
                                                                       int64_t nf, int64_t stride, ParamsT<S> lp,
                                                                       int* status) {
  const ParamsT<S> p = begin_sweep<S>(lp);
  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ uint64_t bar[2];
  __shared__ uint32_t pool_base[2];
  __shared__ int abort_flag;
  const int T = blockDim.x, C = T / 32;
  const int j = threadIdx.x, lane = j & 31, w = j >> 5;
  // buffer b: headers at shead0 + b 18 C, pool slice at spool0 + b (18 T + 8) words (no arrays
  // indexed by b: they would live in local memory)
  uint2* const shead0 = reinterpret_cast<uint2*>(smem);
  uint32_t* const spool0 = reinterpret_cast<uint32_t*>(shead0 + 2 * (Q - 1) * C);
  const int64_t chunks = (nf + 31) / 32;
  const int64_t ntiles = (nf + T - 1) / T;
  if (j == 0) {
    mbar_init(&bar[0], 1);
    mbar_init(&bar[1], 1);
    fence_mbar_init();
    abort_flag = 0;
  }
  __syncthreads();
  auto issue = [&](int64_t tile, int b) {
    const int64_t c0 = tile * C;
    const int64_t c1 = c0 + C < chunks ? c0 + C : chunks;
    const uint32_t hbytes = (uint32_t)((c1 - c0) * (Q - 1) * sizeof(uint2));   // 144 per chunk
    const uint32_t a0 = chunk_start[c0] & ~3u, a1 = (chunk_start[c1] + 3u) & ~3u;
    const uint32_t pbytes = (a1 - a0) * (uint32_t)sizeof(uint32_t);
    pool_base[b] = a0;
    mbar_arrive_expect_tx(&bar[b], hbytes + pbytes);
    bulk_copy_g2s(shead0 + b * (Q - 1) * C, head + c0 * (Q - 1), hbytes, &bar[b]);
    bulk_copy_g2s(spool0 + b * ((Q - 1) * T + 8), pool + a0, pbytes, &bar[b]);
  };
  const unsigned le = (2u << lane) - 1u;   // lanes 0..lane
  int64_t t = blockIdx.x;
  if (j == 0 && t < ntiles) issue(t, 0);
  // pass `it` uses buffer it & 1 in its ((it >> 1) + 1)-th fill: phase parity (it >> 1) & 1
  for (int it = 0; t < ntiles; t += gridDim.x, ++it) {
    const int b = it & 1;
    const int64_t tn = t + gridDim.x;
    if (j == 0 && tn < ntiles) {
      fence_proxy_async_smem();
      issue(tn, b ^ 1);
    }
    if (!mbar_wait_bounded(&bar[b], (uint32_t)(it >> 1) & 1u)) {
      atomicOr(status, kStatusWaitTimeout);
      abort_flag = 1;
    } else {
      const int64_t k = t * T + j;
      if (k < nf)
        ria_node<S, KIND>(src, dst, shead0 + b * (Q - 1) * C + w * (Q - 1), spool0 + b * ((Q - 1) * T + 8),
                          pool_base[b], le, lane, k, stride, p);
    }
    __syncthreads();
    if (abort_flag) {
      // never leave a copy in flight into shared memory that is about to be
      // released: this tile's and, when issued, the next one's
      if (j == 0) {
        mbar_wait_bounded(&bar[b], (uint32_t)(it >> 1) & 1u);
        if (tn < ntiles) mbar_wait_bounded(&bar[b ^ 1], (uint32_t)((it + 1) >> 1) & 1u);
      }
      return;
    }
  }
}

template <typename S, int KIND>
int staged_ria_grid(int threads, int64_t ntiles) {
  static std::once_flag once;
  std::call_once(once, [] {
    cudaFuncSetAttribute(k_list_staged_ria<S, KIND>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)staged_ria_smem_bytes(kStagedMaxThreads));
  });
  int dev = 0, sms = 0, per_sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_list_staged_ria<S, KIND>, threads,
                                                staged_ria_smem_bytes(threads));
  const int64_t g = (int64_t)std::max(1, sms) * std::max(1, per_sm);
  return (int)std::min<int64_t>(g, ntiles);
}

template <typename S, int KIND>
int staged_grid(int threads, int64_t ntiles) {
  static std::once_flag once;
  std::call_once(once, [] {
    cudaFuncSetAttribute(k_list_staged<S, KIND>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)staged_smem_bytes(kStagedMaxThreads));
  });
  int dev = 0, sms = 0, per_sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_list_staged<S, KIND>, threads, staged_smem_bytes(threads));
  const int64_t g = (int64_t)std::max(1, sms) * std::max(1, per_sm);
  return (int)std::min<int64_t>(g, ntiles);
}

template <typename S>
cudaError_t sweep_typed(const LatticeView& v, SweepKind kind, int parity, const void* src_, void* dst_,
                        const TrtParams& tp, int threads, int cells_per_thread, cudaStream_t s) {
  const S* src = static_cast<const S*>(src_);
  S* dst = static_cast<S*>(dst_);
  const ParamsT<S> p = params_as<S>(tp, v, parity);
  if (threads <= 0) threads = 256;
  if (!v.indirect && cells_per_thread == 2) {
    const int bx = std::min(threads, ((v.nx / 2 + 31) / 32) * 32);
    const dim3 grid((unsigned)(v.ny * v.nz), (unsigned)((v.nx + 2 * bx - 1) / (2 * bx)));
    // adjacent-pair kernels: one thread per (x, x+1), x even
    const int px = std::min(threads, ((v.nx / 2 + 31) / 32) * 32);
    const dim3 pair_grid((unsigned)(v.ny * v.nz), (unsigned)((v.nx / 2 + px - 1) / px));
    switch (kind) {
      case kPull:
        if constexpr (kHasPairIO<S>) {
          if (v.nx % 2 == 0 && !v.has_halfway) {
            k_dense_pull_pair<S><<<pair_grid, px, 0, s>>>(src, dst, v.flags, v.nx, v.ny, v.nz, v.stride, p);
            break;
          }
        }
        if (v.has_halfway)
          k_dense_pull2<S, true><<<grid, bx, 0, s>>>(src, dst, v.flags, v.nx, v.ny, v.nz, v.stride, p);
        else
          k_dense_pull2<S, false><<<grid, bx, 0, s>>>(src, dst, v.flags, v.nx, v.ny, v.nz, v.stride, p);
        break;
      case kAAEven:
        if constexpr (kHasPairIO<S>) {
          if (v.nx % 2 == 0) {
            k_dense_aa_even_pair<S><<<pair_grid, px, 0, s>>>(dst, v.flags, v.nx, v.stride, p);
            break;
          }
        }
        k_dense_aa_even2<S><<<grid, bx, 0, s>>>(dst, v.flags, v.nx, v.stride, p);
        break;
      case kAAOdd:
        if constexpr (kHasPairIO<S>) {
          if (v.nx % 2 == 0 && !v.has_halfway) {
            k_dense_aa_odd_pair<S><<<pair_grid, px, 0, s>>>(dst, v.flags, v.nx, v.ny, v.nz, v.stride, p);
            break;
          }
        }
        if (v.has_halfway)
          k_dense_aa_odd2<S, true><<<grid, bx, 0, s>>>(dst, v.flags, v.nx, v.ny, v.nz, v.stride, p);
        else
          k_dense_aa_odd2<S, false><<<grid, bx, 0, s>>>(dst, v.flags, v.nx, v.ny, v.nz, v.stride, p);
        break;
    }
  } else if (!v.indirect) {
    const int bx = std::min(threads, ((v.nx + 31) / 32) * 32);
    const dim3 grid((unsigned)(v.ny * v.nz), (unsigned)((v.nx + bx - 1) / bx));
    switch (kind) {
      case kPull:
        if (v.has_halfway)
          k_dense_pull<S, true><<<grid, bx, 0, s>>>(src, dst, v.flags, v.nx, v.ny, v.nz, v.stride, p);
        else
          k_dense_pull<S, false><<<grid, bx, 0, s>>>(src, dst, v.flags, v.nx, v.ny, v.nz, v.stride, p);
        break;
      case kAAEven:
        k_dense_aa_even<S><<<grid, bx, 0, s>>>(dst, v.flags, v.nx, v.stride, p);
        break;
      case kAAOdd:
        if (v.has_halfway)
          k_dense_aa_odd<S, true><<<grid, bx, 0, s>>>(dst, v.flags, v.nx, v.ny, v.nz, v.stride, p);
        else
          k_dense_aa_odd<S, false><<<grid, bx, 0, s>>>(dst, v.flags, v.nx, v.ny, v.nz, v.stride, p);
        break;
    }
  } else {
    if (v.n_nodes == 0) return cudaSuccess;
    const unsigned blocks = (unsigned)((v.n_nodes + threads - 1) / threads);
    const bool ria = v.status && v.ria_head && v.ria_pool && v.ria_chunk_start;
    switch (kind) {
      case kPull:
        if (ria)
          k_list_staged_ria<S, kPull><<<staged_ria_grid<S, kPull>(threads, blocks), threads,
                                         staged_ria_smem_bytes(threads), s>>>(
              src, dst, v.ria_head, v.ria_pool, v.ria_chunk_start, v.n_nodes, v.stride, p, v.status);
        else if (v.status)
          k_list_staged<S, kPull><<<staged_grid<S, kPull>(threads, blocks), threads, staged_smem_bytes(threads), s>>>(
              src, dst, v.link, v.n_nodes, v.stride, p, v.status);
        else
          k_list_pull<S><<<blocks, threads, 0, s>>>(src, dst, v.link, v.n_nodes, v.stride, p);
        break;
      case kAAEven:
        k_list_aa_even<S><<<blocks, threads, 0, s>>>(dst, v.n_nodes, v.stride, p);
        break;
      case kAAOdd:
        if (ria)
          k_list_staged_ria<S, kAAOdd><<<staged_ria_grid<S, kAAOdd>(threads, blocks), threads,
                                          staged_ria_smem_bytes(threads), s>>>(
              nullptr, dst, v.ria_head, v.ria_pool, v.ria_chunk_start, v.n_nodes, v.stride, p, v.status);
        else if (v.status)
          k_list_staged<S, kAAOdd><<<staged_grid<S, kAAOdd>(threads, blocks), threads, staged_smem_bytes(threads),
                                      s>>>(nullptr, dst, v.link, v.n_nodes, v.stride, p, v.status);
        else
          k_list_aa_odd<S><<<blocks, threads, 0, s>>>(dst, v.link, v.n_nodes, v.stride, p);
        break;
    }
  }
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_sweep(const LatticeView& v, SweepKind kind, int parity, const void* src, void* dst,
                         const TrtParams& p, int threads, int cells_per_thread, cudaStream_t s) {
  switch (v.prec) {
    case kF64: return sweep_typed<double>(v, kind, parity, src, dst, p, threads, cells_per_thread, s);
    case kF32: return sweep_typed<float>(v, kind, parity, src, dst, p, threads, cells_per_thread, s);
    case kF16: return sweep_typed<__half>(v, kind, parity, src, dst, p, threads, cells_per_thread, s);
    case kF64DF: return sweep_typed<f64df>(v, kind, parity, src, dst, p, threads, cells_per_thread, s);
    case kF32DF: return sweep_typed<f32df>(v, kind, parity, src, dst, p, threads, cells_per_thread, s);
    case kF16SR: return sweep_typed<h16sr>(v, kind, parity, src, dst, p, threads, cells_per_thread, s);
  }
  return cudaErrorInvalidValue;
}

}  // namespace lbm
