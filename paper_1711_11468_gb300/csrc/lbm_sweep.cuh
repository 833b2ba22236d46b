// Per-node bodies of the fused collide-and-propagate sweep (Sec. 3 of
// arXiv 1711.11468), shared by the single-lattice kernels and the batched
// kernel. Structure-of-arrays storage: direction i of node n at pdf[i*stride + n].
//
//   pull (two grids, Table 1 "pull-soa" / "list-pull-soa"): gather f_i from
//     slot i of x - c_i in src, collide, write slot i of x in dst.
//   AA even (one grid, Table 1 "aa-soa" / "list-aa-soa"): read slot i of x,
//     collide, write the result of direction i into slot opp(i) of x.
//   AA odd: gather slot opp(i) of x - c_i, collide, scatter into slot i of
//     x + c_i. Each node writes exactly the slots it read, so the in-place
//     update is race-free (Sec. 3 "AA Pattern Kernels").
// Bounce-back (Sec. 2, Sec. 3.2) is fused: a link into a half-way solid cell
// reflects into the node's own opposite slot (the list encodes it as adj = -1);
// a full-way solid cell reverses its populations in the pull sweep and needs no
// work at all in the AA sweep, where the reversed population is the one already
// parked in its slot.
#pragma once

#include <type_traits>

#include "lbm_internal.h"
#include "lbm_model.cuh"

namespace lbm {

template <typename S>
using Arith = typename Storage<S>::A;
template <typename S>
using RawT = typename Storage<S>::Raw;
template <typename S>
using ParamsT = typename Storage<S>::Params;

// TRT constants in the arithmetic type of storage format S (lbm_sweep.cu).
template <typename S>
Trt<Arith<S>> trt_as(const TrtParams& p);

// Launch parameters of one sweep of one lattice: the TRT constants plus, for
// the stochastic format, the lattice's random stream and the sweep counter of
// this parity.
template <typename S>
ParamsT<S> params_as(const TrtParams& p, const LatticeView& v, int parity) {
  if constexpr (std::is_same<S, h16sr>::value) {
    TrtSr q;
    static_cast<Trt<float>&>(q) = trt_as<S>(p);
    // the collision of scaled values (see collide): c4 / 2^14, force terms * 2^14
    const float scale = (float)(1 << kSrScaleLog2);
    for (int c = 0; c < 2; ++c) q.c4[c] /= scale;
    for (int k = 0; k < 9; ++k) q.fk[k] = (float)(p.fk[k] * (double)scale);
    q.seed = v.sr_seed;
    q.base = 0;
    q.ctr = v.sweep_ctr;
    q.parity = parity & 1;
    return q;
  } else {
    return trt_as<S>(p);
  }
}

// Wrapped neighbour offsets of one cell of a full array.
struct Nbr {
  int xm, xp, ym, yp, zm, zp;  // offsets to x-1, x+1, y-1, y+1, z-1, z+1
  __device__ __forceinline__ Nbr(int x, int y, int z, int nx, int ny, int nz) {
    const int plane = nx * ny;
    xm = (x == 0) ? nx - 1 : -1;
    xp = (x == nx - 1) ? 1 - nx : 1;
    ym = (y == 0) ? (ny - 1) * nx : -nx;
    yp = (y == ny - 1) ? -(ny - 1) * nx : nx;
    zm = (z == 0) ? (nz - 1) * plane : -plane;
    zp = (z == nz - 1) ? -(nz - 1) * plane : plane;
  }
  // offset to the upstream cell x - c_i
  __device__ __forceinline__ int up(int i) const {
    return (cx(i) > 0 ? xm : (cx(i) < 0 ? xp : 0)) + (cy(i) > 0 ? ym : (cy(i) < 0 ? yp : 0)) +
           (cz(i) > 0 ? zm : (cz(i) < 0 ? zp : 0));
  }
  // offset to the downstream cell x + c_i
  __device__ __forceinline__ int down(int i) const { return up(opp(i)); }
};

// The odd AA step scatters to the 18 addresses its gather read. Passing the
// node index and the neighbour offsets through an empty asm statement between
// the two hides that from the compiler, which then recomputes the addresses
// after the collision (a few integer instructions each) instead of keeping 18
// 64-bit addresses live across it. Done for the shifted FP32 and FP16 formats,
// whose sweeps are bound by memory requests in flight: 44-72 instead of 78-123
// registers, +2% on the 256^3 duct. The double-float collisions are bound by
// instruction issue and lose more to the extra instructions than they gain;
// plain FP64 is bound by its FP64 pipe either way. With half-way walls (kHW:
// the addresses depend on neighbour flags too) it is done for every format:
// there the FP64 and double-float kernels would otherwise spill 90-290 bytes.
template <typename S, bool kHW>
constexpr bool kRecomputeScatter =
    kHW || std::is_same<S, __half>::value || std::is_same<S, float>::value || std::is_same<S, h16sr>::value;

template <typename S, bool kHW>
__device__ __forceinline__ void opaque(Nbr& nb, int& n) {
  if constexpr (kRecomputeScatter<S, kHW>)
    asm volatile("" : "+r"(n), "+r"(nb.xm), "+r"(nb.xp), "+r"(nb.ym), "+r"(nb.yp), "+r"(nb.zm), "+r"(nb.zp));
}

template <typename S>
__device__ __forceinline__ const S* dir(const S* base, int i, int64_t stride) {
  return base + (int64_t)i * stride;
}
template <typename S>
__device__ __forceinline__ S* dir(S* base, int i, int64_t stride) {
  return base + (int64_t)i * stride;
}

template <typename R>
__device__ __forceinline__ void reverse(R (&f)[Q]) {
#pragma unroll
  for (int k = 1; k <= 9; ++k) {
    const R t = f[k];
    f[k] = f[k + 9];
    f[k + 9] = t;
  }
}

// ------------------------------------------------------------- full array
template <typename S, bool kHW>
__device__ __forceinline__ void pull_dense_node(const S* __restrict__ src, S* __restrict__ dst,
                                                const uint8_t* __restrict__ flags, int x, int y, int z, int n,
                                                int nx, int ny, int nz, int64_t stride, const ParamsT<S>& p) {
  const uint8_t fl = flags[n];
  if (fl == kSolidHalfway) return;
  const Nbr nb(x, y, z, nx, ny, nz);
  RawT<S> f[Q];
#pragma unroll
  for (int i = 0; i < Q; ++i) {
    const int m = n + nb.up(i);
    if (kHW && i != 0 && flags[m] == kSolidHalfway)
      f[i] = Storage<S>::load(dir(src, opp(i), stride) + n);
    else
      f[i] = Storage<S>::load(dir(src, i, stride) + m);
  }
  if (fl == kSolidFullway)
    reverse(f);
  else
    Storage<S>::relax(f, p, (uint32_t)n);
#pragma unroll
  for (int i = 0; i < Q; ++i) Storage<S>::store(dir(dst, i, stride) + n, f[i]);
}

// Node-local even step; the caller skips nodes that are not fluid.
template <typename S>
__device__ __forceinline__ void aa_even_node(S* __restrict__ pdf, int64_t k, int64_t stride,
                                             const ParamsT<S>& p) {
  RawT<S> f[Q];
#pragma unroll
  for (int i = 0; i < Q; ++i) f[i] = Storage<S>::load(dir(pdf, i, stride) + k);
  Storage<S>::relax(f, p, (uint32_t)k);
#pragma unroll
  for (int i = 0; i < Q; ++i) Storage<S>::store(dir(pdf, opp(i), stride) + k, f[i]);
}

// Odd step at fluid cell n of a full array; the caller skips solid cells.
template <typename S, bool kHW>
__device__ __forceinline__ void aa_odd_dense_node(S* __restrict__ pdf, const uint8_t* __restrict__ flags, int x,
                                                  int y, int z, int n, int nx, int ny, int nz, int64_t stride,
                                                  const ParamsT<S>& p) {
  Nbr nb(x, y, z, nx, ny, nz);
  RawT<S> f[Q];
#pragma unroll
  for (int i = 0; i < Q; ++i) {
    const int m = n + nb.up(i);
    if (kHW && i != 0 && flags[m] == kSolidHalfway)
      f[i] = Storage<S>::load(dir(pdf, i, stride) + n);
    else
      f[i] = Storage<S>::load(dir(pdf, opp(i), stride) + m);
  }
  Storage<S>::relax(f, p, (uint32_t)n);
  opaque<S, kHW>(nb, n);
#pragma unroll
  for (int i = 0; i < Q; ++i) {
    const int m = n + nb.down(i);
    if (kHW && i != 0 && flags[m] == kSolidHalfway)
      Storage<S>::store(dir(pdf, opp(i), stride) + n, f[i]);
    else
      Storage<S>::store(dir(pdf, i, stride) + m, f[i]);
  }
}

// ---------------------------------------- full array, two cells per thread
// The bodies above split into gather and scatter phases, so that one thread
// can issue the loads of two cells before it collides either: twice the bytes
// in flight per thread for the same register budget of one collision. The
// arithmetic per cell is unchanged, so results are bitwise those of one cell per
// thread.
template <typename S, bool kHW>
__device__ __forceinline__ void pull_dense_gather(const S* __restrict__ src, const uint8_t* __restrict__ flags,
                                                  const Nbr& nb, int n, int64_t stride, RawT<S> (&f)[Q]) {
#pragma unroll
  for (int i = 0; i < Q; ++i) {
    const int m = n + nb.up(i);
    if (kHW && i != 0 && flags[m] == kSolidHalfway)
      f[i] = Storage<S>::load(dir(src, opp(i), stride) + n);
    else
      f[i] = Storage<S>::load(dir(src, i, stride) + m);
  }
}

template <typename S, bool kHW>
__device__ __forceinline__ void aa_odd_dense_gather(const S* __restrict__ pdf, const uint8_t* __restrict__ flags,
                                                    const Nbr& nb, int n, int64_t stride, RawT<S> (&f)[Q]) {
#pragma unroll
  for (int i = 0; i < Q; ++i) {
    const int m = n + nb.up(i);
    if (kHW && i != 0 && flags[m] == kSolidHalfway)
      f[i] = Storage<S>::load(dir(pdf, i, stride) + n);
    else
      f[i] = Storage<S>::load(dir(pdf, opp(i), stride) + m);
  }
}

template <typename S, bool kHW>
__device__ __forceinline__ void aa_odd_dense_scatter(S* __restrict__ pdf, const uint8_t* __restrict__ flags,
                                                     Nbr nb, int n, int64_t stride, const RawT<S> (&f)[Q]) {
  opaque<S, kHW>(nb, n);
#pragma unroll
  for (int i = 0; i < Q; ++i) {
    const int m = n + nb.down(i);
    if (kHW && i != 0 && flags[m] == kSolidHalfway)
      Storage<S>::store(dir(pdf, opp(i), stride) + n, f[i]);
    else
      Storage<S>::store(dir(pdf, i, stride) + m, f[i]);
  }
}

// ------------------------------------------------------------ fluid list
// link[(i-1)*stride + k]: element offset of f_i for node k, bounce-back
// resolved (see lbm_internal.h). Gathers and scatters are unconditional.
template <typename S>
__device__ __forceinline__ void pull_list_node(const S* __restrict__ src, S* __restrict__ dst,
                                               const uint32_t* __restrict__ link, int64_t k, int64_t stride,
                                               const ParamsT<S>& p) {
  RawT<S> f[Q];
  f[0] = Storage<S>::load(src + k);
#pragma unroll
  for (int i = 1; i < Q; ++i) f[i] = Storage<S>::load(src + __ldg(link + (int64_t)(i - 1) * stride + k));
  Storage<S>::relax(f, p, (uint32_t)k);
#pragma unroll
  for (int i = 0; i < Q; ++i) Storage<S>::store(dir(dst, i, stride) + k, f[i]);
}

template <typename S>
__device__ __forceinline__ void aa_odd_list_node(S* __restrict__ pdf, const uint32_t* __restrict__ link, int64_t k,
                                                 int64_t stride, const ParamsT<S>& p) {
  uint32_t off[Q];
#pragma unroll
  for (int i = 1; i < Q; ++i) off[i] = __ldg(link + (int64_t)(i - 1) * stride + k);
  RawT<S> f[Q];
  f[0] = Storage<S>::load(pdf + k);
#pragma unroll
  for (int i = 1; i < Q; ++i) f[i] = Storage<S>::load(pdf + off[i]);
  Storage<S>::relax(f, p, (uint32_t)k);
  Storage<S>::store(pdf + k, f[0]);
  // f*_i goes where f_opp(i) came from: the downstream node's slot i, or slot opp(i) of k
#pragma unroll
  for (int i = 1; i < Q; ++i) Storage<S>::store(pdf + off[opp(i)], f[i]);
}

// Gather / scatter halves of the list bodies, for two nodes per thread.
template <typename S>
__device__ __forceinline__ void list_gather(const S* __restrict__ pdf, const uint32_t* __restrict__ link, int64_t k,
                                            int64_t stride, RawT<S> (&f)[Q]) {
  f[0] = Storage<S>::load(pdf + k);
#pragma unroll
  for (int i = 1; i < Q; ++i) f[i] = Storage<S>::load(pdf + __ldg(link + (int64_t)(i - 1) * stride + k));
}

// AA odd scatter: f*_i where f_opp(i) was gathered (the links are read again, from cache).
template <typename S>
__device__ __forceinline__ void list_aa_scatter(S* __restrict__ pdf, const uint32_t* __restrict__ link, int64_t k,
                                                int64_t stride, const RawT<S> (&f)[Q]) {
  Storage<S>::store(pdf + k, f[0]);
#pragma unroll
  for (int i = 1; i < Q; ++i) Storage<S>::store(pdf + __ldg(link + (int64_t)(opp(i) - 1) * stride + k), f[i]);
}

// The same two list bodies with the node's links in shared memory:
// slink[(i-1)*T + j] for direction i of the tile's j-th node.
template <typename S>
__device__ __forceinline__ void pull_list_node_staged(const S* __restrict__ src, S* __restrict__ dst,
                                                      const uint32_t* slink, int T, int j, int64_t k, int64_t stride,
                                                      const ParamsT<S>& p) {
  RawT<S> f[Q];
  f[0] = Storage<S>::load(src + k);
#pragma unroll
  for (int i = 1; i < Q; ++i) f[i] = Storage<S>::load(src + slink[(i - 1) * T + j]);
  Storage<S>::relax(f, p, (uint32_t)k);
#pragma unroll
  for (int i = 0; i < Q; ++i) Storage<S>::store(dir(dst, i, stride) + k, f[i]);
}

template <typename S>
__device__ __forceinline__ void aa_odd_list_node_staged(S* __restrict__ pdf, const uint32_t* slink, int T, int j,
                                                        int64_t k, const ParamsT<S>& p) {
  RawT<S> f[Q];
  f[0] = Storage<S>::load(pdf + k);
#pragma unroll
  for (int i = 1; i < Q; ++i) f[i] = Storage<S>::load(pdf + slink[(i - 1) * T + j]);
  Storage<S>::relax(f, p, (uint32_t)k);
  Storage<S>::store(pdf + k, f[0]);
#pragma unroll
  for (int i = 1; i < Q; ++i) {
    // re-read from shared memory rather than keep 18 offsets live across the collision
    const uint32_t o = reinterpret_cast<const volatile uint32_t*>(slink)[(opp(i) - 1) * T + j];
    Storage<S>::store(pdf + o, f[i]);
  }
}

}  // namespace lbm
