// Fused collide-and-propagate sweeps of one lattice (Sec. 3 of arXiv 1711.11468),
// structure-of-arrays storage: direction i of node n lives at pdf[i*stride + n].
//
//   dense pull   : one-step pull with two grids on the full array (Table 1
//                  "pull-soa"): gather f_i from x - c_i, collide, write locally.
//   dense AA     : the AA pattern on one grid (Table 1 "aa-soa", "aa-vec-soa").
//                  Even step: node-local, result of direction i stored in slot
//                  opp(i). Odd step: gather slot opp(i) of x - c_i, collide,
//                  scatter into slot i of x + c_i. Each thread writes exactly the
//                  slots it read, so the sweep is race-free in place.
//   list pull/AA : the same on the fluid list with the int32 adjacency list
//                  (Table 1 "list-pull-soa", "list-aa-soa"): bounce-back and
//                  periodicity are encoded by adj = -1 and by the wrapped
//                  neighbour indices (Sec. 3.2).
// Bounce-back on the full array (Sec. 2, Sec. 3.2) is fused into the sweep
// instead of a separate pass: a full-way solid cell reverses its populations
// (pull) or, in the AA pattern, is left alone -- the reversed population is
// exactly the one already parked in its slot, so the in-place sweep realises
// full-way bounce-back with no work at solid cells. A link into a half-way
// solid cell reflects back into the node's own opposite slot.
#include "lbm_internal.h"
#include "lbm_model.cuh"

namespace lbm {
namespace {

template <typename S>
using Arith = typename Storage<S>::A;

template <typename S>
Trt<Arith<S>> trt_as(const TrtParams& p) {
  Trt<Arith<S>> t;
  t.omega_p = (Arith<S>)p.omega_p;
  t.omega_m = (Arith<S>)p.omega_m;
  for (int k = 0; k < 9; ++k) t.fk[k] = (Arith<S>)p.fk[k];
  return t;
}

// Wrapped neighbour offsets of one cell, and the offset to x - c_i / x + c_i.
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

template <typename S>
__device__ __forceinline__ const S* dir(const S* base, int i, int64_t stride) {
  return base + (int64_t)i * stride;
}
template <typename S>
__device__ __forceinline__ S* dir(S* base, int i, int64_t stride) {
  return base + (int64_t)i * stride;
}

template <typename A>
__device__ __forceinline__ void reverse(A (&f)[Q]) {
#pragma unroll
  for (int k = 1; k <= 9; ++k) {
    const A t = f[k];
    f[k] = f[k + 9];
    f[k + 9] = t;
  }
}

// ------------------------------------------------------------- full array
// Grid: blockIdx.x = row (y + ny*z), blockIdx.y * blockDim.x + threadIdx.x = x.
template <typename S, bool kHW>
__global__ void __launch_bounds__(512) k_dense_pull(const S* __restrict__ src, S* __restrict__ dst,
                                                     const uint8_t* __restrict__ flags, int nx, int ny,
                                                     int nz, int64_t stride, Trt<Arith<S>> p) {
  using A = Arith<S>;
  const int x = blockIdx.y * blockDim.x + threadIdx.x;
  if (x >= nx) return;
  const int row = blockIdx.x;
  const int z = row / ny, y = row - z * ny;
  const int n = x + nx * row;
  const uint8_t fl = flags[n];
  if (fl == kSolidHalfway) return;
  const Nbr nb(x, y, z, nx, ny, nz);
  A f[Q];
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
    collide<A, Storage<S>::kShifted>(f, p);
#pragma unroll
  for (int i = 0; i < Q; ++i) Storage<S>::store(dir(dst, i, stride) + n, f[i]);
}

template <typename S>
__global__ void __launch_bounds__(512) k_dense_aa_even(S* __restrict__ pdf, const uint8_t* __restrict__ flags,
                                                        int nx, int64_t stride, Trt<Arith<S>> p) {
  using A = Arith<S>;
  const int x = blockIdx.y * blockDim.x + threadIdx.x;
  if (x >= nx) return;
  const int n = x + nx * (int)blockIdx.x;
  if (flags[n] != kFluid) return;
  A f[Q];
#pragma unroll
  for (int i = 0; i < Q; ++i) f[i] = Storage<S>::load(dir(pdf, i, stride) + n);
  collide<A, Storage<S>::kShifted>(f, p);
#pragma unroll
  for (int i = 0; i < Q; ++i) Storage<S>::store(dir(pdf, opp(i), stride) + n, f[i]);
}

template <typename S, bool kHW>
__global__ void __launch_bounds__(512) k_dense_aa_odd(S* __restrict__ pdf, const uint8_t* __restrict__ flags,
                                                       int nx, int ny, int nz, int64_t stride, Trt<Arith<S>> p) {
  using A = Arith<S>;
  const int x = blockIdx.y * blockDim.x + threadIdx.x;
  if (x >= nx) return;
  const int row = blockIdx.x;
  const int z = row / ny, y = row - z * ny;
  const int n = x + nx * row;
  if (flags[n] != kFluid) return;
  const Nbr nb(x, y, z, nx, ny, nz);
  A f[Q];
#pragma unroll
  for (int i = 0; i < Q; ++i) {
    const int m = n + nb.up(i);
    if (kHW && i != 0 && flags[m] == kSolidHalfway)
      f[i] = Storage<S>::load(dir(pdf, i, stride) + n);
    else
      f[i] = Storage<S>::load(dir(pdf, opp(i), stride) + m);
  }
  collide<A, Storage<S>::kShifted>(f, p);
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
// adj[(i-1)*stride + k] = list index of the upstream node x_k - c_i, or -1.
template <typename S>
__global__ void __launch_bounds__(512) k_list_pull(const S* __restrict__ src, S* __restrict__ dst,
                                                    const int32_t* __restrict__ adj, int64_t nf, int64_t stride,
                                                    Trt<Arith<S>> p) {
  using A = Arith<S>;
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= nf) return;
  A f[Q];
  f[0] = Storage<S>::load(src + k);
#pragma unroll
  for (int i = 1; i < Q; ++i) {
    const int32_t a = __ldg(adj + (int64_t)(i - 1) * stride + k);
    f[i] = a >= 0 ? Storage<S>::load(dir(src, i, stride) + a) : Storage<S>::load(dir(src, opp(i), stride) + k);
  }
  collide<A, Storage<S>::kShifted>(f, p);
#pragma unroll
  for (int i = 0; i < Q; ++i) Storage<S>::store(dir(dst, i, stride) + k, f[i]);
}

template <typename S>
__global__ void __launch_bounds__(512) k_list_aa_even(S* __restrict__ pdf, int64_t nf, int64_t stride,
                                                       Trt<Arith<S>> p) {
  using A = Arith<S>;
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= nf) return;
  A f[Q];
#pragma unroll
  for (int i = 0; i < Q; ++i) f[i] = Storage<S>::load(dir(pdf, i, stride) + k);
  collide<A, Storage<S>::kShifted>(f, p);
#pragma unroll
  for (int i = 0; i < Q; ++i) Storage<S>::store(dir(pdf, opp(i), stride) + k, f[i]);
}

template <typename S>
__global__ void __launch_bounds__(512) k_list_aa_odd(S* __restrict__ pdf, const int32_t* __restrict__ adj,
                                                      int64_t nf, int64_t stride, Trt<Arith<S>> p) {
  using A = Arith<S>;
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= nf) return;
  int32_t a[Q];
  a[0] = (int32_t)k;
#pragma unroll
  for (int i = 1; i < Q; ++i) a[i] = __ldg(adj + (int64_t)(i - 1) * stride + k);
  A f[Q];
  f[0] = Storage<S>::load(pdf + k);
#pragma unroll
  for (int i = 1; i < Q; ++i)
    f[i] = a[i] >= 0 ? Storage<S>::load(dir(pdf, opp(i), stride) + a[i]) : Storage<S>::load(dir(pdf, i, stride) + k);
  collide<A, Storage<S>::kShifted>(f, p);
  Storage<S>::store(pdf + k, f[0]);
#pragma unroll
  for (int i = 1; i < Q; ++i) {
    const int32_t d = a[opp(i)];   // downstream node x_k + c_i
    if (d >= 0)
      Storage<S>::store(dir(pdf, i, stride) + d, f[i]);
    else
      Storage<S>::store(dir(pdf, opp(i), stride) + k, f[i]);
  }
}

template <typename S>
cudaError_t sweep_typed(const LatticeView& v, SweepKind kind, const void* src_, void* dst_, const TrtParams& tp,
                        int threads, cudaStream_t s) {
  const S* src = static_cast<const S*>(src_);
  S* dst = static_cast<S*>(dst_);
  const Trt<Arith<S>> p = trt_as<S>(tp);
  if (threads <= 0) threads = 256;
  if (!v.indirect) {
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
    switch (kind) {
      case kPull:
        k_list_pull<S><<<blocks, threads, 0, s>>>(src, dst, v.adj, v.n_nodes, v.stride, p);
        break;
      case kAAEven:
        k_list_aa_even<S><<<blocks, threads, 0, s>>>(dst, v.n_nodes, v.stride, p);
        break;
      case kAAOdd:
        k_list_aa_odd<S><<<blocks, threads, 0, s>>>(dst, v.adj, v.n_nodes, v.stride, p);
        break;
    }
  }
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_sweep(const LatticeView& v, SweepKind kind, const void* src, void* dst, const TrtParams& p,
                         int threads, cudaStream_t s) {
  switch (v.prec) {
    case kF64: return sweep_typed<double>(v, kind, src, dst, p, threads, s);
    case kF32: return sweep_typed<float>(v, kind, src, dst, p, threads, s);
    case kF16: return sweep_typed<__half>(v, kind, src, dst, p, threads, s);
  }
  return cudaErrorInvalidValue;
}

}  // namespace lbm
