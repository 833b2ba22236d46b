// State conversions and verification reductions.
//
// The stored state depends on the propagation scheme: the two-grid pull keeps
// post-collision values (pull form), the AA pattern alternates between the
// canonical layout and a post-collision layout with swapped slots (AA form,
// Sec. 3 "AA Pattern Kernels"). Everything the ABI returns is canonical
// f_i(x, t) in FP64, so these kernels translate. The reductions (mass,
// momentum, velocity profile) are the FP64 quantities of the verification
// set-up (Sec. 2.1).
#include "lbm_internal.h"
#include "lbm_model.cuh"

namespace lbm {
namespace {

struct Cell {
  int x, y, z;
};

__device__ __forceinline__ int wrapi(int a, int n) { return a < 0 ? a + n : (a >= n ? a - n : a); }

__device__ __forceinline__ int64_t cell_index(const LatticeView& v, int x, int y, int z) {
  return (int64_t)x + (int64_t)v.nx * ((int64_t)y + (int64_t)v.ny * z);
}

__device__ __forceinline__ Cell cell_coords(const LatticeView& v, int64_t n) {
  Cell c;
  const int64_t row = n / v.nx;
  c.x = (int)(n - row * v.nx);
  c.z = (int)(row / v.ny);
  c.y = (int)(row - (int64_t)c.z * v.ny);
  return c;
}

// Neighbour cell x + s*c_i (s = +1 downstream, -1 upstream), wrapped.
__device__ __forceinline__ int64_t nbr_cell(const LatticeView& v, Cell c, int i, int s) {
  return cell_index(v, wrapi(c.x + s * cx(i), v.nx), wrapi(c.y + s * cy(i), v.ny), wrapi(c.z + s * cz(i), v.nz));
}

template <typename S>
__device__ __forceinline__ double load_f64(const S* base, int i, int64_t stride, int64_t node) {
  return Storage<S>::to_f64(base[(int64_t)i * stride + node], i);
}

// Node of cell n in storage (-1 if the cell stores nothing) and whether the
// cell is a half-way solid (a reflecting neighbour).
struct NodeMap {
  const LatticeView& v;
  __device__ __forceinline__ int64_t node(int64_t n) const {
    if (v.indirect) return v.list_index[n];
    return v.flags[n] == kSolidHalfway ? -1 : n;
  }
  __device__ __forceinline__ bool halfway(int64_t n) const {
    return v.indirect ? v.list_index[n] < 0 : v.flags[n] == kSolidHalfway;
  }
};

// Canonical f_i(x, t) of a storing cell n (node k) from storage in `layout`.
template <typename S>
__device__ void gather_canonical(const LatticeView& v, const NodeMap& map, Layout layout, const S* src, int64_t n,
                                 int64_t k, double (&f)[Q]) {
  if (layout == kCanonical) {
#pragma unroll
    for (int i = 0; i < Q; ++i) f[i] = load_f64(src, i, v.stride, k);
    return;
  }
  const Cell c = cell_coords(v, n);
  f[0] = load_f64(src, 0, v.stride, k);
#pragma unroll
  for (int i = 1; i < Q; ++i) {
    const int64_t up = nbr_cell(v, c, i, -1);
    if (map.halfway(up)) {
      // reflected at mid-link: f*_opp(i)(x) lives in slot opp(i) (pull) / i (AA) of x
      f[i] = load_f64(src, layout == kPullForm ? opp(i) : i, v.stride, k);
    } else {
      const int64_t ku = map.node(up);
      f[i] = load_f64(src, layout == kPullForm ? i : opp(i), v.stride, ku);
    }
  }
}

// Source of canonical values: a device array [19][N] or the equilibrium of rho/u.
// (The equilibrium is evaluated per cell by the kernels that take rho/u; at()
// serves the canonical array.)
struct CanonSource {
  const double* canon;
  const double* rho;
  const double* u;
  int64_t N;
  __device__ __forceinline__ double at(int i, int64_t n) const { return canon[(int64_t)i * N + n]; }
};

// One thread per cell of the full array; writes the slots of its node from a
// canonical array, or, in the canonical layout only, from the cell's own
// equilibrium (the other layouts take rho/u through k_equilibrium_push).
template <typename S>
__global__ void k_from_canonical(LatticeView v, Layout layout,
                                 S* __restrict__ dst, CanonSource src) {
  const int64_t n = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= v.n_cells) return;
  const NodeMap map{v};
  const int64_t k = map.node(n);
  if (k < 0) return;
  if (layout == kCanonical) {
    if (src.canon) {
#pragma unroll
      for (int i = 0; i < Q; ++i) dst[(int64_t)i * v.stride + k] = Storage<S>::from_f64(src.at(i, n), i);
    } else {
      // one read of the cell's density and velocity (possibly over the link to
      // host memory) for all 19 slots
      const double r = src.rho ? src.rho[n] : 1.0;
      const double ux = src.u ? src.u[n] : 0.0, uy = src.u ? src.u[src.N + n] : 0.0,
                   uz = src.u ? src.u[2 * src.N + n] : 0.0;
      double feq[Q];
      equilibria_f64(r, ux, uy, uz, feq);
#pragma unroll
      for (int i = 0; i < Q; ++i) dst[(int64_t)i * v.stride + k] = Storage<S>::from_f64(feq[i], i);
    }
    return;
  }
  const Cell c = cell_coords(v, n);
  dst[k] = Storage<S>::from_f64(src.at(0, n), 0);
#pragma unroll
  for (int i = 1; i < Q; ++i) {
    // post-collision value leaving x along i: f_i(x + c_i, t), or f_opp(i)(x, t)
    // if x + c_i is a half-way solid (it came back reflected)
    const int64_t dn = nbr_cell(v, c, i, +1);
    const double val = map.halfway(dn) ? src.at(opp(i), n) : src.at(i, dn);
    const int slot = layout == kPullForm ? i : opp(i);
    dst[(int64_t)slot * v.stride + k] = Storage<S>::from_f64(val, i);
  }
}

// The equilibrium of rho/u in the pull or AA form, pushed: every storing cell
// x evaluates its own equilibrium once (one read of its density and velocity,
// which may sit in host memory) and writes f_i(x) where the layout keeps it --
// slot i (pull) / opp(i) (AA) of the upstream cell x - c_i, when that cell
// stores anything -- and, where x + c_i is a half-way solid, the reflected
// f_opp(i)(x) into its own slot. Each slot is written once. (Gathering each
// slot's value from its downstream cell instead, as k_from_canonical does for a
// canonical array, would read every cell's inputs 19 times.)
template <typename S>
__global__ void k_equilibrium_push(LatticeView v, Layout layout, S* __restrict__ dst, CanonSource src) {
  const int64_t n = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= v.n_cells) return;
  const NodeMap map{v};
  const int64_t k = map.node(n);
  if (k < 0) return;
  const double r = src.rho ? src.rho[n] : 1.0;
  const double ux = src.u ? src.u[n] : 0.0, uy = src.u ? src.u[src.N + n] : 0.0,
               uz = src.u ? src.u[2 * src.N + n] : 0.0;
  double feq[Q];
  equilibria_f64(r, ux, uy, uz, feq);
  const Cell c = cell_coords(v, n);
  dst[k] = Storage<S>::from_f64(feq[0], 0);
#pragma unroll
  for (int i = 1; i < Q; ++i) {
    const int slot = layout == kPullForm ? i : opp(i);
    if (map.halfway(nbr_cell(v, c, i, +1))) dst[(int64_t)slot * v.stride + k] = Storage<S>::from_f64(feq[opp(i)], i);
    const int64_t ku = map.node(nbr_cell(v, c, i, -1));
    if (ku >= 0) dst[(int64_t)slot * v.stride + ku] = Storage<S>::from_f64(feq[i], i);
  }
}

template <typename S>
__global__ void k_to_canonical(LatticeView v, Layout layout,
                               const S* __restrict__ src, double* __restrict__ out) {
  const int64_t n = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= v.n_cells) return;
  const NodeMap map{v};
  const int64_t k = map.node(n);
  double f[Q];
  if (k < 0) {
#pragma unroll
    for (int i = 0; i < Q; ++i) f[i] = 0.0;
  } else {
    gather_canonical<S>(v, map, layout, src, n, k, f);
  }
#pragma unroll
  for (int i = 0; i < Q; ++i) out[(int64_t)i * v.n_cells + n] = f[i];
}

// rho = sum f_i; u = (sum c_i f_i + F/2) / rho at fluid cells, 0 elsewhere.
template <typename S>
__device__ __forceinline__ bool fluid_moments(const LatticeView& v, const NodeMap& map, Layout layout, const S* src,
                                              int64_t n, const double* F, double& rho, double (&u)[3]) {
  const int64_t k = map.node(n);
  const bool fluid = k >= 0 && (v.indirect || v.flags[n] == kFluid);
  rho = 0.0;
  u[0] = u[1] = u[2] = 0.0;
  if (!fluid) return false;
  double f[Q];
  gather_canonical<S>(v, map, layout, src, n, k, f);
  double j[3] = {0.0, 0.0, 0.0};
#pragma unroll
  for (int i = 0; i < Q; ++i) {
    rho += f[i];
    j[0] += cx(i) * f[i];
    j[1] += cy(i) * f[i];
    j[2] += cz(i) * f[i];
  }
  for (int a = 0; a < 3; ++a) u[a] = (j[a] + 0.5 * F[a]) / rho;
  return true;
}

struct Force3 {
  double F[3];
};

template <typename S>
__global__ void k_macroscopic(LatticeView v, Layout layout,
                              const S* __restrict__ src, Force3 force, double* __restrict__ rho_out,
                              double* __restrict__ u_out) {
  const int64_t n = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= v.n_cells) return;
  const NodeMap map{v};
  double rho, u[3];
  fluid_moments<S>(v, map, layout, src, n, force.F, rho, u);
  if (rho_out) rho_out[n] = rho;
  if (u_out)
    for (int a = 0; a < 3; ++a) u_out[(int64_t)a * v.n_cells + n] = u[a];
}

// One block per plane normal to `axis`; threads walk the plane in a fixed
// order and reduce in a fixed tree, so the result is deterministic.
template <typename S>
__global__ void k_profile(LatticeView v, Layout layout,
                          const S* __restrict__ src, Force3 force, int axis, int comp, double* __restrict__ sums,
                          unsigned long long* __restrict__ counts) {
  const int plane = blockIdx.x;
  const int n0 = axis == 0 ? v.ny : v.nx;        // first in-plane axis
  const int n1 = axis == 2 ? v.ny : v.nz;        // second in-plane axis
  const int64_t cells = (int64_t)n0 * n1;
  const NodeMap map{v};
  double acc = 0.0;
  unsigned long long cnt = 0;
  for (int64_t t = threadIdx.x; t < cells; t += blockDim.x) {
    const int a = (int)(t % n0), b = (int)(t / n0);
    int x, y, z;
    if (axis == 0) { x = plane; y = a; z = b; }
    else if (axis == 1) { x = a; y = plane; z = b; }
    else { x = a; y = b; z = plane; }
    double rho, u[3];
    if (fluid_moments<S>(v, map, layout, src, cell_index(v, x, y, z), force.F, rho, u)) {
      acc += u[comp];
      ++cnt;
    }
  }
  __shared__ double sh[1024];
  __shared__ unsigned long long shc[1024];
  sh[threadIdx.x] = acc;
  shc[threadIdx.x] = cnt;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) {
      sh[threadIdx.x] += sh[threadIdx.x + w];
      shc[threadIdx.x] += shc[threadIdx.x + w];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    sums[plane] = sh[0];
    counts[plane] = shc[0];
  }
}

constexpr int kMomThreads = 256;
constexpr int kMomCellsPerThread = 64;

// Partial FP64 sums of mass and momentum over every stored PDF; block b covers
// cells [b*T*C, (b+1)*T*C) in a fixed assignment, reduced in a fixed tree.
template <typename S>
__global__ void __launch_bounds__(kMomThreads) k_moments_partial(LatticeView v, Layout layout, const S* __restrict__ src,
                                                                 double* __restrict__ partials) {
  const NodeMap map{v};
  double acc[4] = {0.0, 0.0, 0.0, 0.0};
  const int64_t base = (int64_t)blockIdx.x * kMomThreads * kMomCellsPerThread;
  for (int c = 0; c < kMomCellsPerThread; ++c) {
    const int64_t n = base + (int64_t)c * kMomThreads + threadIdx.x;
    if (n >= v.n_cells) break;
    const int64_t k = map.node(n);
    if (k < 0) continue;
    double f[Q];
    gather_canonical<S>(v, map, layout, src, n, k, f);
#pragma unroll
    for (int i = 0; i < Q; ++i) {
      acc[0] += f[i];
      acc[1] += cx(i) * f[i];
      acc[2] += cy(i) * f[i];
      acc[3] += cz(i) * f[i];
    }
  }
  __shared__ double sh[4][kMomThreads];
  for (int a = 0; a < 4; ++a) sh[a][threadIdx.x] = acc[a];
  __syncthreads();
  for (int w = kMomThreads / 2; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w)
      for (int a = 0; a < 4; ++a) sh[a][threadIdx.x] += sh[a][threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x < 4) partials[(int64_t)blockIdx.x * 4 + threadIdx.x] = sh[threadIdx.x][0];
}

__global__ void __launch_bounds__(kMomThreads) k_moments_final(const double* __restrict__ partials, int blocks,
                                                               double* __restrict__ out) {
  double acc[4] = {0.0, 0.0, 0.0, 0.0};
  for (int b = threadIdx.x; b < blocks; b += kMomThreads)
    for (int a = 0; a < 4; ++a) acc[a] += partials[(int64_t)b * 4 + a];
  __shared__ double sh[4][kMomThreads];
  for (int a = 0; a < 4; ++a) sh[a][threadIdx.x] = acc[a];
  __syncthreads();
  for (int w = kMomThreads / 2; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w)
      for (int a = 0; a < 4; ++a) sh[a][threadIdx.x] += sh[a][threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x < 4) out[threadIdx.x] = sh[threadIdx.x][0];
}

unsigned blocks_for(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

}  // namespace

#define LBM_DISPATCH_PREC(prec, S, ...)                         \
  switch (prec) {                                               \
    case kF64: { using S = double; __VA_ARGS__; break; }        \
    case kF32: { using S = float; __VA_ARGS__; break; }         \
    case kF16: { using S = __half; __VA_ARGS__; break; }        \
    case kF64DF: { using S = f64df; __VA_ARGS__; break; }       \
    case kF32DF: { using S = f32df; __VA_ARGS__; break; }       \
    case kF16SR: { using S = h16sr; __VA_ARGS__; break; }       \
    default: return cudaErrorInvalidValue;                      \
  }

cudaError_t launch_from_canonical(const LatticeView& v, Layout layout, void* dst,
                                  const double* canon, const double* rho, const double* u, cudaStream_t s) {
  const CanonSource src{canon, rho, u, v.n_cells};
  if (!canon && layout != kCanonical) {
    LBM_DISPATCH_PREC(v.prec, S,
                      k_equilibrium_push<S><<<blocks_for(v.n_cells, 256), 256, 0, s>>>(v, layout,
                                                                                       static_cast<S*>(dst), src));
  } else {
    LBM_DISPATCH_PREC(v.prec, S,
                      k_from_canonical<S><<<blocks_for(v.n_cells, 256), 256, 0, s>>>(v, layout,
                                                                                     static_cast<S*>(dst), src));
  }
  return cudaGetLastError();
}

cudaError_t launch_to_canonical(const LatticeView& v, Layout layout, const void* src,
                                double* out, cudaStream_t s) {
  LBM_DISPATCH_PREC(v.prec, S,
                    k_to_canonical<S><<<blocks_for(v.n_cells, 256), 256, 0, s>>>(v, layout,
                                                                                 static_cast<const S*>(src), out));
  return cudaGetLastError();
}

cudaError_t launch_macroscopic(const LatticeView& v, Layout layout, const void* src,
                               const double force[3], double* rho, double* u, cudaStream_t s) {
  const Force3 F{{force[0], force[1], force[2]}};
  LBM_DISPATCH_PREC(v.prec, S,
                    k_macroscopic<S><<<blocks_for(v.n_cells, 256), 256, 0, s>>>(v, layout,
                                                                                static_cast<const S*>(src), F, rho, u));
  return cudaGetLastError();
}

cudaError_t launch_profile(const LatticeView& v, Layout layout, const void* src,
                           const double force[3], int axis, int comp, double* sums, unsigned long long* counts,
                           cudaStream_t s) {
  const Force3 F{{force[0], force[1], force[2]}};
  const int planes = axis == 0 ? v.nx : (axis == 1 ? v.ny : v.nz);
  LBM_DISPATCH_PREC(v.prec, S,
                    k_profile<S><<<planes, 256, 0, s>>>(v, layout, static_cast<const S*>(src), F, axis,
                                                        comp, sums, counts));
  return cudaGetLastError();
}

int moments_blocks(const LatticeView& v) {
  return (int)blocks_for(v.n_cells, kMomThreads * kMomCellsPerThread);
}

cudaError_t launch_moments(const LatticeView& v, Layout layout, const void* src,
                           double* partials, int blocks, double* out, cudaStream_t s) {
  LBM_DISPATCH_PREC(v.prec, S,
                    k_moments_partial<S><<<blocks, kMomThreads, 0, s>>>(v, layout,
                                                                        static_cast<const S*>(src), partials));
  k_moments_final<<<1, kMomThreads, 0, s>>>(partials, blocks, out);
  return cudaGetLastError();
}

}  // namespace lbm
