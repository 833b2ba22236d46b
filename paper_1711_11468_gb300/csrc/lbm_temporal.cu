// Temporal blocking of the full-array two-grid pull sweep: two time steps per
// pass over HBM (the paper lists temporal blocking among the optimisations its
// kernels do not cover, Sec. 3 and Sec. 6). A step reads 19 and writes 19
// values per cell, so one step per pass is bound by HBM at 2 x 19 x S bytes
// per update; two steps per pass halve that.
//
// 2.5-D wavefront: a CTA owns an in-plane region of 32 x 8 cells (one warp per
// region row) and marches along z over a segment of planes. For every plane z
// it first runs step A (t -> t+1, gathering from the source grid in HBM) on the
// whole region of plane z+1, keeping the post-collision values in a ring of
// planes in shared memory, then step B (t+1 -> t+2) on the interior
// 30 x 6 cells of plane z, gathering from the ring, and writes them to the
// destination grid. The ring values are rounded to the storage format exactly
// as a one-step sweep stores them, and both steps use the one-step sweep's
// per-node arithmetic, so the result is that of two one-step sweeps, bit for
// bit. The region's one-cell rim and the first two planes of a segment are
// computed twice (by neighbouring CTAs); their gathers mostly hit L2.
//
// The ring keeps each value only as long as step B needs it. Step B of plane z
// pulls direction i from plane z - c_z(i) and, at a half-way wall, the
// reflected direction from plane z itself; step A of plane p runs just before
// step B of plane p - 1. So a value of plane p with c_z = +1 is last read by
// step B of plane p + 1, and one with c_z = 0 or -1 by step B of plane p: the
// three z-classes need 3, 2 and 2 plane slots, 43 direction planes in all
// instead of the 57 of three whole planes, which lets more CTAs share an SM.
#include <algorithm>
#include <mutex>

#include "lbm_internal.h"
#include "lbm_sweep.cuh"

namespace lbm {
namespace {

constexpr int kTbWidth = 32;   // region width in x
constexpr int kTbRows = 8;     // region rows: one warp per row
constexpr int kTbPlane = kTbWidth * kTbRows;

// Ring layout by z-class: [c_z = -1: 5 directions x 2 slots][c_z = 0: 9 x 2][c_z = +1: 5 x 3].
constexpr int kRingPlanes = 5 * 2 + 9 * 2 + 5 * 3;
__host__ __device__ constexpr int ring_slots(int i) { return cz(i) > 0 ? 3 : 2; }
__host__ __device__ constexpr int ring_rank(int i) {   // position of i among the directions of its z-class
  int r = 0;
  for (int k = 0; k < i; ++k) r += cz(k) == cz(i) ? 1 : 0;
  return r;
}
__host__ __device__ constexpr int ring_first(int i) {   // first plane of direction i in the ring
  return (cz(i) < 0 ? 0 : cz(i) == 0 ? 5 * 2 : 5 * 2 + 9 * 2) + ring_rank(i) * ring_slots(i);
}

// Compile-time replay of a z segment's loop (step A of planes z0 - 1 and z0, then
// for each z step A of z + 1 and step B of z) on tags of the values: every slot
// index is in range and owned by one direction, and every value step B reads,
// pulled or reflected, is the one step A wrote for that plane and direction.
__host__ __device__ constexpr int ring_slot_of(int z, int i) { return ring_first(i) + (z + 6) % ring_slots(i); }
constexpr bool ring_liveness_ok() {
  int owner[kRingPlanes] = {};
  for (int i = 0; i < Q; ++i)
    for (int k = 0; k < ring_slots(i); ++k) {
      const int sl = ring_first(i) + k;
      if (sl < 0 || sl >= kRingPlanes || owner[sl] != 0) return false;
      owner[sl] = i + 1;
    }
  for (int z0 = 0; z0 < 3; ++z0) {
    int tag[kRingPlanes] = {};
    auto tag_of = [](int z, int i) { return (z + 2) * 32 + i; };
    for (int z = z0 - 1; z <= z0; ++z)
      for (int i = 0; i < Q; ++i) tag[ring_slot_of(z, i)] = tag_of(z, i);
    for (int z = z0; z < z0 + 12; ++z) {
      for (int i = 0; i < Q; ++i) tag[ring_slot_of(z + 1, i)] = tag_of(z + 1, i);
      for (int i = 0; i < Q; ++i) {
        if (tag[ring_slot_of(z - cz(i), i)] != tag_of(z - cz(i), i)) return false;
        if (tag[ring_slot_of(z, opp(i))] != tag_of(z, opp(i))) return false;
      }
    }
  }
  return true;
}
static_assert(ring_liveness_ok(), "a ring slot is overwritten before its last reader");

__device__ __forceinline__ int wrap_mod(int a, int n) {
  const int r = a % n;
  return r < 0 ? r + n : r;
}

template <typename S, bool kHW>
__global__ void __launch_bounds__(kTbPlane) k_dense_pull_tb2(const S* __restrict__ src, S* __restrict__ dst,
                                                        const uint8_t* __restrict__ flags, int nx, int ny, int nz,
                                                        int64_t stride, int seg, ParamsT<S> lp) {
  ParamsT<S> pa, pb;
  begin_two_sweeps<S>(lp, pa, pb);
  extern __shared__ __align__(16) unsigned char tb_smem[];
  const int rx = threadIdx.x, ry = threadIdx.y;
  S* const ring = reinterpret_cast<S*>(tb_smem) + ry * kTbWidth + rx;   // this thread's cell of ring plane 0
  const int x0 = blockIdx.x * (kTbWidth - 2), y0 = blockIdx.y * (kTbRows - 2);
  const int gx = wrap_mod(x0 - 1 + rx, nx), gy = wrap_mod(y0 - 1 + ry, ny);
  const int zs = blockIdx.z * seg, ze = min(zs + seg, nz);
  const bool interior = rx >= 1 && rx <= kTbWidth - 2 && ry >= 1 && ry <= kTbRows - 2 && x0 + rx - 1 < nx &&
                        y0 + ry - 1 < ny;
  // direction i of plane z (z >= -1) at offset (dx, dy) from this thread's cell
  auto at = [&](int z, int i, int dy, int dx) -> S* {
    return ring + ring_slot_of(z, i) * kTbPlane + dy * kTbWidth + dx;
  };

  // step A on this thread's region cell of plane z (z in [-1, nz], wrapped)
  auto step_a = [&](int z) {
    const int gz = wrap_mod(z, nz);
    const int n = gx + nx * (gy + ny * gz);
    const uint8_t fl = flags[n];
    if (fl == kSolidHalfway) return;   // its ring slots are never read
    RawT<S> f[Q];
    pull_dense_gather<S, kHW>(src, flags, Nbr(gx, gy, gz, nx, ny, nz), n, stride, f);
    if (fl == kSolidFullway)
      reverse(f);
    else
      Storage<S>::relax(f, pa, (uint32_t)n);
#pragma unroll
    for (int i = 0; i < Q; ++i) *at(z, i, 0, 0) = Storage<S>::pack(f[i]);
  };

  // step B on this thread's interior cell of plane z (z in [0, nz))
  auto step_b = [&](int z) {
    if (!interior) return;
    const int n = gx + nx * (gy + ny * z);
    const uint8_t fl = flags[n];
    if (fl == kSolidHalfway) return;
    const Nbr nb(gx, gy, z, nx, ny, nz);
    RawT<S> f[Q];
#pragma unroll
    for (int i = 0; i < Q; ++i) {
      if (kHW && i != 0 && flags[n + nb.up(i)] == kSolidHalfway)
        f[i] = Storage<S>::unpack(*at(z, opp(i), 0, 0));
      else
        f[i] = Storage<S>::unpack(*at(z - cz(i), i, -cy(i), -cx(i)));
    }
    if (fl == kSolidFullway)
      reverse(f);
    else
      Storage<S>::relax(f, pb, (uint32_t)n);
#pragma unroll
    for (int i = 0; i < Q; ++i) Storage<S>::store(dir(dst, i, stride) + n, f[i]);
  };

  // every thread runs the same loop (zs, ze are uniform), so the barriers match
  step_a(zs - 1);
  step_a(zs);
  for (int z = zs; z < ze; ++z) {
    step_a(z + 1);   // overwrites only slots whose last reader, step B of z - 1 or earlier, is done
    __syncthreads();
    step_b(z);
    __syncthreads();
  }
}

template <typename S>
constexpr size_t tb_smem_bytes() {
  return (size_t)kRingPlanes * kTbPlane * sizeof(S);
}
static_assert(tb_smem_bytes<double>() <= 200 * 1024, "ring of the 8-byte formats fits an SM");

template <typename S, bool kHW>
cudaError_t tb_launch(const LatticeView& v, const S* src, S* dst, const ParamsT<S>& p, cudaStream_t s) {
  static std::once_flag once;
  std::call_once(once, [] {
    cudaFuncSetAttribute(k_dense_pull_tb2<S, kHW>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)tb_smem_bytes<S>());
  });
  const size_t smem = tb_smem_bytes<S>();
  const int tiles_x = (v.nx + kTbWidth - 3) / (kTbWidth - 2);
  const int tiles_y = (v.ny + kTbRows - 3) / (kTbRows - 2);
  int dev = 0, sms = 0, per_sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_dense_pull_tb2<S, kHW>, kTbPlane, smem);
  // enough z segments for about four waves of resident CTAs, each at least 8 planes long
  const int64_t resident = (int64_t)std::max(1, sms) * std::max(1, per_sm);
  const int64_t want = (4 * resident + (int64_t)tiles_x * tiles_y - 1) / ((int64_t)tiles_x * tiles_y);
  const int segs = (int)std::max<int64_t>(1, std::min<int64_t>(want, v.nz / 8));
  const int seg = (v.nz + segs - 1) / segs;
  const dim3 grid((unsigned)tiles_x, (unsigned)tiles_y, (unsigned)((v.nz + seg - 1) / seg));
  k_dense_pull_tb2<S, kHW><<<grid, dim3(kTbWidth, kTbRows), smem, s>>>(src, dst, v.flags, v.nx, v.ny, v.nz, v.stride,
                                                                       seg, p);
  return cudaGetLastError();
}

// The region is fixed at 32 x 8 cells (256 threads), so the handle's block size does
// not apply: ring addresses are then compile-time offsets from one base per thread.
template <typename S>
cudaError_t tb_typed(const LatticeView& v, int parity, const void* src, void* dst, const TrtParams& tp,
                     cudaStream_t s) {
  const ParamsT<S> p = params_as<S>(tp, v, parity);
  if (v.has_halfway)
    return tb_launch<S, true>(v, static_cast<const S*>(src), static_cast<S*>(dst), p, s);
  return tb_launch<S, false>(v, static_cast<const S*>(src), static_cast<S*>(dst), p, s);
}

}  // namespace

cudaError_t launch_sweep_pull2(const LatticeView& v, int parity, const void* src, void* dst, const TrtParams& p,
                               cudaStream_t s) {
  if (v.indirect) return cudaErrorInvalidValue;
  switch (v.prec) {
    case kF64: return tb_typed<double>(v, parity, src, dst, p, s);
    case kF32: return tb_typed<float>(v, parity, src, dst, p, s);
    case kF16: return tb_typed<__half>(v, parity, src, dst, p, s);
    case kF64DF: return tb_typed<f64df>(v, parity, src, dst, p, s);
    case kF32DF: return tb_typed<f32df>(v, parity, src, dst, p, s);
    case kF16SR: return tb_typed<h16sr>(v, parity, src, dst, p, s);
  }
  return cudaErrorInvalidValue;
}

}  // namespace lbm
