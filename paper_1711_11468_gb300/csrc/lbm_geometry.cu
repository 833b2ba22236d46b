// Geometry set-up on the device: sphere voxelisation, fluid-list compaction and
// the adjacency list (Sec. 3 "Lattice Representation": fluid nodes in a 1-D
// vector plus an adjacency list of 18 int32 neighbours per node, Table 1).
// All of it is integer work and bit-exact.
#include "lbm_internal.h"
#include "lbm_model.cuh"

namespace lbm {
namespace {

// Minimum-image offset of a along a periodic axis of length n (|result| <= n/2).
__device__ __forceinline__ int min_image(int a, int n) {
  int r = a % n;
  if (r < 0) r += n;
  if (2 * r > n) r -= n;
  return r;
}

// One block per sphere: visit the cells of its bounding box (the whole axis
// when the box would wrap onto itself) and mark those inside.
__global__ void k_voxelize(int nx, int ny, int nz, const int32_t* __restrict__ sph, uint8_t value,
                           uint8_t* __restrict__ flags) {
  const int s = blockIdx.x;
  const int cxs = sph[4 * s + 0], cys = sph[4 * s + 1], czs = sph[4 * s + 2], r = sph[4 * s + 3];
  const int64_t r2 = (int64_t)r * r;
  const bool fx = 2 * r + 1 >= nx, fy = 2 * r + 1 >= ny, fz = 2 * r + 1 >= nz;
  const int ex = fx ? nx : 2 * r + 1, ey = fy ? ny : 2 * r + 1, ez = fz ? nz : 2 * r + 1;
  const int64_t total = (int64_t)ex * ey * ez;
  for (int64_t t = threadIdx.x; t < total; t += blockDim.x) {
    const int ox = (int)(t % ex);
    const int64_t rest = t / ex;
    const int oy = (int)(rest % ey), oz = (int)(rest / ey);
    int x = fx ? ox : cxs - r + ox;
    int y = fy ? oy : cys - r + oy;
    int z = fz ? oz : czs - r + oz;
    x %= nx; if (x < 0) x += nx;
    y %= ny; if (y < 0) y += ny;
    z %= nz; if (z < 0) z += nz;
    const int64_t dx = min_image(x - cxs, nx), dy = min_image(y - cys, ny), dz = min_image(z - czs, nz);
    if (dx * dx + dy * dy + dz * dz <= r2) flags[(int64_t)x + (int64_t)nx * ((int64_t)y + (int64_t)ny * z)] = value;
  }
}

constexpr int kScanThreads = 1024;
constexpr int kScanItems = 8;
constexpr int64_t kScanTile = (int64_t)kScanThreads * kScanItems;

// Exclusive block-wide scan of one int per thread; returns the block total.
__device__ int block_exclusive_scan(int v, int& total) {
  __shared__ int warp_sums[kScanThreads / 32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int incl = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int t = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += t;
  }
  if (lane == 31) warp_sums[warp] = incl;
  __syncthreads();
  if (warp == 0) {
    int w = lane < kScanThreads / 32 ? warp_sums[lane] : 0;
    int wi = w;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int t = __shfl_up_sync(0xffffffffu, wi, o);
      if (lane >= o) wi += t;
    }
    if (lane < kScanThreads / 32) warp_sums[lane] = wi - w;  // exclusive warp offsets
  }
  __syncthreads();
  const int excl = warp_sums[warp] + incl - v;
  // block total = exclusive offset of the last warp + its inclusive sum
  __shared__ int tot;
  if (threadIdx.x == kScanThreads - 1) tot = excl + v;
  __syncthreads();
  total = tot;
  __syncthreads();
  return excl;
}

__global__ void __launch_bounds__(kScanThreads) k_count_fluid(const uint8_t* __restrict__ flags, int64_t n,
                                                              int32_t* __restrict__ tile_counts) {
  const int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
  int c = 0;
#pragma unroll
  for (int j = 0; j < kScanItems; ++j) c += (base + j < n && flags[base + j] == kFluid) ? 1 : 0;
  int total;
  block_exclusive_scan(c, total);
  if (threadIdx.x == 0) tile_counts[blockIdx.x] = total;
}

// Single block: exclusive scan of the tile counts in place, total to *nf.
__global__ void __launch_bounds__(kScanThreads) k_scan_tiles(int32_t* __restrict__ tile_counts, int64_t tiles,
                                                             int64_t* __restrict__ nf) {
  __shared__ int64_t carry;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  for (int64_t b = 0; b < tiles; b += kScanThreads) {
    const int64_t i = b + threadIdx.x;
    const int v = i < tiles ? tile_counts[i] : 0;
    int total;
    const int excl = block_exclusive_scan(v, total);
    if (i < tiles) tile_counts[i] = (int32_t)(carry + excl);
    __syncthreads();
    if (threadIdx.x == 0) carry += total;
    __syncthreads();
  }
  if (threadIdx.x == 0) *nf = carry;
}

__global__ void __launch_bounds__(kScanThreads) k_compact(const uint8_t* __restrict__ flags, int64_t n,
                                                          const int32_t* __restrict__ tile_offsets,
                                                          int32_t* __restrict__ list_index,
                                                          int32_t* __restrict__ cell_of) {
  const int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
  int c = 0;
#pragma unroll
  for (int j = 0; j < kScanItems; ++j) c += (base + j < n && flags[base + j] == kFluid) ? 1 : 0;
  int total;
  int k = tile_offsets[blockIdx.x] + block_exclusive_scan(c, total);
#pragma unroll
  for (int j = 0; j < kScanItems; ++j) {
    const int64_t cell = base + j;
    if (cell >= n) break;
    if (flags[cell] == kFluid) {
      list_index[cell] = k;
      cell_of[k] = (int32_t)cell;
      ++k;
    } else {
      list_index[cell] = -1;
    }
  }
}

// For list node k and direction i: the upstream node a = x_k - c_i (wrapped)
// or -1 if that cell is solid, turned into the element offset the sweep reads
// f_i from (AA: slot opp(i) of a, or slot i of k; pull: slot i of a, or slot
// opp(i) of k). The scatter of the AA odd step writes f*_i where f_opp(i) was
// read, so one table serves both directions.
__global__ void k_links(int nx, int ny, int nz, int64_t nf, int64_t stride, const int32_t* __restrict__ cell_of,
                        const int32_t* __restrict__ list_index, bool aa, uint32_t* __restrict__ link) {
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= nf) return;
  const int64_t n = cell_of[k];
  const int64_t row = n / nx;
  const int x = (int)(n - row * nx);
  const int z = (int)(row / ny);
  const int y = (int)(row - (int64_t)z * ny);
#pragma unroll
  for (int i = 1; i < Q; ++i) {
    int ux = x - cx(i), uy = y - cy(i), uz = z - cz(i);
    ux = ux < 0 ? ux + nx : (ux >= nx ? ux - nx : ux);
    uy = uy < 0 ? uy + ny : (uy >= ny ? uy - ny : uy);
    uz = uz < 0 ? uz + nz : (uz >= nz ? uz - nz : uz);
    const int32_t a = list_index[(int64_t)ux + (int64_t)nx * ((int64_t)uy + (int64_t)ny * uz)];
    const int64_t off = a >= 0 ? (int64_t)(aa ? opp(i) : i) * stride + a : (int64_t)(aa ? i : opp(i)) * stride + k;
    link[(int64_t)(i - 1) * stride + k] = (uint32_t)off;
  }
}

// Every link must address an element of the 19 direction arrays.
__global__ void k_links_check(const uint32_t* __restrict__ link, int64_t nf, int64_t stride, uint64_t limit,
                              unsigned long long* __restrict__ bad) {
  unsigned long long c = 0;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < 18 * nf; t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = t / nf, k = t - i * nf;
    c += (uint64_t)link[i * stride + k] >= limit;
  }
  if (c) atomicAdd(bad, c);
}

// Fluid cells on each boundary face: out[2a] on the low face of axis a, out[2a+1] on the high one.
__global__ void k_face_fluid(const uint8_t* __restrict__ flags, int nx, int ny, int nz,
                             unsigned long long* __restrict__ out) {
  const int face = blockIdx.y;       // 0..5
  const int axis = face >> 1;
  const int n0 = axis == 0 ? ny : nx, n1 = axis == 2 ? ny : nz;
  const int level = (face & 1) ? (axis == 0 ? nx : (axis == 1 ? ny : nz)) - 1 : 0;
  const int64_t cells = (int64_t)n0 * n1;
  unsigned long long c = 0;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < cells; t += (int64_t)gridDim.x * blockDim.x) {
    const int a = (int)(t % n0), b = (int)(t / n0);
    int x, y, z;
    if (axis == 0) { x = level; y = a; z = b; }
    else if (axis == 1) { x = a; y = level; z = b; }
    else { x = a; y = b; z = level; }
    c += flags[(int64_t)x + (int64_t)nx * ((int64_t)y + (int64_t)ny * z)] == kFluid;
  }
  if (c) atomicAdd(out + face, c);
}

// Counts of flag values 0, 1, 2 and anything else into out[0..3]. Four flags
// per 32-bit load, counters in registers, then a warp sum and one atomic per
// block and value (blockDim.x a multiple of 32: every lane reaches the sums).
__device__ __forceinline__ void count_flag(uint32_t f, uint32_t& c0, uint32_t& c1, uint32_t& c2, uint32_t& c3) {
  c0 += f == 0u;
  c1 += f == 1u;
  c2 += f == 2u;
  c3 += f > 2u;
}

__global__ void k_count_flags(const uint8_t* __restrict__ flags, int64_t n, unsigned long long* __restrict__ out) {
  uint32_t c0 = 0, c1 = 0, c2 = 0, c3 = 0;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const int64_t first = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  // bytes before the first 4-byte boundary, whole words, bytes after them
  const uint32_t mis = (uint32_t)(reinterpret_cast<uintptr_t>(flags) & 3u);
  const int64_t head = mis ? (n < (int64_t)(4u - mis) ? n : (int64_t)(4u - mis)) : 0;
  const int64_t words = (n - head) >> 2;
  const uint32_t* w = reinterpret_cast<const uint32_t*>(flags + head);
  for (int64_t t = first; t < words; t += stride) {
    const uint32_t v = w[t];
#pragma unroll
    for (int b = 0; b < 4; ++b) count_flag((v >> (8 * b)) & 0xFFu, c0, c1, c2, c3);
  }
  const int64_t tail = head + 4 * words;
  if (first < head) count_flag(flags[first], c0, c1, c2, c3);
  for (int64_t t = tail + first; t < n; t += stride) count_flag(flags[t], c0, c1, c2, c3);
  c0 = __reduce_add_sync(0xFFFFFFFFu, c0);
  c1 = __reduce_add_sync(0xFFFFFFFFu, c1);
  c2 = __reduce_add_sync(0xFFFFFFFFu, c2);
  c3 = __reduce_add_sync(0xFFFFFFFFu, c3);
  __shared__ unsigned long long sum[4];
  if (threadIdx.x < 4) sum[threadIdx.x] = 0;
  __syncthreads();
  if ((threadIdx.x & 31u) == 0) {
    atomicAdd(&sum[0], (unsigned long long)c0);
    atomicAdd(&sum[1], (unsigned long long)c1);
    atomicAdd(&sum[2], (unsigned long long)c2);
    atomicAdd(&sum[3], (unsigned long long)c3);
  }
  __syncthreads();
  if (threadIdx.x < 4 && sum[threadIdx.x]) atomicAdd(out + threadIdx.x, sum[threadIdx.x]);
}

}  // namespace

cudaError_t launch_voxelize_spheres(int nx, int ny, int nz, const int32_t* d_spheres, int nspheres, uint8_t value,
                                    uint8_t* d_flags, cudaStream_t s) {
  if (nspheres > 0) k_voxelize<<<nspheres, 256, 0, s>>>(nx, ny, nz, d_spheres, value, d_flags);
  return cudaGetLastError();
}

int64_t scan_tmp_elems(int64_t n) { return (n + kScanTile - 1) / kScanTile + 1; }

cudaError_t launch_compact(const uint8_t* d_flags, int64_t n, int32_t* d_list_index, int32_t* d_cell_of,
                           int32_t* scan_tmp, int64_t* d_nf, cudaStream_t s) {
  const int64_t tiles = (n + kScanTile - 1) / kScanTile;
  k_count_fluid<<<(unsigned)tiles, kScanThreads, 0, s>>>(d_flags, n, scan_tmp);
  k_scan_tiles<<<1, kScanThreads, 0, s>>>(scan_tmp, tiles, d_nf);
  k_compact<<<(unsigned)tiles, kScanThreads, 0, s>>>(d_flags, n, scan_tmp, d_list_index, d_cell_of);
  return cudaGetLastError();
}

cudaError_t launch_exclusive_scan(int32_t* data, int64_t n, int64_t* d_total, cudaStream_t s) {
  k_scan_tiles<<<1, kScanThreads, 0, s>>>(data, n, d_total);
  return cudaGetLastError();
}

cudaError_t launch_links(const LatticeView& v, const int32_t* d_list_index, bool aa, uint32_t* d_link,
                         cudaStream_t s) {
  if (v.n_nodes == 0) return cudaSuccess;
  k_links<<<(unsigned)((v.n_nodes + 255) / 256), 256, 0, s>>>(v.nx, v.ny, v.nz, v.n_nodes, v.stride, v.cell_of,
                                                             d_list_index, aa, d_link);
  return cudaGetLastError();
}

cudaError_t launch_links_check(const LatticeView& v, uint64_t limit, unsigned long long* d_bad, cudaStream_t s) {
  if (v.n_nodes == 0) return cudaSuccess;
  const int64_t blocks = std::min<int64_t>((18 * v.n_nodes + 255) / 256, 4096);
  k_links_check<<<(unsigned)blocks, 256, 0, s>>>(v.link, v.n_nodes, v.stride, limit, d_bad);
  return cudaGetLastError();
}

cudaError_t launch_face_fluid(const uint8_t* d_flags, int nx, int ny, int nz, unsigned long long* d_out,
                              cudaStream_t s) {
  k_face_fluid<<<dim3(64, 6), 256, 0, s>>>(d_flags, nx, ny, nz, d_out);
  return cudaGetLastError();
}

cudaError_t launch_count_flags(const uint8_t* d_flags, int64_t n, unsigned long long* d_out, cudaStream_t s) {
  const int64_t blocks = std::min<int64_t>((n + 255) / 256, 4096);
  k_count_flags<<<(unsigned)blocks, 256, 0, s>>>(d_flags, n, d_out);
  return cudaGetLastError();
}

}  // namespace lbm
