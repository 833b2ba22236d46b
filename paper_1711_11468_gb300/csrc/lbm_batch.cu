// Batched sweep: many independent lattices (full arrays and fluid lists, each
// with its own size, geometry and TRT parameters) advance by one time step in
// a single launch. The work list is a sequence of tiles (lattice, first node,
// count); a persistent grid of CTAs strides over it, or, with ctas = 0, one CTA
// takes one tile. The per-node arithmetic is the single-lattice sweep's
// (lbm_sweep.cuh). Not in the paper: its closest analogue is the OpenMP loop
// over the fluid list (Sec. 3.1).
#include "lbm_internal.h"
#include "lbm_sweep.cuh"

namespace lbm {

namespace {

template <typename S>
struct __align__(16) BatchDesc {
  void* pdf[2];            // state grid(s): AA uses pdf[0]; pull alternates
  const uint8_t* flags;    // [N], full array only
  const uint32_t* link;    // [18][stride] element offsets, fluid list only
  int64_t stride;
  int nx, ny, nz;
  int indirect, has_halfway, small;   // small: N < 2^24 (fast coordinate split)
  float inv_nx, inv_ny;
  ParamsT<S> p;
};

// n -> (x, y, z) for a full array. For N < 2^24 the quotient through a float
// reciprocal is off by at most one and is corrected; otherwise plain division.
__device__ __forceinline__ void split_cell(int n, int nx, int ny, bool small, float inv_nx, float inv_ny, int& x,
                                           int& y, int& z) {
  int row, zz;
  if (small) {
    row = __float2int_rz(__int2float_rn(n) * inv_nx);
    int r = n - row * nx;
    while (r < 0) { --row; r += nx; }
    while (r >= nx) { ++row; r -= nx; }
    x = r;
    zz = __float2int_rz(__int2float_rn(row) * inv_ny);
    int r2 = row - zz * ny;
    while (r2 < 0) { --zz; r2 += ny; }
    while (r2 >= ny) { ++zz; r2 -= ny; }
    y = r2;
  } else {
    row = n / nx;
    x = n - row * nx;
    zz = row / ny;
    y = row - zz * ny;
  }
  z = zz;
}

// One node of a tile: the node-local parts shared by both nodes of a pair.
struct NodeRef {
  int64_t node;
  int x, y, z;
  bool live;   // false: nothing to do (solid cell, or past the end of the tile)
};

template <typename S, int KIND, typename D>
__device__ __forceinline__ NodeRef node_ref(const D& sd, int64_t node, bool in_tile) {
  NodeRef r{node, 0, 0, 0, in_tile};
  if (!in_tile || sd.indirect) return r;
  const int n = (int)node;
  const uint8_t fl = sd.flags[n];
  // AA: fluid cells only (solids are a no-op). Pull: half-way solids hold nothing;
  // full-way solids reverse their populations.
  r.live = KIND == kPull ? fl != kSolidHalfway : fl == kFluid;
  if (r.live && KIND != kAAEven) split_cell(n, sd.nx, sd.ny, sd.small, sd.inv_nx, sd.inv_ny, r.x, r.y, r.z);
  return r;
}

template <typename S, int KIND, typename D>
__device__ __forceinline__ void gather(const D& sd, int phase, const NodeRef& r, RawT<S> (&f)[Q]) {
  if (!r.live) return;
  const int64_t stride = sd.stride;
  if (KIND == kAAEven) {
    const S* pdf = static_cast<const S*>(sd.pdf[0]);
#pragma unroll
    for (int i = 0; i < Q; ++i) f[i] = Storage<S>::load(dir(pdf, i, stride) + r.node);
  } else if (sd.indirect) {
    list_gather<S>(static_cast<const S*>(sd.pdf[KIND == kPull ? phase : 0]), sd.link, r.node, stride, f);
  } else {
    const Nbr nb(r.x, r.y, r.z, sd.nx, sd.ny, sd.nz);
    const int n = (int)r.node;
    if (KIND == kPull) {
      const S* src = static_cast<const S*>(sd.pdf[phase]);
      if (sd.has_halfway) pull_dense_gather<S, true>(src, sd.flags, nb, n, stride, f);
      else pull_dense_gather<S, false>(src, sd.flags, nb, n, stride, f);
    } else {
      const S* pdf = static_cast<const S*>(sd.pdf[0]);
      if (sd.has_halfway) aa_odd_dense_gather<S, true>(pdf, sd.flags, nb, n, stride, f);
      else aa_odd_dense_gather<S, false>(pdf, sd.flags, nb, n, stride, f);
    }
  }
}

template <typename S, int KIND, typename D>
__device__ __forceinline__ void relax_scatter(const D& sd, int phase, const NodeRef& r, RawT<S> (&f)[Q]) {
  if (!r.live) return;
  const int64_t stride = sd.stride;
  if (KIND == kPull && !sd.indirect && sd.flags[(int)r.node] == kSolidFullway)
    reverse(f);
  else
    Storage<S>::relax(f, sd.p, (uint32_t)r.node);
  if (KIND == kAAEven) {
    S* pdf = static_cast<S*>(sd.pdf[0]);
#pragma unroll
    for (int i = 0; i < Q; ++i) Storage<S>::store(dir(pdf, opp(i), stride) + r.node, f[i]);
  } else if (KIND == kPull) {
    S* dst = static_cast<S*>(sd.pdf[phase ^ 1]);
#pragma unroll
    for (int i = 0; i < Q; ++i) Storage<S>::store(dir(dst, i, stride) + r.node, f[i]);
  } else if (sd.indirect) {
    list_aa_scatter<S>(static_cast<S*>(sd.pdf[0]), sd.link, r.node, stride, f);
  } else {
    const Nbr nb(r.x, r.y, r.z, sd.nx, sd.ny, sd.nz);
    S* pdf = static_cast<S*>(sd.pdf[0]);
    if (sd.has_halfway) aa_odd_dense_scatter<S, true>(pdf, sd.flags, nb, (int)r.node, stride, f);
    else aa_odd_dense_scatter<S, false>(pdf, sd.flags, nb, (int)r.node, stride, f);
  }
}

// For 4-byte raw values each thread takes its tile's nodes in pairs (j and
// j + blockDim.x) and issues both nodes' loads before colliding either: a
// node's loads cannot otherwise start before the previous node's stores, since
// both touch the same arrays.
// The stochastic format numbers the sweeps in ctr (see begin_sweep): every
// lattice of the batch is at the same sweep, and lattice l draws from its own
// seed, the handle's seed + l.
template <typename S, int KIND>
__global__ void __launch_bounds__(512) k_batch(const BatchDesc<S>* __restrict__ lat,
                                               const BatchTile* __restrict__ tiles, int ntiles, int phase,
                                               unsigned long long* ctr) {
  using D = BatchDesc<S>;
  constexpr bool kSr = std::is_same<S, h16sr>::value;
  __shared__ D sd;
  unsigned long long sweep = 0;
  if constexpr (kSr) {
    sweep = ctr[phase];
    if (blockIdx.x == 0 && threadIdx.x == 0) ctr[phase ^ 1] = sweep + 1;
  }
  for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
    const BatchTile tile = tiles[t];
    __syncthreads();   // the previous tile is done with sd
    {
      const int4* src = reinterpret_cast<const int4*>(lat + tile.lattice);
      int4* dst = reinterpret_cast<int4*>(&sd);
      for (int w = threadIdx.x; w < (int)(sizeof(D) / sizeof(int4)); w += blockDim.x) dst[w] = src[w];
    }
    __syncthreads();
    if constexpr (kSr) {
      if (threadIdx.x == 0) sd.p.base = sd.p.seed + kSplitmixGamma * (1ull + (sweep << 32));
      __syncthreads();
    }
    // pairs only where a node's 19 values fit in 19 registers (FP32 and FP16 raw values)
    constexpr bool kPairs = sizeof(RawT<S>) == 4;
    for (int j = threadIdx.x; j < tile.count; j += (kPairs ? 2 : 1) * blockDim.x) {
      const NodeRef ra = node_ref<S, KIND>(sd, tile.first + j, true);
      RawT<S> f[Q];
      if constexpr (kPairs) {
        const int jb = j + blockDim.x;
        const NodeRef rb = node_ref<S, KIND>(sd, tile.first + jb, jb < tile.count);
        RawT<S> g[Q];
        gather<S, KIND>(sd, phase, ra, f);
        gather<S, KIND>(sd, phase, rb, g);
        relax_scatter<S, KIND>(sd, phase, ra, f);
        relax_scatter<S, KIND>(sd, phase, rb, g);
      } else {
        gather<S, KIND>(sd, phase, ra, f);
        relax_scatter<S, KIND>(sd, phase, ra, f);
      }
    }
  }
}

template <typename S>
cudaError_t batch_typed(SweepKind kind, const void* d_lat, const BatchTile* d_tiles, int ntiles, int threads,
                        int ctas, int phase, unsigned long long* ctr, cudaStream_t s) {
  using D = BatchDesc<S>;
  const D* lat = static_cast<const D*>(d_lat);
  if (ntiles <= 0) return cudaSuccess;
  const unsigned grid = (unsigned)(ctas > 0 ? std::min(ctas, ntiles) : ntiles);
  switch (kind) {
    case kPull: k_batch<S, kPull><<<grid, threads, 0, s>>>(lat, d_tiles, ntiles, phase, ctr); break;
    case kAAEven: k_batch<S, kAAEven><<<grid, threads, 0, s>>>(lat, d_tiles, ntiles, phase, ctr); break;
    case kAAOdd: k_batch<S, kAAOdd><<<grid, threads, 0, s>>>(lat, d_tiles, ntiles, phase, ctr); break;
  }
  return cudaGetLastError();
}

template <typename S>
void fill_typed(void* host_desc, const LatticeView& v, void* pdf_a, void* pdf_b, const TrtParams& p) {
  using D = BatchDesc<S>;
  D d{};
  d.pdf[0] = pdf_a;
  d.pdf[1] = pdf_b;
  d.flags = v.flags;
  d.link = v.link;
  d.stride = v.stride;
  d.nx = v.nx;
  d.ny = v.ny;
  d.nz = v.nz;
  d.indirect = v.indirect ? 1 : 0;
  d.has_halfway = v.has_halfway ? 1 : 0;
  d.small = v.n_cells < (int64_t(1) << 24) ? 1 : 0;
  d.inv_nx = 1.0f / (float)v.nx;
  d.inv_ny = 1.0f / (float)v.ny;
  d.p = params_as<S>(p, v, 0);
  *static_cast<D*>(host_desc) = d;
}

}  // namespace

size_t batch_lattice_bytes(int prec) {
  switch (prec) {
    case kF64: return sizeof(BatchDesc<double>);
    case kF32: return sizeof(BatchDesc<float>);
    case kF64DF: return sizeof(BatchDesc<f64df>);
    case kF32DF: return sizeof(BatchDesc<f32df>);
    case kF16SR: return sizeof(BatchDesc<h16sr>);
    default: return sizeof(BatchDesc<__half>);
  }
}

void fill_batch_lattice(int prec, void* host_desc, const LatticeView& v, void* pdf_a, void* pdf_b,
                        const TrtParams& p) {
  switch (prec) {
    case kF64: fill_typed<double>(host_desc, v, pdf_a, pdf_b, p); break;
    case kF32: fill_typed<float>(host_desc, v, pdf_a, pdf_b, p); break;
    case kF64DF: fill_typed<f64df>(host_desc, v, pdf_a, pdf_b, p); break;
    case kF32DF: fill_typed<f32df>(host_desc, v, pdf_a, pdf_b, p); break;
    case kF16SR: fill_typed<h16sr>(host_desc, v, pdf_a, pdf_b, p); break;
    default: fill_typed<__half>(host_desc, v, pdf_a, pdf_b, p); break;
  }
}

int batch_blocks_per_sm(int prec, SweepKind kind, int threads) {
  int n = 0;
  cudaError_t e = cudaSuccess;
#define LBM_OCC(S)                                                                                      \
  switch (kind) {                                                                                       \
    case kPull: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_batch<S, kPull>, threads, 0); break; \
    case kAAEven: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_batch<S, kAAEven>, threads, 0); break; \
    case kAAOdd: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_batch<S, kAAOdd>, threads, 0); break; \
  }
  if (prec == kF64) { LBM_OCC(double) } else if (prec == kF32) { LBM_OCC(float) }
  else if (prec == kF64DF) { LBM_OCC(f64df) } else if (prec == kF32DF) { LBM_OCC(f32df) }
  else if (prec == kF16SR) { LBM_OCC(h16sr) } else { LBM_OCC(__half) }
#undef LBM_OCC
  return e == cudaSuccess && n > 0 ? n : 1;
}

cudaError_t launch_batch_sweep(int prec, SweepKind kind, const void* d_lattices, const BatchTile* d_tiles,
                               int32_t n_tiles, int threads, int ctas, int phase, unsigned long long* ctr,
                               cudaStream_t s) {
  switch (prec) {
    case kF64: return batch_typed<double>(kind, d_lattices, d_tiles, n_tiles, threads, ctas, phase, ctr, s);
    case kF32: return batch_typed<float>(kind, d_lattices, d_tiles, n_tiles, threads, ctas, phase, ctr, s);
    case kF16: return batch_typed<__half>(kind, d_lattices, d_tiles, n_tiles, threads, ctas, phase, ctr, s);
    case kF64DF: return batch_typed<f64df>(kind, d_lattices, d_tiles, n_tiles, threads, ctas, phase, ctr, s);
    case kF32DF: return batch_typed<f32df>(kind, d_lattices, d_tiles, n_tiles, threads, ctas, phase, ctr, s);
    case kF16SR: return batch_typed<h16sr>(kind, d_lattices, d_tiles, n_tiles, threads, ctas, phase, ctr, s);
  }
  return cudaErrorInvalidValue;
}

}  // namespace lbm
