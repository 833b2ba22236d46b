// Reduced indirect addressing (RIA) of fluid-list lattices: a run-length code
// of the link table (Sec. 3 "AA Pattern Kernels": consecutive nodes that share
// one access pattern need no lookup of their own), laid out for warps.
//
// The list is cut into chunks of 32 consecutive nodes, one warp's worth. For
// chunk c and direction i, a run is a maximal range of the chunk's nodes whose
// links increase by one from node to node (the neighbours are consecutive list
// nodes, or all of them bounce back into their own slots). The code stores
//   head[c][i-1] = {mask, start}: bit j of mask is set when node 32c + j begins
//                  a run; start is the pool index of the chunk's first run in
//                  direction i;
//   pool[start + r] = the link of the first node of run r;
//   chunk_start[c]  = the pool index of chunk c's first run (direction 1);
//                  chunk_start[chunks] = the pool size.
// Lane j recovers its link as pool[start + popc(mask & le) - 1] + (j - first),
// with le the lanes 0..j and first the highest run start at or below j. Regular
// geometry needs one header of 144 bytes per 32 nodes and a few pool entries
// instead of 18 x 128 bytes of links.
#include "lbm_internal.h"
#include "lbm_model.cuh"

namespace lbm {
namespace {

constexpr unsigned kFullMask = 0xffffffffu;

// The mask of lanes of this warp that start a run in direction i; l receives
// the lane's link (0 past the end of the list).
__device__ __forceinline__ unsigned run_starts(const uint32_t* __restrict__ link, int64_t stride, int64_t nf,
                                               int64_t k, int i, int lane, uint32_t& l) {
  const bool live = k < nf;
  l = live ? __ldg(link + (int64_t)(i - 1) * stride + k) : 0u;
  const uint32_t prev = __shfl_up_sync(kFullMask, l, 1);
  return __ballot_sync(kFullMask, live && (lane == 0 || l != prev + 1u));
}

// One warp per chunk (the grid covers whole warps, so a warp exits as a whole).
__global__ void k_ria_count(const uint32_t* __restrict__ link, int64_t stride, int64_t nf, int64_t chunks,
                            uint32_t* __restrict__ chunk_runs) {
  const int64_t c = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (c >= chunks) return;
  const int64_t k = c * 32 + lane;
  unsigned runs = 0;
  for (int i = 1; i < Q; ++i) {
    uint32_t l;
    runs += __popc(run_starts(link, stride, nf, k, i, lane, l));
  }
  if (lane == 0) chunk_runs[c] = runs;
}

__global__ void k_ria_fill(const uint32_t* __restrict__ link, int64_t stride, int64_t nf, int64_t chunks,
                           const uint32_t* __restrict__ chunk_start, uint2* __restrict__ head,
                           uint32_t* __restrict__ pool) {
  const int64_t c = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (c >= chunks) return;
  const int64_t k = c * 32 + lane;
  const unsigned lt = (1u << lane) - 1u;
  uint32_t p = chunk_start[c];
  for (int i = 1; i < Q; ++i) {
    uint32_t l;
    const unsigned m = run_starts(link, stride, nf, k, i, lane, l);
    if (lane == 0) head[c * (Q - 1) + (i - 1)] = make_uint2(m, p);
    if ((m >> lane) & 1u) pool[p + __popc(m & lt)] = l;
    p += __popc(m);
  }
}

__global__ void k_store_total(uint32_t* __restrict__ dst, const int64_t* __restrict__ total) {
  *dst = (uint32_t)*total;
}

// Decode every link through the code and compare with the table; indices are
// bounds-checked, so a broken code is reported rather than followed.
__global__ void k_ria_verify(const uint32_t* __restrict__ link, int64_t stride, int64_t nf, const uint2* __restrict__ head,
                             const uint32_t* __restrict__ pool, uint32_t pool_entries,
                             unsigned long long* __restrict__ mismatches) {
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= nf) return;
  const int64_t c = k >> 5;
  const int lane = (int)(k & 31);
  const unsigned le = (2u << lane) - 1u;
  unsigned bad = 0;
  for (int i = 1; i < Q; ++i) {
    const uint2 h = head[c * (Q - 1) + (i - 1)];
    const unsigned below = h.x & le;
    if (below == 0) {
      ++bad;
      continue;
    }
    const uint32_t idx = h.y + (uint32_t)__popc(below) - 1u;
    if (idx >= pool_entries) {
      ++bad;
      continue;
    }
    const uint32_t first = 31u - (uint32_t)__clz(below);
    if (pool[idx] + ((uint32_t)lane - first) != link[(int64_t)(i - 1) * stride + k]) ++bad;
  }
  if (bad) atomicAdd(mismatches, (unsigned long long)bad);
}

}  // namespace

int64_t ria_chunks(int64_t nf) { return (nf + 31) / 32; }

cudaError_t launch_ria_count(const LatticeView& v, uint32_t* chunk_start, int64_t* d_total, cudaStream_t s) {
  const int64_t chunks = ria_chunks(v.n_nodes);
  if (chunks == 0) return cudaSuccess;
  const unsigned blocks = (unsigned)((chunks * 32 + 255) / 256);
  k_ria_count<<<blocks, 256, 0, s>>>(v.link, v.stride, v.n_nodes, chunks, chunk_start);
  cudaError_t e = launch_exclusive_scan(reinterpret_cast<int32_t*>(chunk_start), chunks, d_total, s);
  if (e != cudaSuccess) return e;
  k_store_total<<<1, 1, 0, s>>>(chunk_start + chunks, d_total);
  return cudaGetLastError();
}

cudaError_t launch_ria_fill(const LatticeView& v, const uint32_t* chunk_start, uint2* head, uint32_t* pool,
                            cudaStream_t s) {
  const int64_t chunks = ria_chunks(v.n_nodes);
  if (chunks == 0) return cudaSuccess;
  const unsigned blocks = (unsigned)((chunks * 32 + 255) / 256);
  k_ria_fill<<<blocks, 256, 0, s>>>(v.link, v.stride, v.n_nodes, chunks, chunk_start, head, pool);
  return cudaGetLastError();
}

cudaError_t launch_ria_verify(const LatticeView& v, const uint2* head, const uint32_t* pool, uint32_t pool_entries,
                              unsigned long long* d_mismatches, cudaStream_t s) {
  if (v.n_nodes == 0) return cudaSuccess;
  k_ria_verify<<<(unsigned)((v.n_nodes + 255) / 256), 256, 0, s>>>(v.link, v.stride, v.n_nodes, head, pool,
                                                                   pool_entries, d_mismatches);
  return cudaGetLastError();
}

}  // namespace lbm
