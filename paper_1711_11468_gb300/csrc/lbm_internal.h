// Internal interfaces between the translation units of liblbm_gb300.so:
// the launchers each .cu file provides and the handle the C ABI manages.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <string>
#include <vector>

#include "lbm_gb300.h"

namespace lbm {

// Where the state of a lattice sits in its storage after t steps.
//   kCanonical: slot i of node x holds f_i(x, t).
//   kPullForm : slot i of node x holds f*_i(x, t-1), the post-collision value
//               that streams to x + c_i; so f_i(x, t) sits in slot i of x - c_i
//               (in slot opp(i) of x across a half-way link). Two-grid pull.
//   kAAForm   : as kPullForm, but in slot opp(i) (in slot i of x across a
//               half-way link). The AA pattern after an odd number of steps.
enum Layout : int { kCanonical = 0, kPullForm = 1, kAAForm = 2 };

enum Prec : int { kF64 = 0, kF32 = 1, kF16 = 2, kF64DF = 3, kF32DF = 4, kF16SR = 5 };

enum SweepKind : int { kPull = 0, kAAEven = 1, kAAOdd = 2 };

inline int elem_bytes(int prec) {
  return (prec == kF64 || prec == kF64DF) ? 8 : ((prec == kF32 || prec == kF32DF) ? 4 : 2);
}

// Everything a kernel needs to address one lattice's storage.
struct LatticeView {
  int nx = 0, ny = 0, nz = 0;
  int64_t n_cells = 0;    // N
  int64_t n_nodes = 0;    // N (direct) or Nf (indirect)
  int64_t stride = 0;     // elements between direction arrays, multiple of 128
  int prec = kF64;
  bool indirect = false;
  bool has_halfway = false;
  const uint8_t* flags = nullptr;     // [N]
  // Indirect only: link[(i-1)*stride + k] is the element offset (slot*stride +
  // node) the sweep reads f_i of node k from, bounce-back already resolved:
  // AA: slot opp(i) of the upstream node, or slot i of k itself across a
  // half-way link; pull: slot i of the upstream node, or slot opp(i) of k.
  const uint32_t* link = nullptr;     // [18][stride]
  const int32_t* cell_of = nullptr;   // [Nf], indirect only
  const int32_t* list_index = nullptr;  // [N] node of each cell or -1, indirect only
  int* status = nullptr;                // device status word of the handle (timeouts)
  // Indirect only, optional: the run-indexed code of `link` (lbm_ria.cu); the
  // staged list sweeps read it instead of the table when ria_head is set.
  const uint2* ria_head = nullptr;            // [chunks][18] {run-start mask, pool start}
  const uint32_t* ria_pool = nullptr;         // first link of each run
  const uint32_t* ria_chunk_start = nullptr;  // [chunks + 1] pool start of each chunk
  // FP16 stochastic format only: the lattice's seed and the handle's pair of
  // sweep counters (a sweep of parity q reads word q and writes word q ^ 1).
  unsigned long long sr_seed = 0;
  unsigned long long* sweep_ctr = nullptr;
};

struct TrtParams {
  double omega_p = 1.0, omega_m = 1.0;
  double fk[9] = {0};     // 3 w_k (c_k . F), k = 1..9
  double force[3] = {0};
};

// ------------------------------------------------------------ sweep launchers
// One time step of one lattice. src == dst for the AA kinds. cells_per_thread
// (1 or 2) applies to full arrays. parity: the step count mod 2.
cudaError_t launch_sweep(const LatticeView& v, SweepKind kind, int parity, const void* src, void* dst,
                         const TrtParams& p, int threads, int cells_per_thread, cudaStream_t s);

// Two time steps of a full-array two-grid pull lattice in one launch (temporal
// blocking, lbm_temporal.cu): src holds f(t), dst receives f(t+2). parity: the
// sweep counter word to read (the handle's buffer index). The launch shape is fixed.
cudaError_t launch_sweep_pull2(const LatticeView& v, int parity, const void* src, void* dst, const TrtParams& p,
                               cudaStream_t s);

// One time step of every lattice of a batch in one launch. d_lattices holds one
// descriptor per lattice (batch_lattice_bytes(prec) bytes each, filled by
// fill_batch_lattice); d_tiles the work list. ctas > 0: a persistent grid of
// that many CTAs strides over the tiles; ctas == 0: one CTA per tile.
struct BatchTile {
  int32_t lattice;
  int32_t count;
  int64_t first;
};
size_t batch_lattice_bytes(int prec);
void fill_batch_lattice(int prec, void* host_desc, const LatticeView& v, void* pdf_a, void* pdf_b,
                        const TrtParams& p);
cudaError_t launch_batch_sweep(int prec, SweepKind kind, const void* d_lattices, const BatchTile* d_tiles,
                               int32_t n_tiles, int threads, int ctas, int phase, unsigned long long* sweep_ctr,
                               cudaStream_t s);
// Resident CTAs of the batched kernel per SM at this block size (occupancy).
int batch_blocks_per_sm(int prec, SweepKind kind, int threads);

// ------------------------------------------------------- state conversions
// Write storage `dst` in `layout` from canonical FP64 values, which come either
// from a device array canon[19][N] (non-null) or, if canon is null, from the
// equilibrium of rho[N] / u[3][N] (either may be null: 1 / 0).
cudaError_t launch_from_canonical(const LatticeView& v, Layout layout, void* dst, const double* canon,
                                  const double* rho, const double* u, cudaStream_t s);
// Canonical FP64 out[19][N] from storage in `layout` (0 at half-way solid cells).
cudaError_t launch_to_canonical(const LatticeView& v, Layout layout, const void* src, double* out,
                                cudaStream_t s);
// rho[N], u[3][N] (either may be null) from storage in `layout`.
cudaError_t launch_macroscopic(const LatticeView& v, Layout layout, const void* src, const double force[3],
                               double* rho, double* u, cudaStream_t s);
// Per-plane sums over fluid cells of u_comp (out[n_axis]) and fluid counts
// (cnt[n_axis]); the caller divides.
cudaError_t launch_profile(const LatticeView& v, Layout layout, const void* src, const double force[3],
                           int axis, int comp, double* sums, unsigned long long* counts, cudaStream_t s);
// FP64 mass and momentum over all stored PDFs: per-block partials written to
// `partials` (4 doubles per block, `blocks` blocks), then reduced in a fixed
// order into out[4].
int moments_blocks(const LatticeView& v);
cudaError_t launch_moments(const LatticeView& v, Layout layout, const void* src, double* partials, int blocks,
                           double* out, cudaStream_t s);

// ------------------------------------------------ run-indexed adjacency (RIA)
// Chunks of 32 list nodes. Count: chunk_start[chunks + 1] receives the
// exclusive prefix of the runs per chunk and, last, the pool size (also in
// *d_total). Fill: head[chunks][18] and pool[pool size]. Verify: adds the number
// of links the code does not reproduce to *d_mismatches.
int64_t ria_chunks(int64_t nf);
cudaError_t launch_ria_count(const LatticeView& v, uint32_t* chunk_start, int64_t* d_total, cudaStream_t s);
cudaError_t launch_ria_fill(const LatticeView& v, const uint32_t* chunk_start, uint2* head, uint32_t* pool,
                            cudaStream_t s);
cudaError_t launch_ria_verify(const LatticeView& v, const uint2* head, const uint32_t* pool, uint32_t pool_entries,
                              unsigned long long* d_mismatches, cudaStream_t s);

// ------------------------------------------------------------- geometry
// Exclusive prefix sum of data[n] in place (single CTA, int64 carry); the total to *d_total.
cudaError_t launch_exclusive_scan(int32_t* data, int64_t n, int64_t* d_total, cudaStream_t s);
cudaError_t launch_voxelize_spheres(int nx, int ny, int nz, const int32_t* d_spheres, int nspheres,
                                    uint8_t value, uint8_t* d_flags, cudaStream_t s);
// Fluid compaction: list_index[N] (-1 for solid), cell_of[Nf]; block sums in
// `scan_tmp` (scan_tmp_elems(N) int32). Returns Nf through *d_nf (device).
int64_t scan_tmp_elems(int64_t n);
cudaError_t launch_compact(const uint8_t* d_flags, int64_t n, int32_t* d_list_index, int32_t* d_cell_of,
                           int32_t* scan_tmp, int64_t* d_nf, cudaStream_t s);
// The link table of an indirectly addressed lattice for the given propagation.
cudaError_t launch_links(const LatticeView& v, const int32_t* d_list_index, bool aa, uint32_t* d_link,
                         cudaStream_t s);
// Fluid cells on the boundary faces, accumulated into out[6] (zeroed by the
// caller): out[2a] on the low face of axis a, out[2a+1] on the high face.
cudaError_t launch_face_fluid(const uint8_t* d_flags, int nx, int ny, int nz, unsigned long long* d_out,
                              cudaStream_t s);
// Count link-table entries outside [0, limit) into *d_bad (zeroed by the caller).
cudaError_t launch_links_check(const LatticeView& v, uint64_t limit, unsigned long long* d_bad, cudaStream_t s);
// Count flags into out[4] (zeroed by the caller): cells with flag 0, 1, 2, other.
cudaError_t launch_count_flags(const uint8_t* d_flags, int64_t n, unsigned long long* d_out, cudaStream_t s);

// ---------------------------------------------------------- micro-benchmarks
cudaError_t launch_copy19(const void* src, void* dst, int64_t n, int64_t stride, int elem, cudaStream_t s);
cudaError_t launch_update19(void* buf, int64_t n, int64_t stride, int elem, cudaStream_t s);
// FP64 fused multiply-add throughput: blocks x 256 threads, 16 x iterations FMAs
// each; out[blocks * 256] receives the sums.
cudaError_t launch_fma64(double* out, int blocks, int iterations, cudaStream_t s);
// CTAs of the FMA probe that one wave of the whole GPU holds at once.
int fma64_wave_blocks();
// Bounded-wait self-test: sets the timeout bit of *status after `polls` polls.
cudaError_t launch_wait_selftest(uint32_t polls, int* status, cudaStream_t s);

}  // namespace lbm
