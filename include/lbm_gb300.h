/*
 * lbm_gb300.h -- C ABI of the GB300 (sm_103a) D3Q19 TRT lattice Boltzmann sweep.
 *
 * The method is the fused collide-and-propagate sweep of Wittmann et al.,
 * "Lattice Boltzmann Benchmark Kernels as a Testbed for Performance Analysis"
 * (arXiv 1711.11468): D3Q19 velocities with the two-relaxation-time (TRT)
 * collision (Sec. 2), half-way or full-way bounce-back (Sec. 2, Sec. 3.2),
 * full-array (direct) or fluid-list (indirect, adjacency list) addressing
 * (Sec. 3 "Lattice Representation"), structure-of-arrays layout (Sec. 3 "Data
 * Layout"), and two-grid one-step pull or in-place AA-pattern propagation
 * (Sec. 3 "One Step Kernels", "AA Pattern Kernels"). The body force is the
 * paper's verification set-up (Sec. 2.1).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  - Every call returns an lbm_status. Nothing throws or aborts across the ABI.
 *    lbm_last_error() gives a thread-local message for the last failure.
 *  - Host pointers are owned by the caller and are only read or written during
 *    the call. Device memory is owned by the library: it is allocated through
 *    the hook set by lbm_set_allocator (default: cudaMalloc/cudaFree) and freed
 *    by lbm_destroy.
 *  - Work is issued on the CUDA stream given at creation (NULL = the legacy
 *    default stream). lbm_step is asynchronous; every lbm_read_* call and
 *    lbm_synchronize wait for that stream before returning.
 *  - A CUDA error observed by any call poisons the handle: that call and every
 *    later one on the handle return LBM_ERR_CUDA.
 *  - Order: create -> set_geometry -> set_params -> init_equilibrium (or
 *    write_pdfs) -> step / read. Out-of-order calls return LBM_ERR_STATE.
 *
 * Lattice conventions
 * -------------------
 *  - Cell index n = x + nx*(y + ny*z), x fastest; N = nx*ny*nz.
 *  - Direction order i = 0..18 (every array indexed by direction uses it):
 *      0 rest; 1..9 = (1,0,0) (0,1,0) (0,0,1) (1,1,0) (1,-1,0) (1,0,1)
 *      (1,0,-1) (0,1,1) (0,1,-1); 10..18 = the negatives of 1..9, so the
 *      opposite of i is i+9 for 1<=i<=9. Weights 1/3, 1/18 (faces), 1/36 (edges).
 *  - Flags (uint8 per cell): 0 fluid; 1 full-way bounce-back solid (holds PDFs
 *    and reverses them instead of colliding; direct addressing only);
 *    2 half-way bounce-back solid (holds nothing; a link into it reflects at
 *    mid-link).
 *  - Index arithmetic wraps in every dimension. A dimension whose periodic flag
 *    is 0 must be closed by solid cells on both boundary layers, so that no
 *    fluid population ever wraps; otherwise set_geometry returns LBM_ERR_ARG.
 *  - Canonical PDFs are f_i(x, t): post-streaming, pre-collision, FP64, laid
 *    out double[19][N]. Half-way solid cells read as 0. Reads and writes are
 *    canonical whatever the storage precision, addressing or AA parity.
 */
#ifndef LBM_GB300_H
#define LBM_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct lbm_lattice_s* lbm_handle;

typedef enum {
  LBM_OK = 0,
  LBM_ERR_ARG = 1,          /* invalid argument (NULL, size, range, geometry) */
  LBM_ERR_STATE = 2,        /* call out of order, or handle poisoned by misuse */
  LBM_ERR_OOM = 3,          /* the allocator returned NULL */
  LBM_ERR_CUDA = 4,         /* a CUDA call failed; the handle is poisoned */
  LBM_ERR_UNSUPPORTED = 5,  /* valid request this build does not serve */
  LBM_ERR_TIMEOUT = 6       /* a bounded device-side wait gave up (copies that never landed) */
} lbm_status;

/* PDF storage and collision arithmetic. The paper stores FP64 only (Sec. 2);
 * the other formats are additions.
 *   LBM_F64              FP64 values, FP64 collision (1/rho from an FP32
 *                        reciprocal refined by one FP64 Newton step: relative
 *                        error about 2^-44, on terms below 1e-3 of the PDFs).
 *   LBM_F32_SHIFTED      the deviation f_i - w_i from the rest state in FP32
 *                        (round to nearest even), FP32 collision.
 *   LBM_F16_SHIFTED      the same deviation in FP16, FP32 collision.
 *   LBM_F64_DOUBLE_FLOAT FP64 values; the collision runs on f_i - w_i in
 *                        double-float arithmetic (pairs of FP32, about 48
 *                        significant bits) and its increment is added to the
 *                        stored FP64 value. For GPUs whose FP64 units are few.
 *   LBM_F32_SHIFTED_DOUBLE_FLOAT
 *                        f_i - w_i in FP32, collided in double-float and rounded
 *                        once when stored: FP32 bytes, with the accuracy that
 *                        FP32 collision arithmetic loses.
 *   LBM_F16_SHIFTED_STOCHASTIC
 *                        2^14 (f_i - w_i) in FP16, FP32 collision, rounded to
 *                        FP16 stochastically. Round-to-nearest FP16 loses every
 *                        per-step change below half an FP16 spacing (a slow
 *                        forced flow stagnates); stochastic rounding keeps them
 *                        on average. The scale puts |f_i - w_i| from 2^-28 to 4
 *                        in FP16's normal range (larger values saturate), where
 *                        the rounding is: add 13 random bits r to the bit
 *                        pattern of the FP32 value and truncate to FP16, i.e.
 *                        round away from zero with probability equal to the
 *                        remainder over the FP16 spacing, exactly. The bits come
 *                        from a counter-based splitmix64 (Steele, Lea and Flood,
 *                        OOPSLA 2014): node k (the cell index, or the list index
 *                        under indirect addressing) at sweep t draws key
 *                        K = output number (t << 32) | k of the stream seeded
 *                        with the lattice's seed, then outputs 0..3 of the stream
 *                        seeded with K; with W_0 = K and W_m those outputs,
 *                        direction j reads the 32-bit half (j mod 4) div 2 of
 *                        W_(j div 4) (0 = low) and takes its bits 0..12 for even
 *                        j, 19..31 for odd j. Results do not depend on the launch
 *                        shape, the propagation pattern or graph replay. The seed
 *                        and the sweep number are set by
 *                        lbm_set_stochastic_rounding. */
typedef enum {
  LBM_F64 = 0,
  LBM_F32_SHIFTED = 1,
  LBM_F16_SHIFTED = 2,
  LBM_F64_DOUBLE_FLOAT = 3,
  LBM_F32_SHIFTED_DOUBLE_FLOAT = 4,
  LBM_F16_SHIFTED_STOCHASTIC = 5
} lbm_precision;

/* Full array with flag field (direct) or fluid list + int32 adjacency list
 * with 18 neighbours per node (indirect), Sec. 3 "Lattice Representation". */
typedef enum { LBM_DIRECT = 0, LBM_INDIRECT = 1 } lbm_addressing;

/* One-step pull with two grids (Sec. 3 "One Step Kernels") or the AA pattern
 * on one grid, alternating a node-local even step and a neighbour-accessing
 * odd step (Sec. 3 "AA Pattern Kernels"). */
typedef enum { LBM_PULL_TWO_GRID = 0, LBM_AA_INPLACE = 1 } lbm_propagation;

typedef struct {
  int32_t nx, ny, nz;     /* each >= 2 */
  uint8_t periodic[3];    /* 1 = periodic; 0 = closed by solid layers (see above) */
  uint8_t reserved;       /* must be 0 */
  int32_t precision;      /* lbm_precision */
  int32_t addressing;     /* lbm_addressing */
  int32_t propagation;    /* lbm_propagation */
} lbm_desc;

/* Device allocator hook, process-wide, used by handles created afterwards.
 * alloc(bytes, ctx) returns a device pointer or NULL; free_(ptr, ctx).
 * Passing alloc == free_ == NULL restores cudaMalloc/cudaFree. No counterpart
 * in the paper (its closest concern is how the lattice and adjacency list are
 * allocated, with huge pages, Sec. 2.2 "Huge Pages"); the hook lets the caller
 * own device memory. LBM_ERR_ARG if exactly one of alloc and free_ is NULL. */
typedef void* (*lbm_alloc_fn)(size_t bytes, void* ctx);
typedef void (*lbm_free_fn)(void* ptr, void* ctx);
int lbm_set_allocator(lbm_alloc_fn alloc, lbm_free_fn free_, void* ctx);

/* Create one lattice (Sec. 3: representation, layout and propagation chosen
 * per kernel, Table 1). cuda_stream is a cudaStream_t or NULL. Allocates the
 * flag field now; PDF storage is allocated by set_geometry (its size depends on
 * the fluid count for indirect addressing). *out receives the handle. */
int lbm_create_lattice(const lbm_desc* desc, void* cuda_stream, lbm_handle* out);

/* Create a batch of `count` independent lattices (1 <= count <= 65536) that
 * advance together: every lbm_step is one launch per time step covering all
 * of them (a work list of tiles over all lattices). All descriptors must share
 * precision and propagation; addressing may differ per lattice. Lattice k of a
 * batch is addressed by `lattice` = k in the calls below. Not in the paper. */
int lbm_create_batch(const lbm_desc* descs, int32_t count, void* cuda_stream, lbm_handle* out);

/* Set the geometry of lattice `lattice` from host flags uint8[N] (values 0, 1
 * or 2; 1 is rejected for indirect addressing, which stores fluid cells only).
 * Sec. 3 "Lattice Representation": the marker-and-cell full array with its
 * flag field (direct addressing), or only the fluid nodes in a 1-D vector with
 * an adjacency list (indirect addressing); the bounce-back kinds of the flags
 * are those of Sec. 2 and Sec. 3.2. Builds, on the device, the fluid list in
 * lexicographic order and the adjacency list (indirect), and allocates PDF
 * storage. LBM_ERR_ARG for a flag value above 2, flag 1 on an indirect
 * lattice, or an open non-periodic face; LBM_ERR_OOM if the allocator fails.
 * Synchronous. */
int lbm_set_geometry(lbm_handle h, int32_t lattice, const uint8_t* flags);

/* Set the geometry to fluid everywhere except the cells inside the given
 * spheres, which become half-way solid (flag 2). cxyzr is int32[4*nspheres]:
 * centre x, y, z and radius r >= 0; a cell is inside when
 * dx^2 + dy^2 + dz^2 <= r^2 with minimum-image periodic offsets. The
 * voxelisation runs on the device (the paper's heterogeneous geometries,
 * Sec. 2 and Sec. 4.5, realised as a porous medium). Synchronous. */
int lbm_set_geometry_spheres(lbm_handle h, int32_t lattice, const int32_t* cxyzr, int32_t nspheres);

/* TRT parameters (Sec. 2): omega in (0, 2) is omega+ (viscosity
 * nu = (1/omega - 1/2)/3); Lambda > 0 is the magic parameter
 * (1/omega+ - 1/2)(1/omega- - 1/2); force[3] is the constant body force of the
 * verification set-up (Sec. 2.1), applied on every fluid node as the source
 * 3 w_i (c_i . F) after collision. lattice = -1 sets every lattice. */
int lbm_set_params(lbm_handle h, int32_t lattice, double omega, double Lambda, const double force[3]);

/* Initial state f_i(x, 0) = equilibrium(rho(x), u(x)) at fluid and full-way
 * solid cells; rho double[N] or NULL (1), u double[3][N] or NULL (0). The
 * equilibrium is the second-order w_i rho (1 + 3 c.u + 9/2 (c.u)^2 - 3/2 u.u).
 * The paper does not write out its initial state; the verification set-up of
 * Sec. 2.1 (a body-force-driven flow between two slabs) is read as starting
 * from rest, rho = 1 and u = 0, which is what NULL pointers give. Resets the
 * step counter to 0. LBM_ERR_STATE before set_geometry and set_params.
 * Synchronous. */
int lbm_init_equilibrium(lbm_handle h, int32_t lattice, const double* rho, const double* u);

/* Advance every lattice of the handle by n >= 0 time steps (the fused
 * collide-and-propagate sweep, Sec. 3). Asynchronous on the handle's stream;
 * runs of steps are replayed from captured CUDA graphs. */
int lbm_step(lbm_handle h, int32_t n);

/* Temporal blocking of the two-grid pull sweep (listed by the paper among the
 * optimisations its kernels do not cover): with steps_per_pass = 2, runs of
 * steps of a single full-array pull lattice advance two steps per launch. A
 * CTA keeps the first step's post-collision values of a 32 x 8 region over
 * the two or three planes the second step still needs in shared memory,
 * rounded to the storage format as a stored step would round them, and runs
 * the second step one plane behind while it marches along z, so each pass
 * reads and writes the lattice once for two steps. Results equal two one-step
 * sweeps bit for bit. The region is fixed (256 threads), so lbm_set_tuning's
 * block size does not apply to these launches. An odd remaining step runs as
 * a one-step sweep. lbm_autotune tries it for such lattices.
 * steps_per_pass = 1 (the default) turns it off. LBM_ERR_ARG unless 1 or 2;
 * LBM_ERR_UNSUPPORTED for 2 on batches, AA or indirect lattices. */
int lbm_set_temporal_blocking(lbm_handle h, int32_t steps_per_pass);
int lbm_get_temporal_blocking(lbm_handle h, int32_t* steps_per_pass);

/* Reduced indirect addressing (RIA, Sec. 3 "AA Pattern Kernels": a run-length
 * code of the adjacency so that consecutive nodes sharing an access pattern
 * need no lookup of their own). For indirectly addressed lattices the library
 * keeps, next to the link table, a code per chunk of 32 consecutive list nodes
 * and direction: a mask of the nodes that start a run of consecutive links,
 * and the first link of each run. With enable = 1 (the default) the
 * single-lattice list sweeps (pull, and the odd AA step) read the code instead
 * of the table; results are identical either way. The batched sweep always
 * reads the table. lbm_autotune tries both. The code is built and checked
 * against the table when the geometry is set; it costs 144 bytes per 32 nodes
 * plus 4 bytes per run. LBM_ERR_ARG unless enable is 0 or 1. */
int lbm_set_run_indexing(lbm_handle h, int32_t enable);
int lbm_get_run_indexing(lbm_handle h, int32_t* enabled);

/* Index bytes one sweep over lattice `lattice` reads per full pass over its
 * nodes: out[0] for the link table (18 x 4 bytes per fluid node), out[1] for
 * the run-indexed code (headers and run pool). Both 0 for direct addressing.
 * LBM_ERR_STATE before the geometry is set. */
int lbm_adjacency_bytes(lbm_handle h, int32_t lattice, int64_t out[2]);

/* Seed and sweep number of the random bits of LBM_F16_SHIFTED_STOCHASTIC
 * storage (see lbm_precision). Lattice l of a batch uses seed + l. `sweep` is
 * the number t that the next time step draws with (t >= 0); every step then
 * advances it by one. At creation the seed is 0; lbm_init_equilibrium and
 * lbm_write_pdfs set the sweep number to 0, so to resume a run from a
 * checkpoint, write the PDFs first and then call this with the saved seed and
 * step count. Not part of the paper (which stores FP64 only). Returns
 * LBM_ERR_UNSUPPORTED for handles of any other precision, LBM_ERR_ARG for
 * sweep < 0. Synchronous. */
int lbm_set_stochastic_rounding(lbm_handle h, uint64_t seed, int64_t sweep);

/* Wait for all work issued on the handle's stream. No counterpart in the
 * paper (its kernels run synchronously on the CPU). */
int lbm_synchronize(lbm_handle h);

/* Steps taken since the last init_equilibrium / write_pdfs (the iteration
 * count of the benchmark loop, Sec. 2.1 "after enough iterations"). */
int lbm_steps_done(lbm_handle h, int64_t* steps);

/* Canonical PDFs f_i(x, t) of one lattice into out double[19*N] (out_len is
 * the element count, >= 19*N): the D3Q19 populations of Sec. 2 in the
 * full-array order, after propagation and before collision. The AA pattern
 * (Sec. 3 "AA Pattern Kernels") leaves them in swapped or shifted slots after
 * an odd number of steps, and indirect lattices (Sec. 3 "Lattice
 * Representation") store fluid nodes only; this call undoes both, un-shifts
 * the reduced-precision formats and converts to FP64. LBM_ERR_ARG if out_len
 * is too small; LBM_ERR_STATE before the state is initialised. Synchronous. */
int lbm_read_pdfs(lbm_handle h, int32_t lattice, double* out, size_t out_len);

/* Replace the state of one lattice by canonical PDFs in double[19*N]
 * (checkpoint restore; values at half-way solid cells are ignored), the
 * inverse of lbm_read_pdfs: the same populations and layouts (Sec. 2, Sec. 3
 * "Lattice Representation", "AA Pattern Kernels"), rounded to the storage
 * format. Checkpointing itself has no counterpart in the paper. Resets the
 * step counter to 0. LBM_ERR_ARG if in_len is too small. Synchronous. */
int lbm_write_pdfs(lbm_handle h, int32_t lattice, const double* in, size_t in_len);

/* Density rho double[N] and velocity u double[3][N] of one lattice, in FP64
 * from the canonical PDFs: rho = sum f_i, u = (sum c_i f_i + F/2) / rho;
 * 0 at solid cells. The velocity field is what the verification set-up of
 * Sec. 2.1 compares with the analytical Poiseuille solution; the F/2 term is
 * the reading of the paper's constant body force taken here (a source added
 * after collision). Either pointer may be NULL. Synchronous. */
int lbm_read_macroscopic(lbm_handle h, int32_t lattice, double* rho, double* u);

/* Mean of velocity component `comp` (0..2) over the fluid cells of every
 * plane normal to `axis` (0..2), in FP64: out double[n_axis] (0 for planes
 * without fluid). The velocity profile compared with the analytic Poiseuille
 * solution in the verification set-up (Sec. 2.1). Synchronous. */
int lbm_read_profile(lbm_handle h, int32_t lattice, int32_t axis, int32_t comp, double* out, size_t out_len);

/* FP64 sums over every stored PDF of one lattice (fluid and full-way solid
 * cells): out[0] = sum_x sum_i f_i (mass), out[1..3] = sum_x sum_i c_i f_i
 * (momentum). Verification quantities for the set-up of Sec. 2.1: the TRT
 * collision (Sec. 2) conserves mass and adds exactly the body force to the
 * momentum of every fluid node. Synchronous. */
int lbm_read_moments(lbm_handle h, int32_t lattice, double out[4]);

/* The same sums as lbm_read_moments, computed by the same kernels, but this
 * call allocates no device memory: it neither calls cudaMalloc/cudaFree nor
 * goes through the allocator hook. It is meant for callers that must not
 * allocate while they run, for example code whose memory budget is fixed up
 * front, or a host whose allocator is busy in a section it cannot re-enter.
 * The paper has no counterpart: this is a deployment convenience.
 *
 * The scratch is one static device array of 32,772 doubles (256 KiB) that every
 * GPU which loads the library keeps until the process exits. Lattices with more
 * than 134,217,728 cells are rejected with LBM_ERR_ARG. The first call on a
 * device looks up the array's device address (cudaGetSymbolAddress); make that
 * first call before capturing any stream into a CUDA graph. All calls share the
 * array: calls whose work overlaps on a GPU (other threads, other streams) race
 * and must be serialised by the caller. Synchronous on the handle's stream. */
int lbm_read_moments_noalloc(lbm_handle h, int32_t lattice, double out[4]);

/* Flags uint8[N] of one lattice as the library holds them (for spheres: the
 * device voxelisation): the flag field of Sec. 3 "Lattice Representation".
 * Synchronous. */
int lbm_read_flags(lbm_handle h, int32_t lattice, uint8_t* out, size_t out_len);

/* Number of fluid cells of one lattice: the nodes a fluid lattice update
 * (FLUP) counts in the paper's performance figures (Sec. 4.1, loop balance
 * per fluid node update). LBM_ERR_STATE before set_geometry. */
int lbm_fluid_count(lbm_handle h, int32_t lattice, int64_t* n_fluid);

/* Adjacency list of an indirectly addressed lattice into out int32[18*Nf],
 * entry (i-1)*Nf + k for direction i = 1..18 and list node k: the list index
 * of the upstream node x_k - c_i (wrapped) if fluid, else -1 (a bounce-back
 * link). Nodes are the fluid cells in lexicographic order. Table 1's int32
 * adjacency with 18 neighbours; the device keeps it as 32-bit element offsets
 * with the bounce-back target already resolved, and this call decodes them.
 * LBM_ERR_ARG for a directly addressed lattice. Synchronous. */
int lbm_read_adjacency(lbm_handle h, int32_t lattice, int32_t* out, size_t out_len);

/* Kernel launch shape of the handle's sweep. threads: threads per block
 * (multiple of 32 in [32, 512]); cells_per_thread: cells each thread takes per
 * tile of a batch (1, 2, 4 or 8), so a tile holds threads*cells_per_thread
 * cells, or, for a single full-array lattice, 1 or 2 cells of a row per thread
 * (fluid lists use 1); ctas_per_sm: for a batch, the persistent
 * grid's CTAs per SM (0 = one CTA per tile instead of a persistent grid).
 * lbm_set_tuning fixes the shape (a negative value keeps the current one);
 * lbm_get_tuning returns {threads, cells_per_thread, ctas_per_sm}; lbm_autotune
 * times candidate shapes for `steps` steps each on the handle's own data (the
 * state is saved and restored around the trials) and keeps the fastest. The
 * launch-shape search is the GPU analogue of the paper's search over blocking
 * factors (Sec. 4.2, Sec. 4.3). The choice (shape, link encoding, steps per
 * pass) is cached for the process, keyed by a signature of the handle: device,
 * precision, propagation, and per lattice its dims, addressing, fluid count and
 * bounce-back kinds; a later lbm_autotune on a handle with the same signature
 * applies the cached choice without trials. lbm_autotune_cache returns
 * {entries, hits since the process started}; lbm_autotune_clear empties it;
 * lbm_autotune_save writes it to a text file (one line per signature: the
 * signature, threads, cells_per_thread, ctas_per_sm, run_indexing,
 * steps_per_pass) and lbm_autotune_load merges such a file into it
 * (LBM_ERR_ARG if the file cannot be read or written, or on a malformed line,
 * in which case nothing is merged). The signature starts with the GPU's name
 * and SM count. */
int lbm_set_tuning(lbm_handle h, int32_t threads, int32_t cells_per_thread, int32_t ctas_per_sm);
int lbm_get_tuning(lbm_handle h, int32_t out[3]);
int lbm_autotune(lbm_handle h, int32_t steps);
int lbm_autotune_cache(int64_t out[2]);
int lbm_autotune_clear(void);
int lbm_autotune_save(const char* path);
int lbm_autotune_load(const char* path);

/* Device bytes the handle holds (flags, PDF storage, fluid and adjacency
 * lists, batch tables). No counterpart in the paper. */
int lbm_memory_bytes(lbm_handle h, int64_t* bytes);

/* Free every device buffer of the handle (through the allocator it was
 * created with) and the handle itself, after waiting for its stream.
 * LBM_ERR_ARG for NULL.
 * No counterpart in the paper. */
int lbm_destroy(lbm_handle h);

/* No counterpart in the paper: a self-test of this library's failure path.
 * Exercise the bounded-wait path of the staged sweeps on purpose: one CTA arms
 * an mbarrier for bytes that no copy delivers and gives up after `polls` polls
 * (1..2^20). Expected result: LBM_ERR_TIMEOUT, with the handle poisoned and the
 * CUDA context still usable. Nothing faults, traps or hangs. Synchronous. */
int lbm_selftest_bounded_wait(lbm_handle h, int32_t polls);

/* Thread-local message describing the last failed call ("" if none). No
 * counterpart in the paper. The string stays valid until the calling thread's
 * next call into the library. */
const char* lbm_last_error(void);

/* ----------------------------------------------------------------------
 * Bandwidth micro-benchmarks (Sec. 4.1): the GPU counterparts of the paper's
 * copy-19 (19 arrays copied concurrently) and update-19 (19 arrays updated in
 * place). Device pointers; arrays are `n` elements of `elem_bytes` (2, 4 or 8)
 * each, at src + k*stride_elems (k = 0..18). Asynchronous on cuda_stream.
 * ---------------------------------------------------------------------- */
int lbm_bench_copy19(const void* src, void* dst, int64_t n, int64_t stride_elems, int32_t elem_bytes,
                     void* cuda_stream);
int lbm_bench_update19(void* buf, int64_t n, int64_t stride_elems, int32_t elem_bytes, void* cuda_stream);

/* FP64 fused multiply-add throughput probe (the bound of the FP64 sweep on
 * this GPU): `blocks` CTAs of 256 threads each run 16 independent chains of
 * `iterations` FMAs and write their sums to out (device, blocks * 256 doubles,
 * caller-owned). Asynchronous on cuda_stream; the caller times it
 * (2 * 16 * iterations * blocks * 256 flops). LBM_ERR_ARG for NULL or
 * non-positive sizes. lbm_bench_fma64_wave writes the number of such CTAs that
 * the GPU holds at once (SMs x resident CTAs per SM), the block count that
 * times the pipe without a partial second wave; LBM_ERR_ARG for NULL. */
int lbm_bench_fma64(double* out, int32_t blocks, int32_t iterations, void* cuda_stream);
int lbm_bench_fma64_wave(int32_t* blocks);

#ifdef __cplusplus
}
#endif
#endif
