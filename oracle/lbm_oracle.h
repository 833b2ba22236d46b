/*
 * Plain FP64 CPU oracle for the D3Q19 TRT lattice Boltzmann sweep
 * (Wittmann et al., "Lattice Boltzmann Benchmark Kernels as a Testbed for
 * Performance Analysis", arXiv 1711.11468).
 *
 * TEST INFRASTRUCTURE ONLY. This library exists to check the CUDA path: only
 * the test suite, the smoke check and the CPU-baseline leg of the benchmark
 * load it. It shares no code, header, table or constant with the CUDA library.
 *
 * The paper names the model (Sec. 2: D3Q19, TRT collision, half-way and
 * full-way bounce-back, constant body force for verification) but does not
 * write it out. Every reading taken here is listed next to the function that
 * takes it.
 *
 * Conventions:
 *   - cell index n = x + nx*(y + ny*z), x fastest;
 *   - PDF arrays are double[19][N] (direction-major, "SoA", Sec. 3 "Data Layout");
 *   - flags: 0 fluid, 1 full-way bounce-back solid (holds PDFs),
 *            2 half-way bounce-back solid (holds nothing; its slots stay 0);
 *   - index arithmetic wraps in every dimension.
 */
#ifndef LBM_ORACLE_H
#define LBM_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define ORC_Q 19

/* Velocity c_i and weight w_i of direction i (0..18). Reading of "D3Q19" (Sec. 2):
 * 0 rest; 1..9 = (1,0,0) (0,1,0) (0,0,1) (1,1,0) (1,-1,0) (1,0,1) (1,0,-1) (0,1,1)
 * (0,1,-1); 10..18 their negatives; w = 1/3, 1/18 (faces), 1/36 (edges). */
void orc_velocity(int i, int c[3]);
double orc_weight(int i);
int orc_opposite(int i);

/* omega_minus from the TRT magic parameter Lambda = (1/w+ - 1/2)(1/w- - 1/2)
 * (TRT, Sec. 2). */
double orc_omega_minus(double omega_plus, double Lambda);

/* Second-order equilibrium e_i = w_i rho (1 + 3 c.u + 9/2 (c.u)^2 - 3/2 u.u). */
void orc_equilibrium(double rho, const double u[3], double feq[ORC_Q]);

/* TRT collision of one fluid node followed by the body-force source
 * 3 w_i (c_i . F). */
void orc_collide_trt(const double f[ORC_Q], double omega_plus, double omega_minus,
                     const double F[3], double fstar[ORC_Q]);

/* Voxelise spheres (cx, cy, cz, r) into flags: a cell is inside when
 * dx^2 + dy^2 + dz^2 <= r^2 with minimum-image periodic offsets. Inside cells
 * get `value`, others are left untouched. Returns 0, or -1 on bad input. */
int orc_voxelize_spheres(int nx, int ny, int nz, const int32_t* cxyzr, int nspheres,
                         uint8_t value, uint8_t* flags);

/* Fluid list and adjacency list (Sec. 3 "Lattice Representation"):
 * fluid cells in lexicographic order; cell_of[k] = cell index of list node k;
 * list_index[n] = k or -1; adj[(i-1)*nf + k] for i = 1..18 = list index of the
 * upstream node n - c_i (wrapped) if it is fluid, else -1 (a bounce-back link).
 * Any arrays may be NULL. Returns the fluid count. */
int64_t orc_build_list(int nx, int ny, int nz, const uint8_t* flags,
                       int32_t* cell_of, int32_t* list_index, int32_t* adj);

/* Equilibrium initial state: f_i(x, 0) = e_i(rho(x), u(x)) at fluid and
 * full-way solid cells, 0 at half-way solid cells. rho may be NULL (1),
 * u may be NULL (0); u is double[3][N]. */
void orc_init_equilibrium(int nx, int ny, int nz, const uint8_t* flags,
                          const double* rho, const double* u, double* f);

/* One time step in two-grid push form: src holds f(t) (post-streaming), dst
 * receives f(t+1). dst must be zero at half-way solid cells on entry.
 * nthreads <= 0 uses the OpenMP default. */
void orc_step(int nx, int ny, int nz, const uint8_t* flags, double omega_plus,
              double omega_minus, const double F[3], const double* src, double* dst,
              int nthreads);

/* Macroscopic fields: rho = sum f_i, u = (sum c_i f_i + F/2) / rho at fluid cells,
 * 0 at solid cells. u is double[3][N]. */
void orc_macroscopic(int nx, int ny, int nz, const uint8_t* flags, const double F[3],
                     const double* f, double* rho, double* u);

/* ---------------------------------------------------------------------------
 * Scaled FP16-shifted storage with stochastic rounding (an accuracy remedy for
 * the FP16-shifted format; not in the paper, whose error study of reduced
 * precision storage is the verification set-up of Sec. 2.1).
 *
 * State: deviations d_i = f_i - w_i, stored as the FP16 value h_i of
 * d_i * 2^14 (so FP16's normal range covers |d| from 2^-28 to 4); held here as
 * doubles d_i = h_i * 2^-14. One step: f = w + d, the FP64 collision and
 * bounce-back of orc_step, then each post-collision value x = (f*_j - w_j) 2^14
 * of a fluid node is rounded to FP16 stochastically with 13 random bits
 * r(seed, t, node, j); full-way solid nodes only reverse their (already FP16)
 * values.
 *
 * Random bits (counter-based, splitmix64 of Steele, Lea and Flood, OOPSLA
 * 2014): node `node` at sweep t draws the key
 *   K = splitmix64 output number ((t << 32) | node) of the stream seeded `seed`,
 * then the words W_0 = K and W_m = output number m-1 of the stream seeded K
 * (m = 1..4). Direction j reads the 32-bit half (j mod 4) div 2 of
 * W_(j div 4) (0 = low) and takes its bits 0..12 for even j, 19..31 for odd j.
 *
 * Rounding rule (stochastic rounding with a 13-bit draw): with a = |x|, u the
 * FP16 spacing at a (2^(e-10) for a in [2^e, 2^(e+1)), e >= -14; 2^-24 below
 * 2^-14, FP16's subnormal range), lo = u floor(a / u) and q = a / u - floor(a / u)
 * the remainder in spacings, the result is sign(x) (lo + u) when
 * q + r / 2^13 >= 1 and sign(x) lo otherwise; results beyond the FP16 range
 * saturate at 65504. Over the 2^13 equally likely draws x rounds away from zero
 * floor(2^13 q) times: the mean is x truncated to the grid of u / 2^13, which
 * is x itself for an FP32 value in FP16's normal range (13 bits below u) and
 * within u / 2^13 of x everywhere, subnormals included.
 * ------------------------------------------------------------------------ */

/* log2 of the storage scale of the format: d * 2^14 is stored. */
#define ORC_F16_SCALE_LOG2 14

/* Output number k (0-based) of splitmix64 seeded `seed`: mix(seed + (k+1) * gamma). */
uint64_t orc_splitmix64(uint64_t seed, uint64_t k);

/* The 13 random bits of direction j of node `node` at sweep t. */
uint32_t orc_sr_bits(uint64_t seed, uint64_t t, uint64_t node, int j);

/* Stochastic rounding of x to FP16 with random bits r (0..8191), the rule
 * above. If margin is not NULL it receives |q + r / 2^13 - 1|, the distance of
 * the decision from its threshold in FP16 spacings (infinite when x is an FP16
 * value or not finite). */
double orc_round_half_stochastic(double x, uint32_t r, double* margin);

/* The same over arrays: out[k] and margin[k] (margin may be NULL) for x[k], r[k]. */
void orc_round_half_stochastic_n(const double* x, const uint32_t* r, int64_t n, double* out, double* margin);

/* One push step of the format: d_src holds the deviations at sweep t (FP16
 * values times 2^-14; 0 at half-way solid cells), d_dst receives them at t+1
 * (must be zero at half-way solid cells on entry). node_of[N] numbers the
 * nodes that draw the random bits (NULL: the cell index). margin (NULL, or
 * double[19][N]) receives, for each slot of d_dst, the margin of the rounding
 * that produced it (INFINITY where no rounding happened). */
void orc_step_f16_stochastic(int nx, int ny, int nz, const uint8_t* flags, double omega_plus,
                             double omega_minus, const double F[3], const double* d_src, double* d_dst,
                             uint64_t seed, uint64_t t, const int32_t* node_of, double* margin);

/* Threads the OpenMP runtime would use (1 when built without OpenMP). */
int orc_max_threads(void);

#ifdef __cplusplus
}
#endif
#endif
