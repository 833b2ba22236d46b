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

/* Threads the OpenMP runtime would use (1 when built without OpenMP). */
int orc_max_threads(void);

#ifdef __cplusplus
}
#endif
#endif
