/*
 * Plain FP64 CPU oracle for the D3Q19 TRT lattice Boltzmann sweep
 * (arXiv 1711.11468). TEST INFRASTRUCTURE ONLY: loaded by the tests, the smoke
 * check and the benchmark's CPU-baseline leg, never by the product path.
 *
 * Written for clarity, not speed: fixed summation order i = 0..18, no FMA
 * (compiled with -ffp-contract=off), two grids, push form. Each function names
 * the passage of the paper it follows and the reading it takes where the paper
 * is silent.
 */
#include "lbm_oracle.h"

#include <math.h>
#include <stddef.h>
#include <stdlib.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* D3Q19 (Sec. 2). The paper names the discretisation only; this order is the
 * reading used throughout: rest, the 9 "positive" directions, their negatives. */
static const int CX[ORC_Q] = {0, 1, 0, 0, 1, 1, 1, 1, 0, 0, -1, 0, 0, -1, -1, -1, -1, 0, 0};
static const int CY[ORC_Q] = {0, 0, 1, 0, 1, -1, 0, 0, 1, 1, 0, -1, 0, -1, 1, 0, 0, -1, -1};
static const int CZ[ORC_Q] = {0, 0, 0, 1, 0, 0, 1, -1, 1, -1, 0, 0, -1, 0, 0, -1, 1, -1, 1};

void orc_velocity(int i, int c[3]) {
  c[0] = CX[i];
  c[1] = CY[i];
  c[2] = CZ[i];
}

/* Weights of D3Q19: 1/3 rest, 1/18 for |c|^2 = 1, 1/36 for |c|^2 = 2. */
double orc_weight(int i) {
  int c2 = CX[i] * CX[i] + CY[i] * CY[i] + CZ[i] * CZ[i];
  if (c2 == 0) return 1.0 / 3.0;
  if (c2 == 1) return 1.0 / 18.0;
  return 1.0 / 36.0;
}

/* The opposite direction: the one whose velocity is -c_i. */
int orc_opposite(int i) {
  for (int j = 0; j < ORC_Q; ++j)
    if (CX[j] == -CX[i] && CY[j] == -CY[i] && CZ[j] == -CZ[i]) return j;
  return -1;
}

/* TRT (Sec. 2, Ginzburg's two-relaxation-time model): the symmetric part relaxes
 * with omega+ (which sets the viscosity nu = (1/omega+ - 1/2)/3), the
 * antisymmetric part with omega-, tied to omega+ by the magic parameter
 * Lambda = (1/omega+ - 1/2)(1/omega- - 1/2). */
double orc_omega_minus(double omega_plus, double Lambda) {
  double tau_plus_half = 1.0 / omega_plus - 0.5;
  double tau_minus_half = Lambda / tau_plus_half;
  return 1.0 / (tau_minus_half + 0.5);
}

/* Equilibrium (reading: the standard compressible second-order form). */
void orc_equilibrium(double rho, const double u[3], double feq[ORC_Q]) {
  double usq = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
  for (int i = 0; i < ORC_Q; ++i) {
    double cu = CX[i] * u[0] + CY[i] * u[1] + CZ[i] * u[2];
    feq[i] = orc_weight(i) * rho * (1.0 + 3.0 * cu + 4.5 * cu * cu - 1.5 * usq);
  }
}

/* TRT collision at a fluid node (Sec. 2) plus the constant body force of the
 * verification set-up (Sec. 2.1). Reading of the force: the source term
 * 3 w_i (c_i . F) is added after collision; the equilibrium uses u = j / rho.
 *   f+_i = (f_i + f_opp(i))/2,  f-_i = (f_i - f_opp(i))/2 (same for e),
 *   f*_i = f_i - omega+ (f+_i - e+_i) - omega- (f-_i - e-_i) + 3 w_i (c_i . F). */
void orc_collide_trt(const double f[ORC_Q], double omega_plus, double omega_minus,
                     const double F[3], double fstar[ORC_Q]) {
  double rho = 0.0, j[3] = {0.0, 0.0, 0.0};
  for (int i = 0; i < ORC_Q; ++i) {
    rho += f[i];
    j[0] += CX[i] * f[i];
    j[1] += CY[i] * f[i];
    j[2] += CZ[i] * f[i];
  }
  double u[3] = {j[0] / rho, j[1] / rho, j[2] / rho};
  double e[ORC_Q];
  orc_equilibrium(rho, u, e);
  for (int i = 0; i < ORC_Q; ++i) {
    int o = orc_opposite(i);
    double fp = 0.5 * (f[i] + f[o]);
    double fm = 0.5 * (f[i] - f[o]);
    double ep = 0.5 * (e[i] + e[o]);
    double em = 0.5 * (e[i] - e[o]);
    double source = 3.0 * orc_weight(i) * (CX[i] * F[0] + CY[i] * F[1] + CZ[i] * F[2]);
    fstar[i] = f[i] - omega_plus * (fp - ep) - omega_minus * (fm - em) + source;
  }
}

static int wrap(int a, int n) {
  int r = a % n;
  return r < 0 ? r + n : r;
}

/* Minimum-image offset of a along a periodic axis of length n. */
static int min_image(int a, int n) {
  int r = wrap(a, n);
  if (2 * r > n) r -= n;
  return r;
}

/* Synthetic porous geometry (Sec. 2, heterogeneous geometries): spheres,
 * integer test dx^2 + dy^2 + dz^2 <= r^2 with minimum-image periodic offsets.
 * Every cell is tested against every sphere: slow and obviously complete. */
int orc_voxelize_spheres(int nx, int ny, int nz, const int32_t* cxyzr, int nspheres,
                         uint8_t value, uint8_t* flags) {
  if (nx < 1 || ny < 1 || nz < 1 || nspheres < 0 || !flags) return -1;
  if (nspheres > 0 && !cxyzr) return -1;
  for (int s = 0; s < nspheres; ++s) {
    if (cxyzr[4 * s + 3] < 0) return -1;
  }
#pragma omp parallel for schedule(static)
  for (int z = 0; z < nz; ++z)
    for (int y = 0; y < ny; ++y)
      for (int x = 0; x < nx; ++x) {
        size_t n = (size_t)x + (size_t)nx * ((size_t)y + (size_t)ny * (size_t)z);
        for (int s = 0; s < nspheres; ++s) {
          int64_t dx = min_image(x - cxyzr[4 * s + 0], nx);
          int64_t dy = min_image(y - cxyzr[4 * s + 1], ny);
          int64_t dz = min_image(z - cxyzr[4 * s + 2], nz);
          int64_t r = cxyzr[4 * s + 3];
          if (dx * dx + dy * dy + dz * dz <= r * r) {
            flags[n] = value;
            break;
          }
        }
      }
  return 0;
}

/* Fluid list and adjacency list (Sec. 3 "Lattice Representation"; the
 * adjacency holds 18 4-byte neighbours per node, Table 1). Lexicographic
 * order (reading: the paper's optional blocked order is not used). Every
 * solid cell bounces back half-way here: the list stores fluid nodes only. */
int64_t orc_build_list(int nx, int ny, int nz, const uint8_t* flags,
                       int32_t* cell_of, int32_t* list_index, int32_t* adj) {
  size_t N = (size_t)nx * ny * nz;
  int32_t* idx = (int32_t*)malloc(N * sizeof(int32_t));
  if (!idx) return -1;
  int64_t nf = 0;
  for (size_t n = 0; n < N; ++n) {
    if (flags[n] == 0) {
      if (cell_of) cell_of[nf] = (int32_t)n;
      idx[n] = (int32_t)nf++;
    } else {
      idx[n] = -1;
    }
  }
  if (list_index)
    for (size_t n = 0; n < N; ++n) list_index[n] = idx[n];
  if (adj) {
    for (int z = 0; z < nz; ++z)
      for (int y = 0; y < ny; ++y)
        for (int x = 0; x < nx; ++x) {
          size_t n = (size_t)x + (size_t)nx * ((size_t)y + (size_t)ny * (size_t)z);
          if (idx[n] < 0) continue;
          for (int i = 1; i < ORC_Q; ++i) {
            int ux = wrap(x - CX[i], nx), uy = wrap(y - CY[i], ny), uz = wrap(z - CZ[i], nz);
            size_t m = (size_t)ux + (size_t)nx * ((size_t)uy + (size_t)ny * (size_t)uz);
            adj[(size_t)(i - 1) * (size_t)nf + (size_t)idx[n]] = idx[m];
          }
        }
  }
  free(idx);
  return nf;
}

void orc_init_equilibrium(int nx, int ny, int nz, const uint8_t* flags,
                          const double* rho, const double* u, double* f) {
  size_t N = (size_t)nx * ny * nz;
  for (size_t n = 0; n < N; ++n) {
    double feq[ORC_Q];
    if (flags[n] == 2) {
      for (int i = 0; i < ORC_Q; ++i) f[(size_t)i * N + n] = 0.0;
      continue;
    }
    double r = rho ? rho[n] : 1.0;
    double v[3] = {u ? u[n] : 0.0, u ? u[N + n] : 0.0, u ? u[2 * N + n] : 0.0};
    orc_equilibrium(r, v, feq);
    for (int i = 0; i < ORC_Q; ++i) f[(size_t)i * N + n] = feq[i];
  }
}

/* One fused collide-and-propagate step in two-grid push form (Sec. 3 "One
 * Step Kernels": read locally, collide, write to the neighbours).
 * Bounce-back (Sec. 2, Sec. 3.2):
 *   - full-way: a solid cell of flag 1 holds PDFs and, instead of colliding,
 *     reverses them, f*_i = f_opp(i); streaming is unchanged;
 *   - half-way: a link into a cell of flag 2 reflects at mid-link,
 *     f_opp(i)(x, t+1) = f*_i(x, t).
 * Periodicity: index arithmetic wraps in every dimension. */
void orc_step(int nx, int ny, int nz, const uint8_t* flags, double omega_plus,
              double omega_minus, const double F[3], const double* src, double* dst,
              int nthreads) {
  size_t N = (size_t)nx * ny * nz;
#ifdef _OPENMP
  if (nthreads <= 0) nthreads = omp_get_max_threads();
#pragma omp parallel for schedule(static) num_threads(nthreads)
#endif
  for (int z = 0; z < nz; ++z)
    for (int y = 0; y < ny; ++y)
      for (int x = 0; x < nx; ++x) {
        size_t n = (size_t)x + (size_t)nx * ((size_t)y + (size_t)ny * (size_t)z);
        if (flags[n] == 2) continue;
        double f[ORC_Q], fs[ORC_Q];
        for (int i = 0; i < ORC_Q; ++i) f[i] = src[(size_t)i * N + n];
        if (flags[n] == 1) {
          for (int i = 0; i < ORC_Q; ++i) fs[i] = f[orc_opposite(i)];
        } else {
          orc_collide_trt(f, omega_plus, omega_minus, F, fs);
        }
        for (int i = 0; i < ORC_Q; ++i) {
          int dx = wrap(x + CX[i], nx), dy = wrap(y + CY[i], ny), dz = wrap(z + CZ[i], nz);
          size_t m = (size_t)dx + (size_t)nx * ((size_t)dy + (size_t)ny * (size_t)dz);
          if (flags[m] == 2)
            dst[(size_t)orc_opposite(i) * N + n] = fs[i];
          else
            dst[(size_t)i * N + m] = fs[i];
        }
      }
  (void)nthreads;
}

/* Density and velocity (Sec. 2.1 verification compares the velocity profile).
 * Reading: with the source term above the physical velocity is
 * u = (j + F/2) / rho. */
void orc_macroscopic(int nx, int ny, int nz, const uint8_t* flags, const double F[3],
                     const double* f, double* rho, double* u) {
  size_t N = (size_t)nx * ny * nz;
  for (size_t n = 0; n < N; ++n) {
    double r = 0.0, j[3] = {0.0, 0.0, 0.0};
    if (flags[n] == 0) {
      for (int i = 0; i < ORC_Q; ++i) {
        double fi = f[(size_t)i * N + n];
        r += fi;
        j[0] += CX[i] * fi;
        j[1] += CY[i] * fi;
        j[2] += CZ[i] * fi;
      }
    }
    if (rho) rho[n] = r;
    if (u) {
      for (int a = 0; a < 3; ++a) u[(size_t)a * N + n] = r != 0.0 ? (j[a] + 0.5 * F[a]) / r : 0.0;
    }
  }
}

/* splitmix64 (Steele, Lea and Flood, "Fast splittable pseudorandom number
 * generators", OOPSLA 2014): the state advances by the golden-ratio gamma and
 * each output is the state passed through the "mix64" finaliser. */
static uint64_t mix64(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

uint64_t orc_splitmix64(uint64_t seed, uint64_t k) {
  return mix64(seed + (k + 1u) * 0x9E3779B97F4A7C15ull);
}

uint32_t orc_sr_bits(uint64_t seed, uint64_t t, uint64_t node, int j) {
  uint64_t key = orc_splitmix64(seed, (t << 32) | node);
  int m = j / 4;
  uint64_t word = m == 0 ? key : orc_splitmix64(key, (uint64_t)(m - 1));
  uint32_t half = (uint32_t)(((j % 4) / 2) == 0 ? word : word >> 32);
  return (j % 2) == 0 ? (half & 0x1FFFu) : (half >> 19);
}

/* Stochastic rounding onto the FP16 grid (see the header). u is a power of
 * two, so a / u, its floor and the remainder q are exact; the threshold
 * 1 - r / 2^13 has 13 bits and is exact too, so the comparison decides
 * exactly, in every binade. */
double orc_round_half_stochastic(double x, uint32_t r, double* margin) {
  if (isnan(x) || isinf(x)) {
    if (margin) *margin = INFINITY;
    return x;
  }
  double a = fabs(x);
  int e;
  (void)frexp(a, &e);                 /* a in [2^(e-1), 2^e) */
  int ue = e - 1 >= -14 ? e - 11 : -24; /* FP16 spacing at a: 2^(ex-10) for a >= 2^-14 */
  double u = ldexp(1.0, ue);
  double lo = floor(a / u);
  double q = a / u - lo;              /* remainder in spacings, in [0, 1) */
  double thr = 1.0 - ldexp((double)r, -13);
  double res;
  if (q == 0.0) {
    res = lo * u;
    if (margin) *margin = INFINITY;
  } else {
    res = (q >= thr ? lo + 1.0 : lo) * u;
    if (margin) *margin = fabs(q - thr);
  }
  if (res > 65504.0) res = 65504.0;
  return x < 0 ? -res : res;
}

void orc_round_half_stochastic_n(const double* x, const uint32_t* r, int64_t n, double* out, double* margin) {
  for (int64_t k = 0; k < n; ++k) out[k] = orc_round_half_stochastic(x[k], r[k], margin ? &margin[k] : NULL);
}

void orc_step_f16_stochastic(int nx, int ny, int nz, const uint8_t* flags, double omega_plus,
                             double omega_minus, const double F[3], const double* d_src, double* d_dst,
                             uint64_t seed, uint64_t t, const int32_t* node_of, double* margin) {
  size_t N = (size_t)nx * ny * nz;
  if (margin)
    for (size_t k = 0; k < (size_t)ORC_Q * N; ++k) margin[k] = INFINITY;
  for (int z = 0; z < nz; ++z)
    for (int y = 0; y < ny; ++y)
      for (int x = 0; x < nx; ++x) {
        size_t n = (size_t)x + (size_t)nx * ((size_t)y + (size_t)ny * (size_t)z);
        if (flags[n] == 2) continue;
        double f[ORC_Q], fs[ORC_Q], ds[ORC_Q], mg[ORC_Q];
        if (flags[n] == 1) {
          for (int i = 0; i < ORC_Q; ++i) {
            ds[i] = d_src[(size_t)orc_opposite(i) * N + n];
            mg[i] = INFINITY;
          }
        } else {
          for (int i = 0; i < ORC_Q; ++i) f[i] = orc_weight(i) + d_src[(size_t)i * N + n];
          orc_collide_trt(f, omega_plus, omega_minus, F, fs);
          uint64_t node = node_of ? (uint64_t)node_of[n] : (uint64_t)n;
          for (int i = 0; i < ORC_Q; ++i) {
            double x = ldexp(fs[i] - orc_weight(i), ORC_F16_SCALE_LOG2);
            ds[i] = ldexp(orc_round_half_stochastic(x, orc_sr_bits(seed, t, node, i), &mg[i]),
                          -ORC_F16_SCALE_LOG2);
          }
        }
        for (int i = 0; i < ORC_Q; ++i) {
          int dx = wrap(x + CX[i], nx), dy = wrap(y + CY[i], ny), dz = wrap(z + CZ[i], nz);
          size_t m = (size_t)dx + (size_t)nx * ((size_t)dy + (size_t)ny * (size_t)dz);
          size_t slot = flags[m] == 2 ? (size_t)orc_opposite(i) * N + n : (size_t)i * N + m;
          d_dst[slot] = ds[i];
          if (margin) margin[slot] = mg[i];
        }
      }
}

int orc_max_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}
