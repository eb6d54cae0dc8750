/*
 * olbm_oracle.c -- plain, slow, FP64 CPU oracle of the D2Q9 generalized
 * Onsager-regularised lattice Boltzmann step (arXiv 2602.21242, Secs. 1-4).
 *
 * TEST INFRASTRUCTURE ONLY. Nothing in the product library (the CUDA path)
 * links, includes or calls this file; only tests/, the smoke check and the
 * benchmark's CPU-baseline leg load it. It shares no code, header or table
 * with the CUDA path.
 *
 * Conventions (readings of the paper, each stated once):
 *   - D2Q9 numbering of Fig. 1a: c0=(0,0), c1=(1,0), c2=(0,1), c3=(-1,0),
 *     c4=(0,-1), c5=(1,1), c6=(-1,1), c7=(-1,-1), c8=(1,-1).
 *   - Fields are stored [i][y][x], x fastest, doubly periodic, node-centred
 *     coordinates x = 0..nx-1, y = 0..ny-1.
 *   - Optional wall nodes (a byte mask [y][x]) use fullway bounce-back, the
 *     wall treatment of the shocktube (Sec. 5.2): they reverse every population
 *     instead of colliding.
 *   - The state is the set of PRE-collision populations f_i(x, t). One step is
 *     collide everywhere (Eq. 1a), then propagate f*_i(x) to x + c_i (Eq. 1b).
 *   - Initial state: f(x, 0) = f^eq(rho0(x), u0(x)) (Eq. 10).
 *   - Diagnostics are taken on the pre-collision populations at time t.
 *   - tau is passed in; the viscosity mapping nu = theta (tau - 1/2) lives in
 *     the Python wrapper.
 *
 * The per-node arithmetic lives in olbm_core.inc and is instantiated for
 * double (the oracle) and for double _Complex (complex-step derivatives).
 * Compile with -ffp-contract=off so that the arithmetic is exactly what is
 * written, on every host.
 */
#include <complex.h>
#include <math.h>
#include <stddef.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define Q9 9
static const int CX[9] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
static const int CY[9] = {0, 0, 1, 0, -1, 1, 1, -1, -1};

/* ---- real instantiation ---- */
#define R double
#define FN(name) r_##name
#include "olbm_core.inc"
#undef R
#undef FN

/* ---- complex instantiation (complex-step differentiation) ---- */
#define R double _Complex
#define FN(name) z_##name
#include "olbm_core.inc"
#undef R
#undef FN

/* ------------------------------------------------------------------------- */
/* Exported entry points (called through ctypes by oracle/oracle.py).        */
/* ------------------------------------------------------------------------- */

int oracle_version(void) { return 2; }

int oracle_set_threads(int n) {
#ifdef _OPENMP
  if (n > 0) omp_set_num_threads(n);
  return omp_get_max_threads();
#else
  (void)n;
  return 1;
#endif
}

/* Eq. 10 at one node. */
void oracle_geq(double rho, double ux, double uy, double theta, double* feq9) {
  r_geq(rho, ux, uy, theta, feq9);
}

/* Eq. 1a at one node: post-collision populations of pre-collision f9. */
void oracle_collide_node(const double* f9, double theta, double tau, int model, double* fs9) {
  r_collide(f9, theta, tau, model, fs9);
}

/*
 * Intermediate quantities of one collision, for the tests that pin them:
 *   mom3 = (rho, u_x, u_y), feq9 (Eq. 10), foreg9 (Eq. 2), psi2 (Eq. 6a),
 *   pref1 (Eq. 12), pit3 = Pi~ (xx, yy, xy) (Eq. 11b),
 *   psiP9 (Eq. 14), psiC9 (Eq. 15).
 */
void oracle_node_terms(const double* f9, double theta, double* mom3, double* feq9,
                       double* foreg9, double* psi2, double* pref1, double* pit3,
                       double* psiP9, double* psiC9) {
  double rho, ux, uy;
  r_moments(f9, &rho, &ux, &uy);
  mom3[0] = rho;
  mom3[1] = ux;
  mom3[2] = uy;
  r_geq(rho, ux, uy, theta, feq9);
  r_oreg(f9, feq9, rho, ux, uy, theta, foreg9);
  r_psi(foreg9, psi2);
  pref1[0] = r_pref(foreg9, theta);
  r_pitilde(pref1[0], ux, uy, theta, pit3);
  r_corr_partial(psi2, psiP9);
  r_corr_complete(psi2, pit3, psiC9);
}

/* Eq. 2 alone, for an arbitrary (f, f^eq, rho, u) -- lets tests feed textbook cases. */
void oracle_oreg_node(const double* f9, const double* feq9, double rho, double ux, double uy,
                      double theta, double* foreg9) {
  r_oreg(f9, feq9, rho, ux, uy, theta, foreg9);
}

/* f(x, 0) = f^eq(rho0(x), u0(x)) on the whole grid; f has 9 * nx * ny entries. */
void oracle_init(int nx, int ny, double theta, const double* rho, const double* ux,
                 const double* uy, double* f) {
  r_init(rho, ux, uy, nx, ny, theta, f);
}

/*
 * nsteps LBE steps (Eq. 1) in place on f (9 * nx * ny pre-collision values);
 * work is caller scratch of the same size. walls: NULL, or nx * ny flags
 * (nonzero = fullway bounce-back node).
 */
void oracle_run_walls(int nx, int ny, double theta, double tau, int model, int nsteps,
                      const unsigned char* walls, double* f, double* work) {
  const size_t n9 = (size_t)9 * nx * ny;
  double* a = f;
  double* b = work;
  for (int s = 0; s < nsteps; ++s) {
    r_step(a, b, nx, ny, theta, tau, model, walls);
    double* t = a;
    a = b;
    b = t;
  }
  if (a != f) memcpy(f, a, n9 * sizeof(double));
}

void oracle_run(int nx, int ny, double theta, double tau, int model, int nsteps, double* f,
                double* work) {
  oracle_run_walls(nx, ny, theta, tau, model, nsteps, NULL, f, work);
}

/* Complex-step twin of oracle_run_walls: f and work are interleaved (re, im) pairs. */
void oracle_run_walls_cplx(int nx, int ny, double theta, double tau, int model, int nsteps,
                           const unsigned char* walls, double* f_ri, double* work_ri) {
  const size_t n9 = (size_t)9 * nx * ny;
  double _Complex* a = (double _Complex*)f_ri;
  double _Complex* b = (double _Complex*)work_ri;
  double _Complex* f = a;
  for (int s = 0; s < nsteps; ++s) {
    z_step(a, b, nx, ny, theta, tau, model, walls);
    double _Complex* t = a;
    a = b;
    b = t;
  }
  if (a != f) memcpy(f, a, n9 * sizeof(double _Complex));
}

void oracle_run_cplx(int nx, int ny, double theta, double tau, int model, int nsteps,
                     double* f_ri, double* work_ri) {
  oracle_run_walls_cplx(nx, ny, theta, tau, model, nsteps, NULL, f_ri, work_ri);
}

/* Complex-step twin of oracle_init (inputs and output interleaved re, im). */
void oracle_init_cplx(int nx, int ny, double theta, const double* rho_ri, const double* ux_ri,
                      const double* uy_ri, double* f_ri) {
  z_init((const double _Complex*)rho_ri, (const double _Complex*)ux_ri,
         (const double _Complex*)uy_ri, nx, ny, theta, (double _Complex*)f_ri);
}

/* Complex-step twin of oracle_collide_node. */
void oracle_collide_node_cplx(const double* f9_ri, double theta, double tau, int model,
                              double* fs9_ri) {
  z_collide((const double _Complex*)f9_ri, theta, tau, model, (double _Complex*)fs9_ri);
}

/* (rho, u_x, u_y) of the pre-collision populations at every node. */
void oracle_moments_field(int nx, int ny, const double* f, double* rho, double* ux, double* uy) {
  const size_t N = (size_t)nx * ny;
  for (size_t n = 0; n < N; ++n) {
    double fl[9];
    for (int i = 0; i < Q9; ++i) fl[i] = f[(size_t)i * N + n];
    r_moments(fl, &rho[n], &ux[n], &uy[n]);
  }
}

/* Complex-step twin of oracle_moments_field. */
void oracle_moments_field_cplx(int nx, int ny, const double* f_ri, double* rho_ri, double* ux_ri,
                               double* uy_ri) {
  const size_t N = (size_t)nx * ny;
  const double _Complex* f = (const double _Complex*)f_ri;
  double _Complex* rho = (double _Complex*)rho_ri;
  double _Complex* ux = (double _Complex*)ux_ri;
  double _Complex* uy = (double _Complex*)uy_ri;
  for (size_t n = 0; n < N; ++n) {
    double _Complex fl[9];
    for (int i = 0; i < Q9; ++i) fl[i] = f[(size_t)i * N + n];
    z_moments(fl, &rho[n], &ux[n], &uy[n]);
  }
}

/* Neumaier (compensated) summation, so the oracle's totals are accurate to roundoff. */
typedef struct {
  double s, c;
} nsum_t;

static void nsum_add(nsum_t* a, double v) {
  const double t = a->s + v;
  if (fabs(a->s) >= fabs(v)) {
    a->c += (a->s - t) + v;
  } else {
    a->c += (v - t) + a->s;
  }
  a->s = t;
}

/*
 * Global diagnostics of the pre-collision populations f(t):
 *   out[0] = sum rho, out[1] = sum rho u_x, out[2] = sum rho u_y,
 *   out[3] = sum 1/2 rho |u|^2, out[4] = number of nodes with a non-finite f_i.
 */
void oracle_diagnostics(int nx, int ny, const double* f, double* out5) {
  const size_t N = (size_t)nx * ny;
  nsum_t m = {0, 0}, px = {0, 0}, py = {0, 0}, ke = {0, 0};
  double bad = 0.0;
  for (size_t n = 0; n < N; ++n) {
    double rho = 0.0, jx = 0.0, jy = 0.0;
    int finite = 1;
    for (int i = 0; i < Q9; ++i) {
      const double v = f[(size_t)i * N + n];
      if (!isfinite(v)) finite = 0;
      rho += v;
      jx += (double)CX[i] * v;
      jy += (double)CY[i] * v;
    }
    if (!finite) {
      bad += 1.0;
      continue;
    }
    nsum_add(&m, rho);
    nsum_add(&px, jx);
    nsum_add(&py, jy);
    nsum_add(&ke, 0.5 * (jx * jx + jy * jy) / rho);
  }
  out5[0] = m.s + m.c;
  out5[1] = px.s + px.c;
  out5[2] = py.s + py.c;
  out5[3] = ke.s + ke.c;
  out5[4] = bad;
}
