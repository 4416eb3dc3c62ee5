/*
 * lb_oracle.c -- FP64 CPU oracle of the two-species soft-glassy lattice
 * Boltzmann step (Benzi, Sbragaglia, Succi, Bernaschi, Chibbaro,
 * arXiv:0906.3611).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the correctness reference that the
 * CUDA path is compared against.  Only the test suite, the smoke check and the
 * CPU-baseline leg of the benchmark may load it.  It shares no code, header,
 * table or constant with the CUDA library: every constant below is written out
 * here from the paper.
 *
 * The step is done as separate whole-lattice passes, in the order the method
 * states them (Sec. II):
 *   1. rho_s(r)  = sum_i f_is(r)                             (below Eq. (be))
 *   2. psi_s(r)  = rho0 (1 - exp(-rho_s/rho0))               Eq. (PSI)
 *   3. F_s(r)    = F^a_s + F^r_s + F^X_s                      Eq. (FORCE), Table I
 *   4. u(r)      = sum_s (1/tau_s) sum_i f_is c_i / sum_s rho_s/tau_s
 *   5. f^eq_is   = w_i rho_s (1 + c.v/cs2 + (c_a c_b - cs2 d_ab) v_a v_b/(2 cs2^2)),
 *                  v = u + tau_s F_s / rho_s, cs2 = 1/3
 *   6. f*_is     = f_is - (f_is - f^eq_is)/tau_s                 Eq. (be)
 *   7. f_is(r+c_i, t+1) = f*_is(r, t)                          Eq. (be), LHS
 *
 * Readings taken where the paper is silent (each is listed in the design notes):
 *   - Couette walls (not in the paper): halfway bounce-back with walls at
 *     y = -1/2 (moving -U) and y = ny - 1/2 (moving +U); a link that would
 *     leave the fluid returns to its own node reversed,
 *         f_{opp(i)}(r, t+1) = f*_i(r, t) - 2 w_i rho_s(r, t) (c_i . U_w) / cs2,
 *     with rho_s(r, t) the density of the node at the start of the step.
 *     For the force stencil the density field is mirrored about each wall:
 *     row -1 reads row 0, row -2 reads row 1, row ny reads row ny-1, ...
 *   - a node with rho_s <= 0 gets no velocity shift for species s and is
 *     counted in the returned status.
 *   - the common velocity reported is the paper's u (no half-force term).
 *
 * Layout of every population array: f[((s*9 + i)*ny + y)*nx + x], x fastest,
 * s = 0 (A), 1 (B).  D2Q9 order i = 0..8:
 *   (0,0) (1,0) (0,1) (-1,0) (0,-1) (1,1) (-1,1) (-1,-1) (1,-1).
 *
 * Parameter vector prm[] (doubles):
 *   0 tau_A   1 tau_B   2 rho0   3 G_AB   4 Ga_A  5 Ga_B  6 Gr_A  7 Gr_B
 *   8 boundary (0 periodic, 1 Couette)    9 U_wall
 *   10 g (Kolmogorov body acceleration amplitude)   11 k (its wave number)
 *
 * Kolmogorov shear (Sec. VII: a flow U_x = U0 sin(ky) imposed by a volumetric
 * body force): every species feels the force density rho_s g sin(2 pi k y / ny)
 * along x, added to F_s of Eq. (FORCE) so that it enters the shifted velocity
 * of Eq. (be) like the interaction forces.
 *
 * Build with -ffp-contract=off so that results do not depend on whether the
 * host compiler fuses multiply-adds.
 */
#define _GNU_SOURCE 1
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* ---- D2Q9 populations (the speeds of Eq. (be); weights w_i of Table I,
 *      second block, used also as the equilibrium weights w_i^(eq)) ---- */
static const int CX9[9] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
static const int CY9[9] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
static const int OPP9[9] = {0, 3, 4, 1, 2, 7, 8, 5, 6};
#define CS2 (1.0 / 3.0)

static double w9(int i) {
  if (i == 0) return 4.0 / 9.0;
  if (i <= 4) return 1.0 / 9.0;
  return 1.0 / 36.0;
}

/* ---- The 25-speed forcing lattice of Table I.
 *      j = 0 rest; belt 1 = j 1..8 (the D2Q9 moving speeds, same order);
 *      belt 2 = j 9..24: (+-2,0),(0,+-2); (+-2,+-1),(+-1,+-2); (+-2,+-2). ---- */
static const int CXF[25] = {0, 1, 0, -1, 0, 1, -1, -1, 1,
                            2, 0, -2, 0,
                            2, 1, -1, -2, -2, -1, 1, 2,
                            2, -2, -2, 2};
static const int CYF[25] = {0, 0, 1, 0, -1, 1, 1, -1, -1,
                            0, 2, 0, -2,
                            1, 2, 2, 1, -1, -2, -2, -1,
                            2, 2, -2, -2};

/* p_j of Table I (forcing weights of F^r), by group of j. */
static double pF(int j) {
  if (j == 0) return 247.0 / 420.0;
  if (j <= 4) return 4.0 / 63.0;
  if (j <= 8) return 4.0 / 135.0;
  if (j <= 12) return 1.0 / 180.0;
  if (j <= 20) return 2.0 / 945.0;
  return 1.0 / 15120.0;
}

/* w_j of Table I restricted to belt 1 (forcing weights of F^a and F^X). */
static double wF(int j) {
  if (j == 0) return 4.0 / 9.0;
  if (j <= 4) return 1.0 / 9.0;
  if (j <= 8) return 1.0 / 36.0;
  return 0.0;
}

/* Expose the tables so the tests can check them against Table I and Eq. (NORM0). */
void lbo_tables(int *cx9, int *cy9, double *w9out, int *cxf, int *cyf,
                double *pout, double *wout) {
  for (int i = 0; i < 9; ++i) {
    cx9[i] = CX9[i];
    cy9[i] = CY9[i];
    w9out[i] = w9(i);
  }
  for (int j = 0; j < 25; ++j) {
    cxf[j] = CXF[j];
    cyf[j] = CYF[j];
    pout[j] = pF(j);
    wout[j] = wF(j);
  }
}

static inline size_t IDX(int s, int i, int y, int x, int nx, int ny) {
  return (((size_t)(s * 9 + i) * (size_t)ny + (size_t)y) * (size_t)nx) + (size_t)x;
}

static inline int wrap(int a, int n) {
  int r = a % n;
  return r < 0 ? r + n : r;
}

/* Row index used by the force stencil: periodic, or mirrored about the walls
 * (y = -1/2 and y = ny - 1/2) for the Couette geometry. */
static inline int stencil_row(int y, int ny, int couette) {
  if (!couette) return wrap(y, ny);
  while (y < 0 || y >= ny) {
    if (y < 0) y = -1 - y;
    if (y >= ny) y = 2 * ny - 1 - y;
  }
  return y;
}

/* ---- pass 1: densities rho_s = sum_i f_is ---- */
void lbo_densities(const double *f, int nx, int ny, double *rho) {
#pragma omp parallel for schedule(static)
  for (int y = 0; y < ny; ++y)
    for (int s = 0; s < 2; ++s)
      for (int x = 0; x < nx; ++x) {
        double r = 0.0;
        for (int i = 0; i < 9; ++i) r += f[IDX(s, i, y, x, nx, ny)];
        rho[((size_t)s * ny + y) * nx + x] = r;
      }
}

/* ---- pass 2: pseudo-potential, Eq. (PSI) with a common rho0 ---- */
static double psi_of(double rho, double rho0) { return rho0 * (1.0 - exp(-rho / rho0)); }

/* ---- pass 3: forces, Eq. (FORCE).  rho[s][y][x] in, F[s][comp][y][x] out.
 *   F^a_s = -Ga_s psi_s(r) sum_{j in belt 1} w_j psi_s(r + c_j) c_j
 *   F^r_s = -Gr_s psi_s(r) sum_{j in belts 1, 2} p_j psi_s(r + c_j) c_j
 *   F^X_s = -(G_AB / rho0^2) rho_s(r) sum_{j in belt 1} w_j rho_s'(r + c_j) c_j
 */
void lbo_forces(const double *rho, int nx, int ny, const double *prm, double *F) {
  const double rho0 = prm[2], GAB = prm[3];
  const int couette = (int)prm[8];
  const size_t N = (size_t)nx * ny;
  double *psi = (double *)malloc(2 * N * sizeof(double));
  for (size_t k = 0; k < 2 * N; ++k) psi[k] = psi_of(rho[k], rho0);
#pragma omp parallel for schedule(static)
  for (int y = 0; y < ny; ++y)
    for (int s = 0; s < 2; ++s) {
      const int so = 1 - s;
      const double Ga = prm[4 + s], Gr = prm[6 + s];
      const double body = prm[10] * sin(2.0 * M_PI * prm[11] * (double)y / (double)ny);
      for (int x = 0; x < nx; ++x) {
        double sa_x = 0, sa_y = 0, sr_x = 0, sr_y = 0, sx_x = 0, sx_y = 0;
        for (int j = 1; j < 25; ++j) {
          const int yy = stencil_row(y + CYF[j], ny, couette);
          const int xx = wrap(x + CXF[j], nx);
          const double ps = psi[((size_t)s * ny + yy) * nx + xx];
          const double ro = rho[((size_t)so * ny + yy) * nx + xx];
          sa_x += wF(j) * ps * CXF[j];
          sa_y += wF(j) * ps * CYF[j];
          sr_x += pF(j) * ps * CXF[j];
          sr_y += pF(j) * ps * CYF[j];
          sx_x += wF(j) * ro * CXF[j];
          sx_y += wF(j) * ro * CYF[j];
        }
        const double pc = psi[((size_t)s * ny + y) * nx + x];
        const double rc = rho[((size_t)s * ny + y) * nx + x];
        const double Fa_x = -Ga * pc * sa_x, Fa_y = -Ga * pc * sa_y;
        const double Fr_x = -Gr * pc * sr_x, Fr_y = -Gr * pc * sr_y;
        const double Fx_x = -(GAB / (rho0 * rho0)) * rc * sx_x;
        const double Fx_y = -(GAB / (rho0 * rho0)) * rc * sx_y;
        const double Fb_x = rc * body;  /* Kolmogorov body force */
        F[(((size_t)s * 2 + 0) * ny + y) * nx + x] = Fa_x + Fr_x + Fx_x + Fb_x;
        F[(((size_t)s * 2 + 1) * ny + y) * nx + x] = Fa_y + Fr_y + Fx_y;
      }
    }
  free(psi);
}

/* Truncated equilibrium of Sec. II with cs2 = 1/3, written as in the paper. */
static double feq(int i, double rho, double vx, double vy) {
  const double cu = CX9[i] * vx + CY9[i] * vy;
  const double cc_xx = CX9[i] * CX9[i] - CS2, cc_yy = CY9[i] * CY9[i] - CS2;
  const double cc_xy = CX9[i] * CY9[i];
  const double quad = cc_xx * vx * vx + 2.0 * cc_xy * vx * vy + cc_yy * vy * vy;
  return w9(i) * rho * (1.0 + cu / CS2 + quad / (2.0 * CS2 * CS2));
}

/* Moments, forces, common velocity and the shifted velocities v_s of one
 * state.  Fills rho[2N], F[4N], v[4N] (v[s][comp][y][x]); returns the number of
 * (site, species) pairs with rho_s <= 0 (no shift applied there). */
static long macro_state(const double *f, int nx, int ny, const double *prm,
                        double *rho, double *F, double *v) {
  const size_t N = (size_t)nx * ny;
  const double tA = prm[0], tB = prm[1];
  lbo_densities(f, nx, ny, rho);
  lbo_forces(rho, nx, ny, prm, F);
  long bad = 0;
#pragma omp parallel for schedule(static) reduction(+ : bad)
  for (int y = 0; y < ny; ++y)
    for (int x = 0; x < nx; ++x) {
      const size_t r = (size_t)y * nx + x;
      double jx[2] = {0, 0}, jy[2] = {0, 0};
      for (int s = 0; s < 2; ++s)
        for (int i = 0; i < 9; ++i) {
          jx[s] += f[IDX(s, i, y, x, nx, ny)] * CX9[i];
          jy[s] += f[IDX(s, i, y, x, nx, ny)] * CY9[i];
        }
      const double rA = rho[r], rB = rho[N + r];
      const double den = rA / tA + rB / tB;
      const double ux = (jx[0] / tA + jx[1] / tB) / den;
      const double uy = (jy[0] / tA + jy[1] / tB) / den;
      for (int s = 0; s < 2; ++s) {
        const double ts = prm[s];
        const double rs = rho[s * N + r];
        double sx = 0.0, sy = 0.0;
        if (rs > 0.0) {
          sx = ts * F[(s * 2 + 0) * N + r] / rs;
          sy = ts * F[(s * 2 + 1) * N + r] / rs;
        } else {
          ++bad;
        }
        v[(s * 2 + 0) * N + r] = ux + sx;
        v[(s * 2 + 1) * N + r] = uy + sy;
      }
    }
  return bad;
}

/* One time step, f -> fn (separate buffers).  Returns the bad-density count. */
static long one_step(const double *f, double *fn, int nx, int ny, const double *prm,
                     double *rho, double *F, double *v, double *fpost) {
  const size_t N = (size_t)nx * ny;
  const int couette = (int)prm[8];
  const double U = prm[9];
  long bad = macro_state(f, nx, ny, prm, rho, F, v);
  /* pass 5-6: equilibrium and BGK relaxation, Eq. (be) */
#pragma omp parallel for schedule(static)
  for (int y = 0; y < ny; ++y)
    for (int s = 0; s < 2; ++s) {
      const double ts = prm[s];
      for (int x = 0; x < nx; ++x) {
        const size_t r = (size_t)y * nx + x;
        const double rs = rho[s * N + r];
        const double vx = v[(s * 2 + 0) * N + r], vy = v[(s * 2 + 1) * N + r];
        for (int i = 0; i < 9; ++i) {
          const size_t k = IDX(s, i, y, x, nx, ny);
          fpost[k] = f[k] - (f[k] - feq(i, rs, vx, vy)) / ts;
        }
      }
    }
  /* pass 7: streaming, with bounce-back at the moving walls */
#pragma omp parallel for schedule(static)
  for (int y = 0; y < ny; ++y)
    for (int s = 0; s < 2; ++s)
      for (int i = 0; i < 9; ++i)
        for (int x = 0; x < nx; ++x) {
          const double val = fpost[IDX(s, i, y, x, nx, ny)];
          const int yd = y + CY9[i];
          if (couette && (yd < 0 || yd >= ny)) {
            const double Uw = (yd >= ny) ? U : -U; /* wall velocity (Uw, 0) */
            const double rs = rho[s * N + (size_t)y * nx + x];
            fn[IDX(s, OPP9[i], y, x, nx, ny)] = val - 2.0 * w9(i) * rs * (CX9[i] * Uw) / CS2;
          } else {
            fn[IDX(s, i, wrap(yd, ny), wrap(x + CX9[i], nx), nx, ny)] = val;
          }
        }
  return bad;
}

/* Advance f (in place) by nsteps.  nthreads <= 0 keeps the OpenMP default.
 * Returns the accumulated count of (site, species, step) with rho_s <= 0, or
 * -1 on allocation failure. */
long lbo_step(double *f, int nx, int ny, const double *prm, long nsteps, int nthreads) {
#ifdef _OPENMP
  if (nthreads > 0) omp_set_num_threads(nthreads);
#else
  (void)nthreads;
#endif
  const size_t N = (size_t)nx * ny;
  double *fn = (double *)malloc(18 * N * sizeof(double));
  double *fpost = (double *)malloc(18 * N * sizeof(double));
  double *rho = (double *)malloc(2 * N * sizeof(double));
  double *F = (double *)malloc(4 * N * sizeof(double));
  double *v = (double *)malloc(4 * N * sizeof(double));
  if (!fn || !fpost || !rho || !F || !v) {
    free(fn); free(fpost); free(rho); free(F); free(v);
    return -1;
  }
  long bad = 0;
  for (long t = 0; t < nsteps; ++t) {
    bad += one_step(f, fn, nx, ny, prm, rho, F, v, fpost);
    memcpy(f, fn, 18 * N * sizeof(double));
  }
  free(fn); free(fpost); free(rho); free(F); free(v);
  return bad;
}

/* Threads the OpenMP runtime will use for the step passes. */
int lbo_max_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

/* ---- Observables of a state f(t) (FP64 sums in a fixed serial order).
 * mass[4]   = { sum rho_A, sum rho_B, P_x, P_y }, P = sum_s sum_i f_is c_i
 * stress[3] = { mean sigma_xy, wall_top, wall_bottom }
 *   sigma_xy(r) = -sum_s (1 - 1/(2 tau_s)) sum_i (f_is - f^eq_is) c_ix c_iy,
 *                 f^eq with the shifted velocity of the collision;
 *   wall_top    = -(1/nx) x-force on the top wall from the next streaming,
 *   wall_bottom = +(1/nx) x-force on the bottom wall from the next streaming;
 *   both are the shear stress at the wall (zero for periodic lattices).
 * rho_out[2][ny][nx] and u_out[2][ny][nx] (the paper's common velocity) are
 * optional (NULL skips). */
long lbo_observables(const double *f, int nx, int ny, const double *prm,
                     double *rho_out, double *u_out, double *stress, double *mass) {
  const size_t N = (size_t)nx * ny;
  const int couette = (int)prm[8];
  const double U = prm[9];
  double *rho = (double *)malloc(2 * N * sizeof(double));
  double *F = (double *)malloc(4 * N * sizeof(double));
  double *v = (double *)malloc(4 * N * sizeof(double));
  if (!rho || !F || !v) {
    free(rho); free(F); free(v);
    return -1;
  }
  long bad = macro_state(f, nx, ny, prm, rho, F, v);
  double MA = 0, MB = 0, Px = 0, Py = 0, sxy = 0, wt = 0, wb = 0;
  for (int y = 0; y < ny; ++y)
    for (int x = 0; x < nx; ++x) {
      const size_t r = (size_t)y * nx + x;
      double jx[2] = {0, 0}, jy[2] = {0, 0};
      for (int s = 0; s < 2; ++s) {
        const double ts = prm[s];
        const double rs = rho[s * N + r];
        const double vx = v[(s * 2 + 0) * N + r], vy = v[(s * 2 + 1) * N + r];
        double neq_xy = 0.0;
        for (int i = 0; i < 9; ++i) {
          const double fi = f[IDX(s, i, y, x, nx, ny)];
          jx[s] += fi * CX9[i];
          jy[s] += fi * CY9[i];
          neq_xy += (fi - feq(i, rs, vx, vy)) * CX9[i] * CY9[i];
          if (couette && (y + CY9[i] < 0 || y + CY9[i] >= ny)) {
            const double fp = fi - (fi - feq(i, rs, vx, vy)) / ts;
            const int top = (y + CY9[i] >= ny);
            const double Uw = top ? U : -U;
            const double back = fp - 2.0 * w9(i) * rs * (CX9[i] * Uw) / CS2;
            const double push = CX9[i] * (fp + back); /* x-momentum to the wall */
            if (top) wt -= push; else wb += push;
          }
        }
        sxy -= (1.0 - 1.0 / (2.0 * ts)) * neq_xy;
      }
      MA += rho[r];
      MB += rho[N + r];
      Px += jx[0] + jx[1];
      Py += jy[0] + jy[1];
      if (u_out) {
        const double tA = prm[0], tB = prm[1];
        const double den = rho[r] / tA + rho[N + r] / tB;
        u_out[r] = (jx[0] / tA + jx[1] / tB) / den;
        u_out[N + r] = (jy[0] / tA + jy[1] / tB) / den;
      }
    }
  if (rho_out) memcpy(rho_out, rho, 2 * N * sizeof(double));
  if (mass) {
    mass[0] = MA; mass[1] = MB; mass[2] = Px; mass[3] = Py;
  }
  if (stress) {
    stress[0] = sxy / (double)N;
    stress[1] = couette ? wt / nx : 0.0;
    stress[2] = couette ? wb / nx : 0.0;
  }
  free(rho); free(F); free(v);
  return bad;
}

/* ---- Shear diagnostics (Sec. VII).
 *   out[0] = U_k: the sine amplitude at the forcing wave number k of the
 *            line-averaged x velocity Ubar(y) = sum_x u_x(x, y) / nx, i.e.
 *            (2/ny) sum_y Ubar(y) sin(2 pi k y / ny); the response of Eq.
 *            (RESPONSE) is R = U_k / U0.  u is the paper's common velocity.
 *   out[1] = I_AB of Eq. (INDICATOR): -sum_{x,y} grad rho_A . grad rho_B, with
 *            central differences (rho(r + e) - rho(r - e)) / 2, periodic in x,
 *            and in y periodic or mirrored about the walls as the force stencil.
 * Returns the number of (site, species) pairs with rho_s <= 0. ---- */
long lbo_shear_diagnostics(const double *f, int nx, int ny, const double *prm, double *out) {
  const size_t N = (size_t)nx * ny;
  const int couette = (int)prm[8];
  double *rho = (double *)malloc(2 * N * sizeof(double));
  double *u = (double *)malloc(2 * N * sizeof(double));
  if (!rho || !u) {
    free(rho); free(u);
    return -1;
  }
  const long bad = lbo_observables(f, nx, ny, prm, rho, u, NULL, NULL);
  double uk = 0.0, iab = 0.0;
  for (int y = 0; y < ny; ++y) {
    double ubar = 0.0;
    for (int x = 0; x < nx; ++x) ubar += u[(size_t)y * nx + x];
    uk += (ubar / nx) * sin(2.0 * M_PI * prm[11] * (double)y / (double)ny);
    const int ym = stencil_row(y - 1, ny, couette), yp = stencil_row(y + 1, ny, couette);
    for (int x = 0; x < nx; ++x) {
      const int xm = wrap(x - 1, nx), xp = wrap(x + 1, nx);
      double g[2][2];
      for (int s = 0; s < 2; ++s) {
        const double *r = rho + (size_t)s * N;
        g[s][0] = 0.5 * (r[(size_t)y * nx + xp] - r[(size_t)y * nx + xm]);
        g[s][1] = 0.5 * (r[(size_t)yp * nx + x] - r[(size_t)ym * nx + x]);
      }
      iab -= g[0][0] * g[1][0] + g[0][1] * g[1][1];
    }
  }
  out[0] = 2.0 * uk / ny;
  out[1] = iab;
  free(rho); free(u);
  return bad;
}

/* ---- Ageing overlap (Sec. VII, Eq. (CORRE)).
 *   phi = rho_A - rho_B, the order parameter of the overlap.
 *   out[0] = sum_{x,y} phi(x,y; t_w) phi(x,y; t_w + dt_w)
 *   out[1] = sum_{x,y} phi(x,y; t_w)^2
 * of one realisation: f_w is the state at the waiting time t_w, f the state
 * dt_w steps later.  C(t_w, dt_w) of Eq. (CORRE) is the ratio of the two sums,
 * each averaged over an ensemble of realisations (the caller's average). ---- */
void lbo_phi_overlap(const double *f_w, const double *f, int nx, int ny, double *out) {
  const size_t N = (size_t)nx * ny;
  double num = 0.0, den = 0.0;
  for (size_t r = 0; r < N; ++r) {
    double rho_w[2] = {0.0, 0.0}, rho_t[2] = {0.0, 0.0};
    for (int s = 0; s < 2; ++s)
      for (int i = 0; i < 9; ++i) {
        rho_w[s] += f_w[(size_t)(s * 9 + i) * N + r];
        rho_t[s] += f[(size_t)(s * 9 + i) * N + r];
      }
    const double phi_w = rho_w[0] - rho_w[1];
    const double phi_t = rho_t[0] - rho_t[1];
    num += phi_w * phi_t;
    den += phi_w * phi_w;
  }
  out[0] = num;
  out[1] = den;
}

/* ---- Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random numbers:
 * as easy as 1, 2, 3", SC'11): ten rounds of two 32x32->64 multiplies with the
 * round keys bumped by the Weyl constants between rounds. ---- */
void lbo_philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2], uint32_t out[4]) {
  uint32_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
  uint32_t k0 = key_in[0], k1 = key_in[1];
  for (int round = 0; round < 10; ++round) {
    if (round > 0) {
      k0 += 0x9E3779B9u;
      k1 += 0xBB67AE85u;
    }
    const uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)c0;
    const uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)c2;
    const uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    const uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    const uint32_t n0 = hi1 ^ c1 ^ k0, n1 = lo1, n2 = hi0 ^ c3 ^ k1, n3 = lo0;
    c0 = n0; c1 = n1; c2 = n2; c3 = n3;
  }
  out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* ---- Seeded initial state: densities per site from one Philox block per
 * site (counter = site index y*nx + x, key = seed), then f_is = w_i rho_s at
 * zero velocity.  u_k = word_k * 2^-32 in [0, 1).
 *  kind 0 (uniform noise):  rho_A = init[0] + init[2] (2 u_1 - 1)
 *                           rho_B = init[1] + init[2] (2 u_2 - 1)
 *  kind 1 (Bernoulli mix):  u_0 < init[0] ? (rho_A, rho_B) = (init[1], init[2])
 *                                         : (init[2], init[1]);
 *                           then rho_A += init[3] u_1, rho_B += init[3] u_2.
 * ---- */
void lbo_init_densities(int nx, int ny, uint64_t seed, int kind, const double *init,
                        double *rho) {
  const size_t N = (size_t)nx * ny;
  const uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
  for (size_t site = 0; site < N; ++site) {
    const uint32_t ctr[4] = {(uint32_t)site, (uint32_t)((uint64_t)site >> 32), 0u, 0u};
    uint32_t w[4];
    lbo_philox4x32_10(ctr, key, w);
    const double u0 = (double)w[0] * 0x1p-32;
    const double u1 = (double)w[1] * 0x1p-32;
    const double u2 = (double)w[2] * 0x1p-32;
    double rA, rB;
    if (kind == 0) {
      rA = init[0] + init[2] * (2.0 * u1 - 1.0);
      rB = init[1] + init[2] * (2.0 * u2 - 1.0);
    } else {
      if (u0 < init[0]) {
        rA = init[1];
        rB = init[2];
      } else {
        rA = init[2];
        rB = init[1];
      }
      rA = rA + init[3] * u1;
      rB = rB + init[3] * u2;
    }
    rho[site] = rA;
    rho[N + site] = rB;
  }
}

void lbo_init(double *f, int nx, int ny, uint64_t seed, int kind, const double *init) {
  const size_t N = (size_t)nx * ny;
  double *rho = (double *)malloc(2 * N * sizeof(double));
  if (!rho) return;
  lbo_init_densities(nx, ny, seed, kind, init, rho);
  for (int s = 0; s < 2; ++s)
    for (int i = 0; i < 9; ++i)
      for (size_t site = 0; site < N; ++site)
        f[((size_t)(s * 9 + i)) * N + site] = w9(i) * rho[s * N + site];
  free(rho);
}

/* ======================================================================
 * N_s species (Sec. II: Eq. (be) and Eq. (FORCE) are written for species
 * s = 1..N_s with a symmetric cross-coupling matrix G_ss', s' != s).  The
 * same whole-lattice passes as above, for any number of species ns >= 1.
 *
 * Layout: f[((s*9 + i)*ny + y)*nx + x], s = 0..ns-1.
 * Parameter vector q[] (doubles):
 *   0 ns   1 rho0   2 boundary (0 periodic, 1 Couette)   3 U_wall
 *   4 g (Kolmogorov amplitude)   5 k (its wave number)
 *   6 .. 6+ns-1          tau_s
 *   6+ns .. 6+2ns-1      Ga_s   (G^a_s: belt 1, weights w)
 *   6+2ns .. 6+3ns-1     Gr_s   (G^r_s: belts 1 and 2, weights p)
 *   6+3ns .. 6+3ns+ns^2-1  G[s][s'] row-major (symmetric; diagonal unused)
 *
 *   F^X_s = -(1/rho0^2) rho_s(r) sum_{s' != s} G_ss' sum_{j in belt 1} w_j rho_s'(r + c_j) c_j
 * taken as a sum over s' (in increasing order) of the per-pair terms, so
 * that with ns = 2 every term is the two-species pass's own expression.
 * ====================================================================== */
#define QNS(q) ((int)(q)[0])
#define QTAU(q, s) ((q)[6 + (s)])
#define QGA(q, s) ((q)[6 + QNS(q) + (s)])
#define QGR(q, s) ((q)[6 + 2 * QNS(q) + (s)])
#define QG(q, s, t) ((q)[6 + 3 * QNS(q) + (s) * QNS(q) + (t)])

static inline size_t IDXN(int s, int i, int y, int x, int nx, int ny) {
  return (((size_t)(s * 9 + i) * (size_t)ny + (size_t)y) * (size_t)nx) + (size_t)x;
}

/* pass 1: rho[s][y][x] = sum_i f_is */
void lbo_densities_ns(const double *f, int ns, int nx, int ny, double *rho) {
#pragma omp parallel for schedule(static)
  for (int y = 0; y < ny; ++y)
    for (int s = 0; s < ns; ++s)
      for (int x = 0; x < nx; ++x) {
        double r = 0.0;
        for (int i = 0; i < 9; ++i) r += f[IDXN(s, i, y, x, nx, ny)];
        rho[((size_t)s * ny + y) * nx + x] = r;
      }
}

/* passes 2-3: psi of Eq. (PSI) and the forces of Eq. (FORCE); F[s][comp][y][x] */
void lbo_forces_ns(const double *rho, int nx, int ny, const double *q, double *F) {
  const int ns = QNS(q);
  const double rho0 = q[1];
  const int couette = (int)q[2];
  const size_t N = (size_t)nx * ny;
  double *psi = (double *)malloc((size_t)ns * N * sizeof(double));
  if (!psi) return;
  for (size_t k = 0; k < (size_t)ns * N; ++k) psi[k] = psi_of(rho[k], rho0);
#pragma omp parallel for schedule(static)
  for (int y = 0; y < ny; ++y) {
    double sxx[16], sxy[16]; /* belt-1 sums of the other species' densities (ns <= 16) */
    const double body = q[4] * sin(2.0 * M_PI * q[5] * (double)y / (double)ny);
    for (int s = 0; s < ns; ++s) {
      const double Ga = QGA(q, s), Gr = QGR(q, s);
      for (int x = 0; x < nx; ++x) {
        double sa_x = 0, sa_y = 0, sr_x = 0, sr_y = 0;
        for (int t = 0; t < ns; ++t) sxx[t] = sxy[t] = 0.0;
        for (int j = 1; j < 25; ++j) {
          const int yy = stencil_row(y + CYF[j], ny, couette);
          const int xx = wrap(x + CXF[j], nx);
          const double ps = psi[((size_t)s * ny + yy) * nx + xx];
          sa_x += wF(j) * ps * CXF[j];
          sa_y += wF(j) * ps * CYF[j];
          sr_x += pF(j) * ps * CXF[j];
          sr_y += pF(j) * ps * CYF[j];
          for (int t = 0; t < ns; ++t) {
            if (t == s) continue;
            const double ro = rho[((size_t)t * ny + yy) * nx + xx];
            sxx[t] += wF(j) * ro * CXF[j];
            sxy[t] += wF(j) * ro * CYF[j];
          }
        }
        const double pc = psi[((size_t)s * ny + y) * nx + x];
        const double rc = rho[((size_t)s * ny + y) * nx + x];
        const double Fa_x = -Ga * pc * sa_x, Fa_y = -Ga * pc * sa_y;
        const double Fr_x = -Gr * pc * sr_x, Fr_y = -Gr * pc * sr_y;
        double Fx_x = 0.0, Fx_y = 0.0;
        int first = 1;
        for (int t = 0; t < ns; ++t) {
          if (t == s) continue;
          const double G = QG(q, s, t);
          const double tx = -(G / (rho0 * rho0)) * rc * sxx[t];
          const double ty = -(G / (rho0 * rho0)) * rc * sxy[t];
          if (first) {
            Fx_x = tx;
            Fx_y = ty;
            first = 0;
          } else {
            Fx_x += tx;
            Fx_y += ty;
          }
        }
        const double Fb_x = rc * body;
        F[(((size_t)s * 2 + 0) * ny + y) * nx + x] = Fa_x + Fr_x + Fx_x + Fb_x;
        F[(((size_t)s * 2 + 1) * ny + y) * nx + x] = Fa_y + Fr_y + Fx_y;
      }
    }
  }
  free(psi);
}

/* moments, common velocity u = sum_s j_s/tau_s / sum_s rho_s/tau_s and the
 * shifted velocities v_s = u + tau_s F_s / rho_s (no shift where rho_s <= 0,
 * counted) */
static long macro_state_ns(const double *f, int nx, int ny, const double *q, double *rho,
                           double *F, double *v) {
  const int ns = QNS(q);
  const size_t N = (size_t)nx * ny;
  lbo_densities_ns(f, ns, nx, ny, rho);
  lbo_forces_ns(rho, nx, ny, q, F);
  long bad = 0;
#pragma omp parallel for schedule(static) reduction(+ : bad)
  for (int y = 0; y < ny; ++y)
    for (int x = 0; x < nx; ++x) {
      const size_t r = (size_t)y * nx + x;
      double den = 0.0, nux = 0.0, nuy = 0.0;
      for (int s = 0; s < ns; ++s) {
        double jx = 0.0, jy = 0.0;
        for (int i = 0; i < 9; ++i) {
          jx += f[IDXN(s, i, y, x, nx, ny)] * CX9[i];
          jy += f[IDXN(s, i, y, x, nx, ny)] * CY9[i];
        }
        const double ts = QTAU(q, s);
        if (s == 0) {
          den = rho[r] / ts;
          nux = jx / ts;
          nuy = jy / ts;
        } else {
          den += rho[s * N + r] / ts;
          nux += jx / ts;
          nuy += jy / ts;
        }
      }
      const double ux = nux / den, uy = nuy / den;
      for (int s = 0; s < ns; ++s) {
        const double ts = QTAU(q, s);
        const double rs = rho[s * N + r];
        double sx = 0.0, sy = 0.0;
        if (rs > 0.0) {
          sx = ts * F[(s * 2 + 0) * N + r] / rs;
          sy = ts * F[(s * 2 + 1) * N + r] / rs;
        } else {
          ++bad;
        }
        v[(s * 2 + 0) * N + r] = ux + sx;
        v[(s * 2 + 1) * N + r] = uy + sy;
      }
    }
  return bad;
}

/* one step f -> fn: BGK toward the shifted equilibrium (Eq. (be)), then
 * streaming with halfway bounce-back at moving walls */
static long one_step_ns(const double *f, double *fn, int nx, int ny, const double *q,
                        double *rho, double *F, double *v, double *fpost) {
  const int ns = QNS(q);
  const size_t N = (size_t)nx * ny;
  const int couette = (int)q[2];
  const double U = q[3];
  long bad = macro_state_ns(f, nx, ny, q, rho, F, v);
#pragma omp parallel for schedule(static)
  for (int y = 0; y < ny; ++y)
    for (int s = 0; s < ns; ++s) {
      const double ts = QTAU(q, s);
      for (int x = 0; x < nx; ++x) {
        const size_t r = (size_t)y * nx + x;
        const double rs = rho[s * N + r];
        const double vx = v[(s * 2 + 0) * N + r], vy = v[(s * 2 + 1) * N + r];
        for (int i = 0; i < 9; ++i) {
          const size_t k = IDXN(s, i, y, x, nx, ny);
          fpost[k] = f[k] - (f[k] - feq(i, rs, vx, vy)) / ts;
        }
      }
    }
#pragma omp parallel for schedule(static)
  for (int y = 0; y < ny; ++y)
    for (int s = 0; s < ns; ++s)
      for (int i = 0; i < 9; ++i)
        for (int x = 0; x < nx; ++x) {
          const double val = fpost[IDXN(s, i, y, x, nx, ny)];
          const int yd = y + CY9[i];
          if (couette && (yd < 0 || yd >= ny)) {
            const double Uw = (yd >= ny) ? U : -U;
            const double rs = rho[s * N + (size_t)y * nx + x];
            fn[IDXN(s, OPP9[i], y, x, nx, ny)] = val - 2.0 * w9(i) * rs * (CX9[i] * Uw) / CS2;
          } else {
            fn[IDXN(s, i, wrap(yd, ny), wrap(x + CX9[i], nx), nx, ny)] = val;
          }
        }
  return bad;
}

/* Advance f (in place) by nsteps; returns the bad-density count or -1. */
long lbo_step_ns(double *f, int nx, int ny, const double *q, long nsteps, int nthreads) {
#ifdef _OPENMP
  if (nthreads > 0) omp_set_num_threads(nthreads);
#else
  (void)nthreads;
#endif
  const int ns = QNS(q);
  if (ns < 1 || ns > 16) return -1;
  const size_t N = (size_t)nx * ny;
  double *fn = (double *)malloc((size_t)ns * 9 * N * sizeof(double));
  double *fpost = (double *)malloc((size_t)ns * 9 * N * sizeof(double));
  double *rho = (double *)malloc((size_t)ns * N * sizeof(double));
  double *F = (double *)malloc((size_t)ns * 2 * N * sizeof(double));
  double *v = (double *)malloc((size_t)ns * 2 * N * sizeof(double));
  if (!fn || !fpost || !rho || !F || !v) {
    free(fn); free(fpost); free(rho); free(F); free(v);
    return -1;
  }
  long bad = 0;
  for (long t = 0; t < nsteps; ++t) {
    bad += one_step_ns(f, fn, nx, ny, q, rho, F, v, fpost);
    memcpy(f, fn, (size_t)ns * 9 * N * sizeof(double));
  }
  free(fn); free(fpost); free(rho); free(F); free(v);
  return bad;
}

/* Observables of an ns-species state: mass[ns + 2] = {M_0 .. M_{ns-1}, P_x, P_y}
 * (P = sum_s sum_i f_is c_i), stress[3] = {mean sigma_xy, wall_top,
 * wall_bottom} as for two species.  Returns the bad-density count or -1. */
long lbo_observables_ns(const double *f, int nx, int ny, const double *q, double *stress,
                        double *mass) {
  const int ns = QNS(q);
  const size_t N = (size_t)nx * ny;
  const int couette = (int)q[2];
  const double U = q[3];
  double *rho = (double *)malloc((size_t)ns * N * sizeof(double));
  double *F = (double *)malloc((size_t)ns * 2 * N * sizeof(double));
  double *v = (double *)malloc((size_t)ns * 2 * N * sizeof(double));
  if (!rho || !F || !v) {
    free(rho); free(F); free(v);
    return -1;
  }
  long bad = macro_state_ns(f, nx, ny, q, rho, F, v);
  double Px = 0, Py = 0, sxy = 0, wt = 0, wb = 0;
  for (int s = 0; s < ns; ++s) mass[s] = 0.0;
  for (int y = 0; y < ny; ++y)
    for (int x = 0; x < nx; ++x) {
      const size_t r = (size_t)y * nx + x;
      for (int s = 0; s < ns; ++s) {
        const double ts = QTAU(q, s);
        const double rs = rho[s * N + r];
        const double vx = v[(s * 2 + 0) * N + r], vy = v[(s * 2 + 1) * N + r];
        double neq_xy = 0.0;
        for (int i = 0; i < 9; ++i) {
          const double fi = f[IDXN(s, i, y, x, nx, ny)];
          Px += fi * CX9[i];
          Py += fi * CY9[i];
          neq_xy += (fi - feq(i, rs, vx, vy)) * CX9[i] * CY9[i];
          if (couette && (y + CY9[i] < 0 || y + CY9[i] >= ny)) {
            const double fp = fi - (fi - feq(i, rs, vx, vy)) / ts;
            const int top = (y + CY9[i] >= ny);
            const double Uw = top ? U : -U;
            const double back = fp - 2.0 * w9(i) * rs * (CX9[i] * Uw) / CS2;
            const double push = CX9[i] * (fp + back);
            if (top) wt -= push; else wb += push;
          }
        }
        sxy -= (1.0 - 1.0 / (2.0 * ts)) * neq_xy;
        mass[s] += rs;
      }
    }
  mass[ns] = Px;
  mass[ns + 1] = Py;
  if (stress) {
    stress[0] = sxy / (double)N;
    stress[1] = couette ? wt / nx : 0.0;
    stress[2] = couette ? wb / nx : 0.0;
  }
  free(rho); free(F); free(v);
  return bad;
}

/* Seeded ns-species initial state at rest: species s of site r draws one
 * Philox4x32-10 block with counter (r_lo, r_hi, 1 + s, 0) and key (seed),
 * u = word_0 * 2^-32, rho_s = mean[s] + amp[s] (2u - 1), f_is = w_i rho_s. */
void lbo_init_ns(double *f, int ns, int nx, int ny, uint64_t seed, const double *mean,
                 const double *amp) {
  const size_t N = (size_t)nx * ny;
  const uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
  for (int s = 0; s < ns; ++s)
    for (size_t site = 0; site < N; ++site) {
      const uint32_t ctr[4] = {(uint32_t)site, (uint32_t)((uint64_t)site >> 32),
                               (uint32_t)(1 + s), 0u};
      uint32_t w[4];
      lbo_philox4x32_10(ctr, key, w);
      const double u = (double)w[0] * 0x1p-32;
      const double rs = mean[s] + amp[s] * (2.0 * u - 1.0);
      for (int i = 0; i < 9; ++i) f[(size_t)(s * 9 + i) * N + site] = w9(i) * rs;
    }
}
