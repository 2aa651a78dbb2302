/*
 * FP64 CPU oracle for the S1xR2 StePS hot path (arXiv 2602.20787).
 *
 * TEST INFRASTRUCTURE ONLY: loaded by the tests, the smoke check and the
 * benchmark's CPU-baseline leg, never by the product path. It shares no code
 * with the CUDA library. It is written to be read against the paper: plain
 * loops, FP64, no blocking or reordering beyond what the definitions state.
 * j-sums are Neumaier-compensated in double so that the result is the
 * definition up to rounding (no long double: it is software quad on aarch64).
 *
 * Readings of the paper taken here:
 *  - Eq. Force_spline_kernel: the "-\\-" inside the middle branch is a LaTeX
 *    line break, i.e. a single minus sign. h is the support radius (Newtonian
 *    for r >= h) and the pair uses h_i + h_j (eq. ComovingEquationsOfMotion).
 *  - Eq. ForceCylindrical: images n in [-Ncut, Ncut] with |r_z - n L| < Ncut L
 *    (strict), r_z the raw difference of z in [0, L).
 *  - Eq. F_horiz is garbled; it is re-derived as the mid-plane radial field of a
 *    homogeneous cylinder of radius R, z in [-Lw, Lw], Lw = Ncut L:
 *      F(rho) = 2 G rho0 Int_0^R [ 2 ln((sqrt(Lw^2+A)+Lw)/(sqrt(Lw^2+B)+Lw)) - ln(A/B) ] dY,
 *      A,B = R^2 + rho^2 +- 2 rho sqrt(R^2 - Y^2).
 *    It tends to eq. F_horiz_infty (-2 pi G rho0 rho) as Lw -> inf and is 0 at Lw = 0.
 *  - Eq. ComovingEquationsOfMotionCylindrical: the background term carries the
 *    same 1/a^3 as the pair term (rho0 is the comoving mean density), so that a
 *    homogeneous load feels no force in comoving coordinates (Sect. 2.1).
 *  - KDK in cosmic time (Sect. 2.1) with canonical momentum p = a^2 dx/dt:
 *    dp/dt = g/a, dx/dt = p/a^2 with g = a^3 (pair + background), which is the
 *    comoving EOM with the Hubble drag absorbed exactly. Kick factors are
 *    Int dt/a over each half step, the drift factor Int dt/a^2 over the step,
 *    all integrated together with a(t) by RK4 (Sect. 2.3) in two half steps.
 */
#include "steps_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define OR_PI 3.14159265358979323846

int32_t or_num_threads(void) {
#ifdef _OPENMP
  return (int32_t)omp_get_max_threads();
#else
  return 1;
#endif
}

/* ---------------------------------------------------------------------------
 * Eq. Force_spline_kernel: softened force magnitude F(r, h).
 * ------------------------------------------------------------------------- */
double or_spline_F(double r, double h) {
  if (r >= h) return 1.0 / (r * r);
  double h3 = h * h * h, h4 = h3 * h, h5 = h4 * h, h6 = h5 * h;
  double r2 = r * r, r3 = r2 * r, r4 = r3 * r;
  if (r < 0.5 * h) return 32.0 * r4 / h6 - 38.4 * r3 / h5 + 32.0 * r / (3.0 * h3);
  return -32.0 * r4 / (3.0 * h6) + 38.4 * r3 / h5 - 48.0 * r2 / h4 + 64.0 * r / (3.0 * h3) -
         1.0 / (15.0 * r2);
}

/* F(r, h) / r, written out so that it stays finite at r = 0 (value 32/(3h^3)). */
double or_spline_F_over_r(double r, double h) {
  if (r >= h) return 1.0 / (r * r * r);
  double h3 = h * h * h, h4 = h3 * h, h5 = h4 * h, h6 = h5 * h;
  double r2 = r * r, r3 = r2 * r;
  if (r < 0.5 * h) return 32.0 * r3 / h6 - 38.4 * r2 / h5 + 32.0 / (3.0 * h3);
  return -32.0 * r3 / (3.0 * h6) + 38.4 * r2 / h5 - 48.0 * r / h4 + 64.0 / (3.0 * h3) -
         1.0 / (15.0 * r3);
}

/* ---------------------------------------------------------------------------
 * Eq. ForceCylindrical per unit G: out = -sum_n F(|r_n|,h) r_n/|r_n|,
 * r_n = r - n L e_z, n in [-Ncut, Ncut], |r_z - n L| < Ncut L.
 * Returns the number of images used.
 * ------------------------------------------------------------------------- */
int or_image_force(double rx, double ry, double rz, double h, double L, int32_t n_cut,
                   double out[3]) {
  int count = 0;
  out[0] = out[1] = out[2] = 0.0;
  for (int n = -n_cut; n <= n_cut; ++n) {
    double dz = rz - (double)n * L;
    if (!(fabs(dz) < (double)n_cut * L)) continue;
    double r = sqrt(rx * rx + ry * ry + dz * dz);
    double f = or_spline_F_over_r(r, h);
    out[0] -= f * rx;
    out[1] -= f * ry;
    out[2] -= f * dz;
    ++count;
  }
  return count;
}

/* Neumaier compensated accumulation. */
typedef struct { double s, c; } or_sum;
static inline void or_add(or_sum* a, double v) {
  double t = a->s + v;
  if (fabs(a->s) >= fabs(v)) a->c += (a->s - t) + v;
  else a->c += (v - t) + a->s;
  a->s = t;
}

/* ---------------------------------------------------------------------------
 * Pair term of eq. ComovingEquationsOfMotionCylindrical times a^3:
 *   g_i = G sum_{j != i} m_j F_S1R2(x_i - x_j, h_i + h_j).
 * idx == NULL evaluates every i (ni must equal n); otherwise the listed i.
 * ------------------------------------------------------------------------- */
void or_pair_field(int64_t n, const double* x, const double* y, const double* z, const double* m,
                   const double* h, double G, double L, int32_t n_cut, int64_t ni,
                   const int64_t* idx, double* gx, double* gy, double* gz) {
#pragma omp parallel for schedule(dynamic, 4)
  for (int64_t q = 0; q < ni; ++q) {
    int64_t i = idx ? idx[q] : q;
    or_sum sx = {0, 0}, sy = {0, 0}, sz = {0, 0};
    for (int64_t j = 0; j < n; ++j) {
      if (j == i) continue;
      double f[3];
      or_image_force(x[i] - x[j], y[i] - y[j], z[i] - z[j], h[i] + h[j], L, n_cut, f);
      or_add(&sx, G * m[j] * f[0]);
      or_add(&sy, G * m[j] * f[1]);
      or_add(&sz, G * m[j] * f[2]);
    }
    gx[q] = sx.s + sx.c;
    gy[q] = sy.s + sy.c;
    gz[q] = sz.s + sz.c;
  }
}

/* ---------------------------------------------------------------------------
 * Background field (eq. F_horiz, re-derived; see header). The Y integral is
 * taken in theta with Y = R sin(theta), which removes the square-root endpoint
 * behaviour at Y = R; what is left is a log singularity at theta = 0 when
 * rho = R, which adaptive Gauss-Legendre handles (no endpoint evaluations).
 * ------------------------------------------------------------------------- */
static double or_cyl_integrand(double th, double rho, double R, double Lw) {
  /* A, B = R^2 + rho^2 +- 2 rho R cos(theta), written as (R +- rho)^2 -+ 4 rho R sin^2(theta/2)
   * so that B keeps full relative precision when rho is close to R. */
  double s2 = sin(0.5 * th);
  double q = 4.0 * rho * R * s2 * s2;
  double A = (R + rho) * (R + rho) - q;
  double B = (R - rho) * (R - rho) + q;
  double finite = 2.0 * log((sqrt(Lw * Lw + A) + Lw) / (sqrt(Lw * Lw + B) + Lw));
  double inf = log(A / B);
  return (finite - inf) * R * cos(th); /* dY = R cos(theta) dtheta */
}

static const double or_gl_x[8] = {-0.9602898564975363, -0.7966664774136267, -0.5255324099163290,
                                  -0.1834346424956498, 0.1834346424956498,  0.5255324099163290,
                                  0.7966664774136267,  0.9602898564975363};
static const double or_gl_w[8] = {0.1012285362903763, 0.2223810344533745, 0.3137066458778873,
                                  0.3626837833783620, 0.3626837833783620, 0.3137066458778873,
                                  0.2223810344533745, 0.1012285362903763};

/* 8-point Gauss-Legendre on [a, b]; *absint receives the same rule applied to |f|. */
static double or_gl8(double a, double b, double rho, double R, double Lw, double* absint) {
  double mid = 0.5 * (a + b), half = 0.5 * (b - a), s = 0.0, sa = 0.0;
  for (int k = 0; k < 8; ++k) {
    double f = or_cyl_integrand(mid + half * or_gl_x[k], rho, R, Lw);
    s += or_gl_w[k] * f;
    sa += or_gl_w[k] * fabs(f);
  }
  *absint = sa * half;
  return s * half;
}

/* Adaptive bisection. Tolerance: 1e-14 R per unit length of theta (total error
 * below 1e-14 R pi/2), floored at the rounding level of the rule itself so that
 * the recursion always ends; only an interval that touches the log
 * singularity at theta = 0 (rho = R) keeps splitting, so depth grows linearly. */
static double or_adapt(double a, double b, double whole, double rho, double R, double Lw,
                       int depth) {
  double m = 0.5 * (a + b), al, ar;
  double l = or_gl8(a, m, rho, R, Lw, &al), r = or_gl8(m, b, rho, R, Lw, &ar);
  double tol = 1e-14 * R * (b - a);
  double floor_ = 64.0 * 2.220446049250313e-16 * (al + ar);
  if (tol < floor_) tol = floor_;
  if (depth <= 0 || fabs(l + r - whole) <= tol) return l + r;
  return or_adapt(a, m, l, rho, R, Lw, depth - 1) + or_adapt(m, b, r, rho, R, Lw, depth - 1);
}

double or_cylinder_field(double varrho, double R, double Lw, double G, double rho0) {
  if (varrho <= 0.0) return 0.0;
  double a = 0.0, b = 0.5 * OR_PI, ab;
  double I = or_adapt(a, b, or_gl8(a, b, varrho, R, Lw, &ab), varrho, R, Lw, 60);
  return 2.0 * G * rho0 * I;
}

/* Background acceleration of eq. ComovingEquationsOfMotionCylindrical (times a^3):
 * -F_h(rho) along the radial unit vector (F_h < 0, so it points outward). */
void or_background_field(int64_t ni, const double* x, const double* y, double R, double Lw,
                         double G, double rho0, double* gx, double* gy) {
#pragma omp parallel for schedule(dynamic, 16)
  for (int64_t q = 0; q < ni; ++q) {
    double rho = sqrt(x[q] * x[q] + y[q] * y[q]);
    if (rho <= 0.0) { gx[q] = gy[q] = 0.0; continue; }
    double F = or_cylinder_field(rho, R, Lw, G, rho0);
    gx[q] = -F * x[q] / rho;
    gy[q] = -F * y[q] / rho;
  }
}

/* ---------------------------------------------------------------------------
 * Eqs. Friedmann, DEdensity, CPLw0wa. The DEdensity integral of the CPL w(a)
 * is elementary: Int_1^a (1 + w0 + wa (1 - a'))/a' da' = (1+w0+wa) ln a - wa (a-1).
 * ------------------------------------------------------------------------- */
double or_hubble(const or_cosmo* c, double a) {
  double Ok = 1.0 - c->Omega_m - c->Omega_r - c->Omega_L;
  double ode = c->Omega_L * exp(-3.0 * ((1.0 + c->w0 + c->wa) * log(a) - c->wa * (a - 1.0)));
  double E2 = c->Omega_r / (a * a * a * a) + c->Omega_m / (a * a * a) + Ok / (a * a) + ode;
  return c->H0 * sqrt(E2);
}

/* One RK4 step of the autonomous system y = (a, Int dt/a, Int dt/a^2). */
static void or_rk4_aug(const or_cosmo* c, double y[3], double dt) {
  double k[4][3], s[3];
  for (int st = 0; st < 4; ++st) {
    double f = (st == 0) ? 0.0 : (st == 3 ? 1.0 : 0.5);
    for (int q = 0; q < 3; ++q) s[q] = y[q] + (st == 0 ? 0.0 : f * dt * k[st - 1][q]);
    double a = s[0];
    k[st][0] = a * or_hubble(c, a);
    k[st][1] = 1.0 / a;
    k[st][2] = 1.0 / (a * a);
  }
  for (int q = 0; q < 3; ++q) y[q] += dt / 6.0 * (k[0][q] + 2.0 * k[1][q] + 2.0 * k[2][q] + k[3][q]);
}

double or_a_of_t_step(const or_cosmo* c, double a, double dt) {
  double y[3] = {a, 0.0, 0.0};
  or_rk4_aug(c, y, dt);
  return y[0];
}

void or_kdk_factors(const or_cosmo* c, double a, double dt, double* K1, double* D, double* K2,
                    double* a_next) {
  if (!c->comoving) {
    *K1 = 0.5 * dt; *K2 = 0.5 * dt; *D = dt; *a_next = 1.0;
    return;
  }
  double y1[3] = {a, 0.0, 0.0};
  or_rk4_aug(c, y1, 0.5 * dt);
  double y2[3] = {y1[0], 0.0, 0.0};
  or_rk4_aug(c, y2, 0.5 * dt);
  *K1 = y1[1];
  *K2 = y2[1];
  *D = y1[2] + y2[2];
  *a_next = y2[0];
}

/* ---------------------------------------------------------------------------
 * R^3 topology (Sect. 2.1, eq. NewtonianForce): the softened Newtonian pair
 * force with no periodic images, g_i = -G sum_{j != i} m_j F(|r|, h_i + h_j) r/|r|
 * with r = x_i - x_j, and the radial term +(4 pi G / 3) rho0 x that keeps a
 * comoving homogeneous ball from collapsing (read, like the cylinder's term,
 * with the same 1/a^3 as the pair term).
 * ------------------------------------------------------------------------- */
void or_pair_field_r3(int64_t n, const double* x, const double* y, const double* z, const double* m,
                      const double* h, double G, int64_t ni, const int64_t* idx, double* gx, double* gy,
                      double* gz) {
#pragma omp parallel for schedule(dynamic, 16)
  for (int64_t q = 0; q < ni; ++q) {
    int64_t i = idx ? idx[q] : q;
    or_sum sx = {0, 0}, sy = {0, 0}, sz = {0, 0};
    for (int64_t j = 0; j < n; ++j) {
      if (j == i) continue;
      double rx = x[i] - x[j], ry = y[i] - y[j], rz = z[i] - z[j];
      double r = sqrt(rx * rx + ry * ry + rz * rz);
      double f = -G * m[j] * or_spline_F_over_r(r, h[i] + h[j]);
      or_add(&sx, f * rx);
      or_add(&sy, f * ry);
      or_add(&sz, f * rz);
    }
    gx[q] = sx.s + sx.c;
    gy[q] = sy.s + sy.c;
    gz[q] = sz.s + sz.c;
  }
}

void or_background_sphere(int64_t ni, const double* x, const double* y, const double* z, double G, double rho0,
                          double* gx, double* gy, double* gz) {
  double c = 4.0 * OR_PI * G * rho0 / 3.0;
  for (int64_t i = 0; i < ni; ++i) {
    gx[i] = c * x[i];
    gy[i] = c * y[i];
    gz[i] = c * z[i];
  }
}

/* A field that could not be computed (out of memory) is NaN, which every
 * comparison rejects. */
static void or_fill_nan(int64_t n, double* gx, double* gy, double* gz) {
  for (int64_t i = 0; i < n; ++i) gx[i] = gy[i] = gz[i] = NAN;
}

/* Total comoving field g = a^3 (pair + background) at the current positions. */
static void or_total_field(int64_t n, const double* x, const double* y, const double* z,
                           const double* m, const double* h, double G, double L, int32_t n_cut,
                           double R_bg, double rho0, int32_t background, int32_t topology, double* gx,
                           double* gy, double* gz) {
  if (topology == 1) {
    or_pair_field_r3(n, x, y, z, m, h, G, n, NULL, gx, gy, gz);
    if (background != 3) return;
    double* b = (double*)malloc(sizeof(double) * 3 * (size_t)n);
    if (!b) { or_fill_nan(n, gx, gy, gz); return; }
    or_background_sphere(n, x, y, z, G, rho0, b, b + n, b + 2 * n);
    for (int64_t i = 0; i < n; ++i) { gx[i] += b[i]; gy[i] += b[n + i]; gz[i] += b[2 * n + i]; }
    free(b);
    return;
  }
  or_pair_field(n, x, y, z, m, h, G, L, n_cut, n, NULL, gx, gy, gz);
  if (background == 0) return;
  double* bx = (double*)malloc(sizeof(double) * (size_t)n);
  double* by = (double*)malloc(sizeof(double) * (size_t)n);
  if (!bx || !by) { free(bx); free(by); or_fill_nan(n, gx, gy, gz); return; }
  if (background == 1) {
    or_background_field(n, x, y, R_bg, (double)n_cut * L, G, rho0, bx, by);
  } else {
    /* eq. F_horiz_infty inside the cylinder; the infinite cylinder's exterior field outside */
    for (int64_t i = 0; i < n; ++i) {
      double rho = sqrt(x[i] * x[i] + y[i] * y[i]);
      double F = rho <= R_bg ? -2.0 * OR_PI * G * rho0 * rho
                             : -2.0 * OR_PI * G * rho0 * R_bg * R_bg / rho;
      bx[i] = rho > 0 ? -F * x[i] / rho : 0.0;
      by[i] = rho > 0 ? -F * y[i] / rho : 0.0;
    }
  }
  for (int64_t i = 0; i < n; ++i) { gx[i] += bx[i]; gy[i] += by[i]; }
  free(bx);
  free(by);
}

/* KDK leapfrog in cosmic time on (x, p), p = a^2 dx/dt. z is kept in [0, L). */
int or_kdk_topo(int64_t n, double* x, double* y, double* z, double* px, double* py, double* pz,
                const double* m, const double* h, double G, double L, int32_t n_cut, double R_bg,
                double rho0, int32_t background, int32_t topology, const or_cosmo* c, double* a, double* t,
                double dt, int32_t nsteps) {
  double* gx = (double*)malloc(sizeof(double) * (size_t)n);
  double* gy = (double*)malloc(sizeof(double) * (size_t)n);
  double* gz = (double*)malloc(sizeof(double) * (size_t)n);
  if (!gx || !gy || !gz) { free(gx); free(gy); free(gz); return -1; }
  or_total_field(n, x, y, z, m, h, G, L, n_cut, R_bg, rho0, background, topology, gx, gy, gz);
  for (int32_t s = 0; s < nsteps; ++s) {
    double K1, D, K2, an;
    or_kdk_factors(c, *a, dt, &K1, &D, &K2, &an);
    for (int64_t i = 0; i < n; ++i) {
      px[i] += gx[i] * K1; py[i] += gy[i] * K1; pz[i] += gz[i] * K1;
      x[i] += px[i] * D; y[i] += py[i] * D; z[i] += pz[i] * D;
      if (topology == 0) {
        z[i] -= L * floor(z[i] / L);
        if (z[i] >= L) z[i] -= L; /* floor rounding can leave z == L */
      }
    }
    or_total_field(n, x, y, z, m, h, G, L, n_cut, R_bg, rho0, background, topology, gx, gy, gz);
    for (int64_t i = 0; i < n; ++i) { px[i] += gx[i] * K2; py[i] += gy[i] * K2; pz[i] += gz[i] * K2; }
    *a = an;
    *t += dt;
  }
  free(gx); free(gy); free(gz);
  return 0;
}

int or_kdk(int64_t n, double* x, double* y, double* z, double* px, double* py, double* pz,
           const double* m, const double* h, double G, double L, int32_t n_cut, double R_bg,
           double rho0, int32_t background, const or_cosmo* c, double* a, double* t, double dt,
           int32_t nsteps) {
  return or_kdk_topo(n, x, y, z, px, py, pz, m, h, G, L, n_cut, R_bg, rho0, background, 0, c, a, t, dt,
                     nsteps);
}

/* ---------------------------------------------------------------------------
 * Diagnostics of a state (Sect. 1: in S1xR2 the axial momentum P_z and the
 * angular momentum L_z about the axis are conserved, by invariance under
 * translations along the axis and rotations about it). Given positions and
 * canonical momenta p = a^2 dx/dt at expansion factor a, plain sums over the
 * particles in index order with long double accumulators:
 *   out[0..2] = sum m p,  out[3] = L_z = sum m (x p_y - y p_x),
 *   out[4] = kinetic energy sum m |dx/dt|^2 / 2 = sum m |p|^2 / (2 a^4),
 *   out[5] = total mass sum m.
 * ------------------------------------------------------------------------- */
void or_diagnostics(int64_t n, const double* x, const double* y, const double* px, const double* py,
                    const double* pz, const double* m, double a, double out[6]) {
  long double P0 = 0.0L, P1 = 0.0L, P2 = 0.0L, Lz = 0.0L, K = 0.0L, M = 0.0L;
  for (int64_t i = 0; i < n; ++i) {
    const long double mi = m[i];
    P0 += mi * px[i];
    P1 += mi * py[i];
    P2 += mi * pz[i];
    Lz += mi * ((long double)x[i] * py[i] - (long double)y[i] * px[i]);
    const long double vx = (long double)px[i] / ((long double)a * a);
    const long double vy = (long double)py[i] / ((long double)a * a);
    const long double vz = (long double)pz[i] / ((long double)a * a);
    K += 0.5L * mi * (vx * vx + vy * vy + vz * vz);
    M += mi;
  }
  out[0] = (double)P0;
  out[1] = (double)P1;
  out[2] = (double)P2;
  out[3] = (double)Lz;
  out[4] = (double)K;
  out[5] = (double)M;
}

/* ---------------------------------------------------------------------------
 * Far-image tail of eq. ForceCylindrical for the learned surrogate.
 * In the wrapped frame dzw in [-L/2, L/2) the window of eq. ForceCylindrical
 * is the set of offsets o_k = dzw + k L with |o_k| < Ncut L. The near set is
 * |k| <= n0; the tail is the rest of the window. Returned per unit G:
 *   SR = sum_tail F(r_k,h)/r_k,  Sz = sum_tail o_k F(r_k,h)/r_k,
 * so that the tail force on i from j is -G m_j (dx SR, dy SR, Sz).
 * ------------------------------------------------------------------------- */
void or_tail_sums(double dR, double dzw, double h, double L, int32_t n_cut, int32_t n0, double* SR,
                  double* Sz) {
  double sr = 0.0, sz = 0.0;
  for (int k = -n_cut - 1; k <= n_cut + 1; ++k) {
    if (k >= -n0 && k <= n0) continue;
    double o = dzw + (double)k * L;
    if (!(fabs(o) < (double)n_cut * L)) continue;
    double r = sqrt(dR * dR + o * o);
    double f = or_spline_F_over_r(r, h);
    sr += f;
    sz += o * f;
  }
  *SR = sr;
  *Sz = sz;
}

/* ---------------------------------------------------------------------------
 * Surrogate MLP 3 -> 32 -> 32 -> 2, ReLU hidden activations, FP64.
 * Flat parameter layout: W1[32][3], b1[32], W2[32][32], b2[32], W3[2][32], b3[2].
 * ------------------------------------------------------------------------- */
#define OR_H 32
#define OR_NW (OR_H * 3 + OR_H + OR_H * OR_H + OR_H + 2 * OR_H + 2)

static void or_mlp_fwd_full(const double* w, const double* u, double* z1, double* a1, double* z2,
                            double* a2, double* y) {
  const double *W1 = w, *b1 = W1 + OR_H * 3, *W2 = b1 + OR_H, *b2 = W2 + OR_H * OR_H,
               *W3 = b2 + OR_H, *b3 = W3 + 2 * OR_H;
  for (int o = 0; o < OR_H; ++o) {
    double s = b1[o];
    for (int q = 0; q < 3; ++q) s += W1[o * 3 + q] * u[q];
    z1[o] = s;
    a1[o] = s > 0.0 ? s : 0.0;
  }
  for (int o = 0; o < OR_H; ++o) {
    double s = b2[o];
    for (int q = 0; q < OR_H; ++q) s += W2[o * OR_H + q] * a1[q];
    z2[o] = s;
    a2[o] = s > 0.0 ? s : 0.0;
  }
  for (int o = 0; o < 2; ++o) {
    double s = b3[o];
    for (int q = 0; q < OR_H; ++q) s += W3[o * OR_H + q] * a2[q];
    y[o] = s;
  }
}

void or_mlp_forward(const double* w, const double* u, double* y) {
  double z1[OR_H], a1[OR_H], z2[OR_H], a2[OR_H];
  or_mlp_fwd_full(w, u, z1, a1, z2, a2, y);
}

/* Loss = 1/(2 ns) sum_s sum_o (y_o(u_s) - t_so)^2 ; grad has OR_NW entries. */
double or_mlp_loss_grad(const double* w, int64_t ns, const double* u, const double* t,
                        double* grad) {
  const double *W2 = w + OR_H * 3 + OR_H, *W3 = W2 + OR_H * OR_H + OR_H;
  double *gW1 = grad, *gb1 = gW1 + OR_H * 3, *gW2 = gb1 + OR_H, *gb2 = gW2 + OR_H * OR_H,
         *gW3 = gb2 + OR_H, *gb3 = gW3 + 2 * OR_H;
  memset(grad, 0, sizeof(double) * OR_NW);
  double loss = 0.0;
  for (int64_t s = 0; s < ns; ++s) {
    double z1[OR_H], a1[OR_H], z2[OR_H], a2[OR_H], y[2], dy[2], d2[OR_H], d1[OR_H];
    const double* us = u + 3 * s;
    or_mlp_fwd_full(w, us, z1, a1, z2, a2, y);
    for (int o = 0; o < 2; ++o) {
      double e = y[o] - t[2 * s + o];
      loss += 0.5 * e * e;
      dy[o] = e / (double)ns;
    }
    for (int o = 0; o < 2; ++o) {
      gb3[o] += dy[o];
      for (int q = 0; q < OR_H; ++q) gW3[o * OR_H + q] += dy[o] * a2[q];
    }
    for (int q = 0; q < OR_H; ++q) {
      double g = dy[0] * W3[q] + dy[1] * W3[OR_H + q];
      d2[q] = z2[q] > 0.0 ? g : 0.0;
    }
    for (int o = 0; o < OR_H; ++o) {
      gb2[o] += d2[o];
      for (int q = 0; q < OR_H; ++q) gW2[o * OR_H + q] += d2[o] * a1[q];
    }
    for (int q = 0; q < OR_H; ++q) {
      double g = 0.0;
      for (int o = 0; o < OR_H; ++o) g += d2[o] * W2[o * OR_H + q];
      d1[q] = z1[q] > 0.0 ? g : 0.0;
    }
    for (int o = 0; o < OR_H; ++o) {
      gb1[o] += d1[o];
      for (int q = 0; q < 3; ++q) gW1[o * 3 + q] += d1[o] * us[q];
    }
  }
  return loss / (double)ns;
}

/* Adam (Kingma & Ba 2015), bias-corrected, step counted from 1. */
void or_adam_step(int64_t nw, double* w, const double* g, double* m1, double* m2, double lr,
                  double beta1, double beta2, double eps, int64_t step) {
  double c1 = 1.0 - pow(beta1, (double)step), c2 = 1.0 - pow(beta2, (double)step);
  for (int64_t k = 0; k < nw; ++k) {
    m1[k] = beta1 * m1[k] + (1.0 - beta1) * g[k];
    m2[k] = beta2 * m2[k] + (1.0 - beta2) * g[k] * g[k];
    w[k] -= lr * (m1[k] / c1) / (sqrt(m2[k] / c2) + eps);
  }
}

/* ---------------------------------------------------------------------------
 * Learned far-image surrogate. The paper has no such method: this is the
 * project's definition of the surrogate tail, written here plainly in FP64 so
 * that the CUDA kernel's evaluation of the same definition can be checked.
 * Units: lengths in units of L (period 1); dz is the wrapped separation in
 * [-1/2, 1/2]; near images are |k| <= n0, the tail is the rest of the window.
 *
 * Base: each side of the tail is a run of unit cells centred on the images;
 * the image sum over a run is its continuum integral minus (1/24)[f'(end) -
 * f'(start)] (midpoint Euler-Maclaurin, first correction), with
 *   f(z) = (R^2 + z^2)^(-3/2)  for SR,   z f(z)  for SZ.
 * Envelope: e = 1 / (R^2 + (n0 + 1/2 + |dz|)^2), ER = e^3, EZ = e^(5/2).
 * Inputs: u = (2 min(R, dR_max)/dR_max - 1, 4|dz| - 1, 2 min(h, n0+1/2)/(n0+1/2) - 1).
 * ------------------------------------------------------------------------- */
static void or_side_integrals(double R2, double lo, double hi, double* IR, double* IZ, double* dR_lo,
                              double* dR_hi, double* dZ_lo, double* dZ_hi) {
  double rl = sqrt(R2 + lo * lo), rh = sqrt(R2 + hi * hi);
  /* Int_lo^hi (R^2+z^2)^-1.5 dz = [z / (R^2 sqrt(R^2+z^2))], in a form without
   * cancellation at small R: (hi^2 - lo^2) / (rl rh (hi rl + lo rh)) */
  *IR = (hi * hi - lo * lo) / (rl * rh * (hi * rl + lo * rh));
  /* Int_lo^hi z (R^2+z^2)^-1.5 dz = 1/rl - 1/rh */
  *IZ = 1.0 / rl - 1.0 / rh;
  /* derivatives of f and z f */
  *dR_lo = -3.0 * lo / pow(rl, 5.0);
  *dR_hi = -3.0 * hi / pow(rh, 5.0);
  *dZ_lo = 1.0 / pow(rl, 3.0) - 3.0 * lo * lo / pow(rl, 5.0);
  *dZ_hi = 1.0 / pow(rh, 3.0) - 3.0 * hi * hi / pow(rh, 5.0);
}

void or_tail_base(double dR, double adz, int32_t n_cut, int32_t n0, double* BR, double* BZ) {
  double R2 = dR * dR, A = n0 + 0.5;
  /* images dz + k with |dz + k| < n_cut: for dz >= 0 the positive side ends at
   * k = n_cut - 1, the negative side at k = -n_cut if dz > 0, else -(n_cut - 1) */
  int kpos = n_cut - 1, kneg = adz > 0.0 ? n_cut : n_cut - 1;
  double IR, IZ, a, b, c, d;
  /* positive side: cells [A + adz, kpos + 1/2 + adz] */
  or_side_integrals(R2, A + adz, kpos + 0.5 + adz, &IR, &IZ, &a, &b, &c, &d);
  double sr = IR - (b - a) / 24.0, sz = IZ - (d - c) / 24.0;
  /* negative side mirrored to z' = -z > 0: cells [A - adz, kneg + 1/2 - adz]; z f is odd */
  or_side_integrals(R2, A - adz, kneg + 0.5 - adz, &IR, &IZ, &a, &b, &c, &d);
  sr += IR - (b - a) / 24.0;
  sz -= IZ - (d - c) / 24.0;
  *BR = sr;
  *BZ = sz;
}

void or_tail_envelope(double dR, double adz, int32_t n0, double* ER, double* EZ) {
  double A = n0 + 0.5, e = 1.0 / (dR * dR + (A + adz) * (A + adz));
  *ER = e * e * e;
  *EZ = e * e * sqrt(e);
}

void or_surrogate_inputs(double dR, double adz, double h, int32_t n0, double dR_max, double u[3]) {
  double A = n0 + 0.5;
  u[0] = 2.0 * (dR < dR_max ? dR : dR_max) / dR_max - 1.0;
  u[1] = 4.0 * adz - 1.0;
  u[2] = 2.0 * (h < A ? h : A) / A - 1.0;
}

void or_tail_surrogate(double dR, double dz, double h, const double* w, const or_surr_cfg* c, double* SR,
                       double* SZ) {
  double adz = fabs(dz), BR, BZ, ER, EZ, u[3], y[2];
  if (c->n_cut == 0) /* the infinite window (Ncut -> infinity) */
    or_tail_base_inf(dR, adz, c->n0, &BR, &BZ);
  else
    or_tail_base(dR, adz, c->n_cut, c->n0, &BR, &BZ);
  or_tail_envelope(dR, adz, c->n0, &ER, &EZ);
  or_surrogate_inputs(dR, adz, h, c->n0, c->dR_max, u);
  or_mlp_forward(w, u, y);
  double sr = BR + ER * (y[0] * c->out_sc[0] + c->out_mu[0]);
  double sz = BZ + EZ * (y[1] * c->out_sc[1] + c->out_mu[1]);
  double sg = dz > 0.0 ? 1.0 : (dz < 0.0 ? -1.0 : 0.0);
  sz *= sg;
  /* tail images inside the softening support: the surrogate is Newtonian there;
   * replace 1/r^3 by F(r,h)/r exactly (an infinite window: every k with |o| < h) */
  int kmax = c->n_cut > 0 ? c->n_cut + 1 : (int)ceil(h) + 2;
  for (int k = -kmax; k <= kmax; ++k) {
    if (k >= -c->n0 && k <= c->n0) continue;
    double o = dz + (double)k;
    if (c->n_cut > 0 && !(fabs(o) < (double)c->n_cut)) continue;
    double r = sqrt(dR * dR + o * o);
    if (r >= h) continue;
    double d = or_spline_F_over_r(r, h) - 1.0 / (r * r * r);
    sr += d;
    sz += o * d;
  }
  *SR = sr;
  *SZ = sz;
}

/* Pair term with a modelled tail: near images (|k| <= n0 in the wrapped frame)
 * summed exactly, far tail from tail(dR, dz, h, ctx). */
typedef void (*or_tail_fn)(double dR, double dz, double h, const void* ctx, double* SR, double* SZ);

static void or_pair_field_with_tail(int64_t n, const double* x, const double* y, const double* z,
                                    const double* m, const double* h, double G, double L, int32_t n0,
                                    or_tail_fn tail, const void* ctx, int64_t ni, const int64_t* idx,
                                    double* gx, double* gy, double* gz) {
#pragma omp parallel for schedule(dynamic, 4)
  for (int64_t q = 0; q < ni; ++q) {
    int64_t i = idx ? idx[q] : q;
    or_sum sx = {0, 0}, sy = {0, 0}, sz = {0, 0};
    for (int64_t j = 0; j < n; ++j) {
      if (j == i) continue;
      double dx = (x[i] - x[j]) / L, dy = (y[i] - y[j]) / L, rz = (z[i] - z[j]) / L;
      double dzw = rz - floor(rz + 0.5);
      double hh = (h[i] + h[j]) / L, dR = sqrt(dx * dx + dy * dy);
      double sr = 0.0, szz = 0.0;
      for (int k = -n0; k <= n0; ++k) {
        double o = dzw + (double)k;
        double f = or_spline_F_over_r(sqrt(dR * dR + o * o), hh);
        sr += f;
        szz += o * f;
      }
      double tr, tz;
      tail(dR, dzw, hh, ctx, &tr, &tz);
      sr += tr;
      szz += tz;
      /* lengths were in units of L: F/r scales as 1/L^3, the vector as L */
      or_add(&sx, -G * m[j] * dx * sr / (L * L));
      or_add(&sy, -G * m[j] * dy * sr / (L * L));
      or_add(&sz, -G * m[j] * szz / (L * L));
    }
    gx[q] = sx.s + sx.c;
    gy[q] = sy.s + sy.c;
    gz[q] = sz.s + sz.c;
  }
}

typedef struct {
  const double* w;
  const or_surr_cfg* c;
} or_surr_ctx;

static void or_tail_surrogate_cb(double dR, double dz, double h, const void* ctx, double* SR, double* SZ) {
  const or_surr_ctx* s = (const or_surr_ctx*)ctx;
  or_tail_surrogate(dR, dz, h, s->w, s->c, SR, SZ);
}

void or_pair_field_surrogate(int64_t n, const double* x, const double* y, const double* z, const double* m,
                             const double* h, double G, double L, const double* w, const or_surr_cfg* c,
                             int64_t ni, const int64_t* idx, double* gx, double* gy, double* gz) {
  or_surr_ctx s = {w, c};
  or_pair_field_with_tail(n, x, y, z, m, h, G, L, c->n0, or_tail_surrogate_cb, &s, ni, idx, gx, gy, gz);
}

/* ---------------------------------------------------------------------------
 * Ncut -> infinity (Sect. 2.2: the window grows without bound and the
 * background becomes eq. F_horiz_infty): the whole periodic line of images.
 * Images |k| <= OR_KINF are summed exactly (softened); beyond them, on each
 * side, the continuum integral over the unit cells from K + 1/2 (Newtonian,
 * since h << K). The midpoint rule's error there is O(f'(K)) ~ 1/(8 K^4).
 * Returned per unit G for the images with |k| > n0 (n0 = -1: every image):
 *   SR = sum F(r_k,h)/r_k,  SZ = sum o_k F(r_k,h)/r_k,  o_k = dzw + k.
 * ------------------------------------------------------------------------- */
#define OR_KINF 512

void or_image_sums_inf(double dR, double dzw, double h, int32_t n0, double* SR, double* SZ) {
  double R2 = dR * dR;
  or_sum sr = {0, 0}, sz = {0, 0};
  for (int k = -OR_KINF; k <= OR_KINF; ++k) {
    if (k >= -n0 && k <= n0) continue;
    double o = dzw + (double)k;
    double f = or_spline_F_over_r(sqrt(R2 + o * o), h);
    or_add(&sr, f);
    or_add(&sz, o * f);
  }
  /* cells [top, inf) and, mirrored, [bot, inf): Int dx/(R2+x^2)^1.5 from a to inf
   * = 1/(r (r + a)), Int x dx/(...)^1.5 = 1/r (r = sqrt(R2 + a^2)), plus the near
   * end's Euler-Maclaurin term f'(a)/24 of the unit cells (f' = -3 a / r^5 and
   * (x f)' = 1/r^3 - 3 a^2 / r^5); the z part of the mirrored side is negative */
  double top = dzw + OR_KINF + 0.5, bot = -(dzw - OR_KINF - 0.5);
  double rt = sqrt(R2 + top * top), rb = sqrt(R2 + bot * bot);
  double it = 1.0 / rt, ib = 1.0 / rb, it5 = it * it * it * it * it, ib5 = ib * ib * ib * ib * ib;
  or_add(&sr, 1.0 / (rt * (rt + top)) - 3.0 * top * it5 / 24.0);
  or_add(&sr, 1.0 / (rb * (rb + bot)) - 3.0 * bot * ib5 / 24.0);
  or_add(&sz, it + (it * it * it - 3.0 * top * top * it5) / 24.0);
  or_add(&sz, -(ib + (ib * ib * ib - 3.0 * bot * bot * ib5) / 24.0));
  *SR = sr.s + sr.c;
  *SZ = sz.s + sz.c;
}

/* ---------------------------------------------------------------------------
 * Ewald summation of the infinite periodic line (Sect. 2.3, eqs.
 * cylindricalEwaldSplit, EwaldRealSum, EwaldRecSum and the m = 0 term), in
 * units of L (period 1), returning the sums of the images |k| > n0 in the
 * convention of or_image_sums_inf (point masses: force -G m (dR SR, SZ)).
 * The split parameter alpha is in units of 1/L.
 *   Real space (eq. EwaldRealSum): an image at distance r contributes
 *     [erfc(a r) + (2 a r / sqrt(pi)) exp(-a^2 r^2)] / r^3 = 1/r^3 - a^3 E(a r),
 *     E(x) = [erf(x) - (2 x / sqrt(pi)) exp(-x^2)] / x^3,
 *   summed over |n| <= nmax. The images |n| <= n0 are left out of the tail, so
 *   for them only -a^3 E(a r) remains, which is finite at r = 0 (E(0) =
 *   4 / (3 sqrt(pi))); E comes from its series below x = 0.25.
 *   Fourier space (eq. EwaldRecSum): mode k = 2 pi m of the screened line has
 *   the potential -2 cos(k z) B(k, rho), with the kernel re-derived: writing
 *   erf(a r)/r = (2/sqrt(pi)) Int_0^a exp(-r^2 s^2) ds and integrating along z,
 *     B(k, rho) = Int_0^{a^2} exp(-rho^2 t - k^2 / (4t)) dt / t,
 *   which tends to 2 K0(k rho) as a grows. The printed eq. Bkernel tends to
 *   2 exp(-k rho) instead, the kernel of a doubly periodic slab. The sums get
 *     SR += 4 cos(k z) J(k, rho), J = Int_0^{a^2} exp(-rho^2 t - k^2/(4t)) dt,
 *     SZ += 2 k sin(k z) B(k, rho),
 *   both integrals taken in s = ln t with composite 8-point Gauss-Legendre.
 *   m = 0: the line's mean radial field, SR += 2 (1 - exp(-a^2 rho^2)) / rho^2.
 * ------------------------------------------------------------------------- */
static double or_ewald_E(double x) {
  const double sqpi = 1.7724538509055160273;
  if (x < 0.25) {
    /* (2/sqrt(pi)) sum_{n>=1} (-1)^(n+1) 2n x^(2n-2) / (n! (2n+1)) */
    double x2 = x * x, term = 1.0, sum = 0.0, fact = 1.0;
    for (int n = 1; n <= 12; ++n) {
      fact *= (double)n;
      sum += ((n % 2) ? 1.0 : -1.0) * 2.0 * n * term / (fact * (2.0 * n + 1.0));
      term *= x2;
    }
    return 2.0 / sqpi * sum;
  }
  return (erf(x) - 2.0 * x / sqpi * exp(-x * x)) / (x * x * x);
}

/* J (with_t = 0) or B (with_t = 1) of the Fourier kernel: Int over s = ln t from
 * ln(k^2 / 300) (where exp(-k^2 / (4t)) < e^-75) to ln(a^2) */
static double or_ewald_mode_integral(double k, double rho, double a, int with_t) {
  const double s_hi = log(a * a), s_lo = log(k * k / 300.0);
  if (s_lo >= s_hi) return 0.0;
  const int panels = 256;
  const double h = (s_hi - s_lo) / panels;
  double tot = 0.0;
  for (int p = 0; p < panels; ++p) {
    const double mid = s_lo + (p + 0.5) * h, half = 0.5 * h;
    double acc = 0.0;
    for (int q = 0; q < 8; ++q) {
      const double sv = mid + half * or_gl_x[q];
      const double t = exp(sv);
      const double g = exp(-rho * rho * t - k * k / (4.0 * t));
      acc += or_gl_w[q] * (with_t ? g : g * t);
    }
    tot += acc * half;
  }
  return tot;
}

void or_ewald_tail(double dR, double dzw, int32_t n0, double alpha, int32_t nmax, int32_t mmax, double* SR,
                   double* SZ) {
  const double R2 = dR * dR, a = alpha, a3 = a * a * a;
  or_sum sr = {0, 0}, sz = {0, 0};
  for (int k = -nmax; k <= nmax; ++k) {
    const double o = dzw + (double)k, r = sqrt(R2 + o * o);
    const double screened = -a3 * or_ewald_E(a * r);
    const double f = (k >= -n0 && k <= n0) ? screened : 1.0 / (r * r * r) + screened;
    or_add(&sr, f);
    or_add(&sz, o * f);
  }
  const double two_pi = 6.283185307179586477;
  for (int m = 1; m <= mmax; ++m) {
    const double k = two_pi * m;
    or_add(&sr, 4.0 * cos(k * dzw) * or_ewald_mode_integral(k, dR, a, 0));
    or_add(&sz, 2.0 * k * sin(k * dzw) * or_ewald_mode_integral(k, dR, a, 1));
  }
  const double y = a * a * R2;
  or_add(&sr, y > 0 ? -2.0 * a * a * expm1(-y) / y : 2.0 * a * a);
  /* the images |k| > n0 that the real-space sum missed are screened away */
  *SR = sr.s + sr.c;
  *SZ = sz.s + sz.c;
}

/* Pair term with the infinite window: a_i = -G sum_j m_j (dx SR, dy SR, SZ)/L^2 */
void or_pair_field_inf(int64_t n, const double* x, const double* y, const double* z, const double* m,
                       const double* h, double G, double L, int64_t ni, const int64_t* idx, double* gx,
                       double* gy, double* gz) {
#pragma omp parallel for schedule(dynamic, 4)
  for (int64_t q = 0; q < ni; ++q) {
    int64_t i = idx ? idx[q] : q;
    or_sum sx = {0, 0}, sy = {0, 0}, sz = {0, 0};
    for (int64_t j = 0; j < n; ++j) {
      if (j == i) continue;
      double dx = (x[i] - x[j]) / L, dy = (y[i] - y[j]) / L, rz = (z[i] - z[j]) / L;
      double dzw = rz - floor(rz + 0.5);
      double sr, szz;
      or_image_sums_inf(sqrt(dx * dx + dy * dy), dzw, (h[i] + h[j]) / L, -1, &sr, &szz);
      or_add(&sx, -G * m[j] * dx * sr / (L * L));
      or_add(&sy, -G * m[j] * dy * sr / (L * L));
      or_add(&sz, -G * m[j] * szz / (L * L));
    }
    gx[q] = sx.s + sx.c;
    gy[q] = sy.s + sy.c;
    gz[q] = sz.s + sz.c;
  }
}

/* Continuum base of the infinite tail beyond |k| <= n0 (the order-1
 * Euler-Maclaurin form of or_tail_base with both far ends at infinity): per
 * side the integral over the cells [A +- |dz|, inf) minus 1/24 of the near
 * end's derivative, A = n0 + 1/2. */
void or_tail_base_inf(double dR, double adz, int32_t n0, double* BR, double* BZ) {
  double R2 = dR * dR, A = n0 + 0.5, lo[2] = {A + adz, A - adz}, br[2], bz[2];
  for (int s = 0; s < 2; ++s) {
    double l = lo[s], r = sqrt(R2 + l * l), il = 1.0 / r, il2 = il * il, il5 = il2 * il2 * il;
    /* f = (x^2+R2)^-1.5: Int = 1/(r (r + l)); f' = -3 x il^5; (x f)' = il^3 - 3 x^2 il^5 */
    br[s] = 1.0 / (r * (r + l)) - 3.0 * l * il5 / 24.0;
    bz[s] = il + (il2 * il - 3.0 * l * l * il5) / 24.0;
  }
  *BR = br[0] + br[1];
  *BZ = bz[0] - bz[1];
}
/* ---------------------------------------------------------------------------
 * Correction-table tail (Sect. 2.3, eq. S1R2EwaldCorrectionTable: a 2D table of
 * the periodic images beyond the nearest, read by cloud-in-cell interpolation
 * during the run), restated for the windowed sum beyond the near images
 * |k| <= n0 and for point masses. The tabulated quantity is the residual of the
 * tail over the continuum base in envelope units,
 *   r = ((SR - BR) / ER, (SZ - BZ) / EZ)   at dz = +|dz| (SZ odd in dz),
 * at nodes dR_i = i dR_max / (nx - 1), |dz|_j = j / (2 (ny - 1)). The tail at
 * (dR, dz) is B + E * bilinear(r), with dR beyond dR_max read on the last
 * column, plus the exact spline correction of tail images inside the
 * softening support (the table is Newtonian), as for the surrogate.
 * ------------------------------------------------------------------------- */
/* The frame a table is stored in: the residual over the continuum base in
 * envelope units for n0 >= 1; for n0 = 0 (the paper's table over the nearest
 * image alone, D = F_S1xR2 - F_R3(nearest)) the base's near end would reach the
 * pair itself at |dz| = 1/2, so that table holds the tail sums themselves (no
 * base, unit envelope). */
static void or_table_frame(double dR, double adz, int32_t n_cut, int32_t n0, double* BR, double* BZ, double* ER,
                           double* EZ) {
  if (n0 == 0) {
    *BR = *BZ = 0.0;
    *ER = *EZ = 1.0;
    return;
  }
  if (n_cut == 0)
    or_tail_base_inf(dR, adz, n0, BR, BZ);
  else
    or_tail_base(dR, adz, n_cut, n0, BR, BZ);
  or_tail_envelope(dR, adz, n0, ER, EZ);
}

void or_tail_residual(double dR, double adz, int32_t n_cut, int32_t n0, double r[2]) {
  double SR, SZ, BR, BZ, ER, EZ;
  if (n_cut == 0) /* infinite window */
    or_image_sums_inf(dR, adz, 0.0, n0, &SR, &SZ);
  else
    or_tail_sums(dR, adz, 0.0, 1.0, n_cut, n0, &SR, &SZ);
  or_table_frame(dR, adz, n_cut, n0, &BR, &BZ, &ER, &EZ);
  r[0] = (SR - BR) / ER;
  r[1] = (SZ - BZ) / EZ;
}

void or_tail_table_build(const or_table_cfg* c, double* tab) {
#pragma omp parallel for schedule(dynamic, 1)
  for (int j = 0; j < c->ny; ++j)
    for (int i = 0; i < c->nx; ++i)
      or_tail_residual(c->dR_max * i / (c->nx - 1), 0.5 * j / (c->ny - 1), c->n_cut, c->n0,
                       tab + 2 * ((size_t)j * c->nx + i));
}

/* TSC read: in node units x, the nearest node i = round(x) and d = x - i carry
 * the triangular-shaped-cloud weights (1/2 - d)^2 / 2, 3/4 - d^2, (1/2 + d)^2 / 2
 * on nodes i - 1, i, i + 1 (the overlap of a unit-width triangle cloud centred
 * at x with each node's cell), one factor per axis; a node outside the table
 * takes the value of the nearest edge node. */
static void or_tsc_weights(double x, int n, int idx[3], double w[3]) {
  int i = (int)floor(x + 0.5);
  double d = x - i;
  w[0] = 0.5 * (0.5 - d) * (0.5 - d);
  w[1] = 0.75 - d * d;
  w[2] = 0.5 * (0.5 + d) * (0.5 + d);
  for (int k = 0; k < 3; ++k) {
    int q = i - 1 + k;
    idx[k] = q < 0 ? 0 : (q > n - 1 ? n - 1 : q);
  }
}

static void or_tail_table_read_tsc(const double* tab, const or_table_cfg* c, double fx, double fy, double r[2]) {
  int ix[3], iy[3];
  double wx[3], wy[3];
  or_tsc_weights(fx, c->nx, ix, wx);
  or_tsc_weights(fy, c->ny, iy, wy);
  for (int q = 0; q < 2; ++q) {
    double acc = 0.0;
    for (int b = 0; b < 3; ++b)
      for (int a = 0; a < 3; ++a) acc += wx[a] * wy[b] * tab[2 * ((size_t)iy[b] * c->nx + ix[a]) + q];
    r[q] = acc;
  }
}

void or_tail_table_read(const double* tab, const or_table_cfg* c, double dR, double adz, double r[2]) {
  double fx = (dR < c->dR_max ? dR : c->dR_max) / c->dR_max * (c->nx - 1);
  double fy = adz / 0.5 * (c->ny - 1);
  if (c->read == OR_TABLE_TSC) {
    or_tail_table_read_tsc(tab, c, fx, fy, r);
    return;
  }
  int i = (int)floor(fx), j = (int)floor(fy);
  if (i > c->nx - 2) i = c->nx - 2;
  if (j > c->ny - 2) j = c->ny - 2;
  double a = fx - i, b = fy - j;
  for (int q = 0; q < 2; ++q) {
    double t00 = tab[2 * ((size_t)j * c->nx + i) + q], t10 = tab[2 * ((size_t)j * c->nx + i + 1) + q];
    double t01 = tab[2 * ((size_t)(j + 1) * c->nx + i) + q], t11 = tab[2 * ((size_t)(j + 1) * c->nx + i + 1) + q];
    r[q] = (1 - a) * (1 - b) * t00 + a * (1 - b) * t10 + (1 - a) * b * t01 + a * b * t11;
  }
}

void or_tail_table(double dR, double dz, double h, const double* tab, const or_table_cfg* c, double* SR,
                   double* SZ) {
  double adz = fabs(dz), BR, BZ, ER, EZ, r[2];
  or_table_frame(dR, adz, c->n_cut, c->n0, &BR, &BZ, &ER, &EZ);
  or_tail_table_read(tab, c, dR, adz, r);
  double sr = BR + ER * r[0];
  double sz = BZ + EZ * r[1];
  double sg = dz > 0.0 ? 1.0 : (dz < 0.0 ? -1.0 : 0.0);
  sz *= sg;
  /* tail images inside the support (an infinite window: every k with |o| < h) */
  int kmax = c->n_cut > 0 ? c->n_cut + 1 : (int)ceil(h) + 2;
  for (int k = -kmax; k <= kmax; ++k) {
    if (k >= -c->n0 && k <= c->n0) continue;
    double o = dz + (double)k;
    if (c->n_cut > 0 && !(fabs(o) < (double)c->n_cut)) continue;
    double rr = sqrt(dR * dR + o * o);
    if (rr >= h) continue;
    double d = or_spline_F_over_r(rr, h) - 1.0 / (rr * rr * rr);
    sr += d;
    sz += o * d;
  }
  *SR = sr;
  *SZ = sz;
}

typedef struct {
  const double* tab;
  const or_table_cfg* c;
} or_table_ctx;

static void or_tail_table_cb(double dR, double dz, double h, const void* ctx, double* SR, double* SZ) {
  const or_table_ctx* t = (const or_table_ctx*)ctx;
  or_tail_table(dR, dz, h, t->tab, t->c, SR, SZ);
}

void or_pair_field_table(int64_t n, const double* x, const double* y, const double* z, const double* m,
                         const double* h, double G, double L, const double* tab, const or_table_cfg* c,
                         int64_t ni, const int64_t* idx, double* gx, double* gy, double* gz) {
  or_table_ctx t = {tab, c};
  or_pair_field_with_tail(n, x, y, z, m, h, G, L, c->n0, or_tail_table_cb, &t, ni, idx, gx, gy, gz);
}

/* ---------------------------------------------------------------------------
 * Octree (Sect. 2.4, "Octree": a Barnes-Hut tree whose root is a cube twice the
 * largest dimension of the volume, re-drawn with a random shift along the axis
 * and a random rotation about it at every force evaluation).
 *
 * Tree frame: x' = c x - s y, y' = s x + c y (c, s = cos, sin phi),
 * z' = z + zeta, minus L when >= L. Root: side S = 2 max(L, 2 R_sim), centre
 * (0, 0, L/2). Normalised coordinates u = (x'/S + 1/2, y'/S + 1/2,
 * (z' - L/2)/S + 1/2) in [0, 1), rounded to FP32, and 21 bits of each give a
 * 63-bit Morton key (x bit b at key bit 3b + 2, y at 3b + 1, z at 3b). The
 * particles are sorted by (key, index). A node is a key prefix; it is a leaf
 * when it holds <= leaf particles or sits at depth 21. Its moments: mass M,
 * centre of mass (x, y in the frame of the particles; z from the tree frame,
 * shifted back by zeta), and the largest softening.
 *
 * Walk. Groups of 32 consecutive particles in key order share one walk: a
 * node is opened for the whole group when any member opens it (a group walk,
 * the form the GPU's warps take). A member opens node n (side s, centre C,
 * normalised coordinates) when s^2 >= theta^2 d^2 or
 * |d| - (sqrt(3)/2) s <= hu_i + hu_max(n), with d the offset of u_i from C,
 * z wrapped to the nearest image, and hu = h / S: accepted nodes are far and
 * beyond every member's softening. (With d taken to the nearest image, a node
 * accepted at small cylindrical distance has s <= theta L / 2, and one at
 * large cylindrical distance is far from all of its images.)
 * This decision is taken in FP32, operation by operation as written, on FP32
 * inputs, so that the GPU takes it identically. An accepted node acts as a
 * point mass M at its centre of mass with softening h_max; an opened leaf
 * gives its particles one by one. Each interaction is the pair term of the
 * direct form (the plain window, or near images plus the correction table).
 * ------------------------------------------------------------------------- */
typedef struct {
  int32_t level, nchild;
  int64_t begin, end, child0;
  float c[3], s, hm;        /* normalised centre, side, largest hu */
  double M, com[3], hmax;   /* mass, centre of mass, largest softening */
} or_tnode;

typedef struct {
  or_tnode* v;
  int64_t n, cap;
} or_tnodes;

static int64_t or_tnode_new(or_tnodes* t) {
  if (t->n == t->cap) {
    int64_t cap = t->cap ? 2 * t->cap : 1024;
    or_tnode* v = (or_tnode*)realloc(t->v, sizeof(or_tnode) * (size_t)cap);
    if (!v) return -1;
    t->v = v;
    t->cap = cap;
  }
  return t->n++;
}

typedef struct {
  uint64_t key;
  int64_t idx;
} or_keyidx;

static int or_keyidx_cmp(const void* a, const void* b) {
  const or_keyidx *p = (const or_keyidx*)a, *q = (const or_keyidx*)b;
  if (p->key != q->key) return p->key < q->key ? -1 : 1;
  return p->idx < q->idx ? -1 : (p->idx > q->idx ? 1 : 0);
}

static uint64_t or_spread3(uint32_t v) { /* bit b of v to bit 3b */
  uint64_t r = 0;
  for (int b = 0; b < 21; ++b) r |= (uint64_t)((v >> b) & 1u) << (3 * b);
  return r;
}

typedef struct {
  const uint64_t* key;   /* sorted keys */
  const int64_t* ord;    /* sorted position -> particle */
  const double *x, *y, *zt, *m, *h;
  const float* hu;
  int32_t leaf;
  double zeta, L;
} or_tbuild;

/* Node of level `level` over sorted positions [begin, end) with integer
 * coordinates (ix, iy, iz) at that level; children are built recursively. */
static int or_tree_build(or_tnodes* t, const or_tbuild* B, int64_t id, int32_t level, int64_t begin,
                         int64_t end, uint32_t ix, uint32_t iy, uint32_t iz) {
  or_tnode* nd = &t->v[id];
  float s = ldexpf(1.0f, -level);
  nd->level = level;
  nd->begin = begin;
  nd->end = end;
  nd->s = s;
  nd->c[0] = ((float)ix + 0.5f) * s;
  nd->c[1] = ((float)iy + 0.5f) * s;
  nd->c[2] = ((float)iz + 0.5f) * s;
  double M = 0, mx = 0, my = 0, mz = 0, hmax = 0;
  float hm = 0.0f;
  for (int64_t q = begin; q < end; ++q) {
    int64_t i = B->ord[q];
    M += B->m[i];
    mx += B->m[i] * B->x[i];
    my += B->m[i] * B->y[i];
    mz += B->m[i] * B->zt[i];
    if (B->h[i] > hmax) hmax = B->h[i];
    if (B->hu[i] > hm) hm = B->hu[i];
  }
  nd->M = M;
  nd->com[0] = mx / M;
  nd->com[1] = my / M;
  nd->com[2] = mz / M - B->zeta; /* back to the frame of the particles (any period) */
  nd->hmax = hmax;
  nd->hm = hm;
  nd->nchild = 0;
  nd->child0 = -1;
  if (end - begin <= B->leaf || level == 21) return 0;
  int sh = 3 * (21 - level - 1);
  int64_t lo[8], hi[8];
  int32_t dig[8], nc = 0;
  for (int64_t q = begin; q < end;) {
    int32_t d = (int32_t)((B->key[q] >> sh) & 7u);
    int64_t e = q;
    while (e < end && (int32_t)((B->key[e] >> sh) & 7u) == d) ++e;
    lo[nc] = q;
    hi[nc] = e;
    dig[nc] = d;
    ++nc;
    q = e;
  }
  int64_t c0 = t->n;
  for (int k = 0; k < nc; ++k)
    if (or_tnode_new(t) < 0) return -2;
  nd = &t->v[id]; /* the array may have moved */
  nd->child0 = c0;
  nd->nchild = nc;
  for (int k = 0; k < nc; ++k) {
    int rc = or_tree_build(t, B, c0 + k, level + 1, lo[k], hi[k], 2 * ix + ((dig[k] >> 2) & 1),
                           2 * iy + ((dig[k] >> 1) & 1), 2 * iz + (dig[k] & 1));
    if (rc) return rc;
  }
  return 0;
}

/* The opening rule of one member (FP32, as written). */
static int or_tree_opens(const float u[3], float hu, const or_tnode* nd, float Lu, float th2) {
  float dx = u[0] - nd->c[0];
  float dy = u[1] - nd->c[1];
  float dz = u[2] - nd->c[2];
  float hLu = 0.5f * Lu;
  if (dz > hLu) dz = dz - Lu;
  else if (dz < -hLu) dz = dz + Lu;
  float d2 = dx * dx + dy * dy;
  d2 = d2 + dz * dz;
  if (nd->s * nd->s >= th2 * d2) return 1;
  float clear = sqrtf(d2) - 0.8660254f * nd->s;
  return clear <= hu + nd->hm;
}

/* Pair term per unit G m_j of one interaction (separation r, softening hh):
 * the plain window (tab == NULL), or the near images |k| <= n0 plus the
 * correction-table tail. */
static void or_tree_pair(double rx, double ry, double rz, double hh, double L, int32_t n_cut, const double* tab,
                         const or_table_cfg* tc, double out[3]) {
  if (!tab) {
    or_image_force(rx, ry, rz, hh, L, n_cut, out);
    return;
  }
  double dx = rx / L, dy = ry / L, r = rz / L, h = hh / L;
  double dzw = r - floor(r + 0.5), dR = sqrt(dx * dx + dy * dy), sr = 0.0, sz = 0.0;
  for (int k = -tc->n0; k <= tc->n0; ++k) {
    double o = dzw + (double)k;
    double f = or_spline_F_over_r(sqrt(dR * dR + o * o), h);
    sr += f;
    sz += o * f;
  }
  double tr, tz;
  or_tail_table(dR, dzw, h, tab, tc, &tr, &tz);
  sr += tr;
  sz += tz;
  out[0] = -dx * sr / (L * L);
  out[1] = -dy * sr / (L * L);
  out[2] = -sz / (L * L);
}

/* The tree's frame: S1xR2 (shift zeta along the axis, rotation phi about it, root
 * side S = 2 max(L, 2 R_sim) centred at (0, 0, L/2)), or R^3 (the domain centre
 * moved to cen, a rotation R about a random axis, root side S = 4 R_sim centred
 * at cen; no period). */
typedef struct {
  int32_t r3;
  double S, zeta, c, s;   /* S1xR2 */
  double cen[3], R[9];    /* R^3 */
} or_tframe;

/* Rotation by angle about the unit axis (Rodrigues' formula), each entry with
 * the explicit fma/mul sequence written here. */
static void or_rotation(const double ax[3], double angle, double R[9]) {
  double cs = cos(angle), sn = sin(angle), t = 1.0 - cs;
  double tx = t * ax[0], ty = t * ax[1], tz = t * ax[2];
  double sx = sn * ax[0], sy = sn * ax[1], sz = sn * ax[2];
  R[0] = fma(tx, ax[0], cs);  R[1] = fma(tx, ax[1], -sz); R[2] = fma(tx, ax[2], sy);
  R[3] = fma(ty, ax[0], sz);  R[4] = fma(ty, ax[1], cs);  R[5] = fma(ty, ax[2], -sx);
  R[6] = fma(tz, ax[0], -sy); R[7] = fma(tz, ax[1], sx);  R[8] = fma(tz, ax[2], cs);
}

/* R^3 pair term per unit G m_j (eq. NewtonianForce): -F(r, hh)/r r. */
static void or_r3_pair(double rx, double ry, double rz, double hh, double out[3]) {
  double f = or_spline_F_over_r(sqrt(rx * rx + ry * ry + rz * rz), hh);
  out[0] = -f * rx;
  out[1] = -f * ry;
  out[2] = -f * rz;
}

static int or_tree_core(int64_t n, const double* x, const double* y, const double* z, const double* m,
                        const double* h, double G, double L, int32_t n_cut, const double* tab, const or_table_cfg* tc,
                        double theta, int32_t leaf, const or_tframe* F, int64_t ni, const int64_t* idx, double* gx,
                        double* gy, double* gz, int64_t* stats) {
  double S = F->S, invS = 1.0 / S, c = F->c, s = F->s, halfL = 0.5 * L, zeta = F->r3 ? 0.0 : F->zeta;
  /* R^3 has no period: an infinite period never wraps */
  float Lu = F->r3 ? (float)INFINITY : (float)(L * invS), th2 = (float)(theta * theta);
  float* u = (float*)malloc(sizeof(float) * 3 * (size_t)n);
  float* hu = (float*)malloc(sizeof(float) * (size_t)n);
  double* zt = (double*)malloc(sizeof(double) * (size_t)n);
  or_keyidx* ki = (or_keyidx*)malloc(sizeof(or_keyidx) * (size_t)n);
  uint64_t* key = (uint64_t*)malloc(sizeof(uint64_t) * (size_t)n);
  int64_t* ord = (int64_t*)malloc(sizeof(int64_t) * (size_t)n);
  int64_t* slot = (int64_t*)malloc(sizeof(int64_t) * (size_t)n); /* particle -> output slot, -1: none */
  unsigned char* want = (unsigned char*)calloc((size_t)(n + 31) / 32 + 1, 1);
  or_tnodes t = {NULL, 0, 0};
  int rc = 0;
  if (!u || !hu || !zt || !ki || !key || !ord || !slot || !want) { rc = -2; goto done; }
  for (int64_t i = 0; i < n; ++i) {
    if (F->r3) {
      const double* R = F->R;
      double dx = x[i] - F->cen[0], dy = y[i] - F->cen[1], dz = z[i] - F->cen[2];
      double xr = fma(R[0], dx, fma(R[1], dy, R[2] * dz));
      double yr = fma(R[3], dx, fma(R[4], dy, R[5] * dz));
      double zr = fma(R[6], dx, fma(R[7], dy, R[8] * dz));
      zt[i] = z[i]; /* centres of mass in the particles' own frame */
      u[3 * i] = (float)fma(xr, invS, 0.5);
      u[3 * i + 1] = (float)fma(yr, invS, 0.5);
      u[3 * i + 2] = (float)fma(zr, invS, 0.5);
    } else {
      double xr = fma(c, x[i], -(s * y[i]));
      double yr = fma(s, x[i], c * y[i]);
      double zr = z[i] + zeta;
      if (zr >= L) zr = zr - L;
      zt[i] = zr;
      u[3 * i] = (float)fma(xr, invS, 0.5);
      u[3 * i + 1] = (float)fma(yr, invS, 0.5);
      u[3 * i + 2] = (float)fma(zr - halfL, invS, 0.5);
    }
    hu[i] = (float)(h[i] * invS);
    uint32_t q[3];
    for (int a = 0; a < 3; ++a) {
      float v = u[3 * i + a];
      if (!(v >= 0.0f && v < 1.0f)) { rc = -1; goto done; } /* outside the root cube */
      q[a] = (uint32_t)(v * 2097152.0f);
    }
    ki[i].key = (or_spread3(q[0]) << 2) | (or_spread3(q[1]) << 1) | or_spread3(q[2]);
    ki[i].idx = i;
  }
  qsort(ki, (size_t)n, sizeof(or_keyidx), or_keyidx_cmp);
  for (int64_t q = 0; q < n; ++q) {
    key[q] = ki[q].key;
    ord[q] = ki[q].idx;
  }
  for (int64_t i = 0; i < n; ++i) slot[i] = idx ? -1 : i;
  if (idx) {
    for (int64_t k = 0; k < ni; ++k) {
      if (idx[k] < 0 || idx[k] >= n) { rc = -3; goto done; }
      slot[idx[k]] = k;
    }
  }
  for (int64_t q = 0; q < n; ++q)
    if (slot[ord[q]] >= 0) want[q / 32] = 1;
  {
    or_tbuild B = {key, ord, x, y, zt, m, h, hu, leaf, zeta, L};
    if (or_tnode_new(&t) < 0) { rc = -2; goto done; }
    rc = or_tree_build(&t, &B, 0, 0, 0, n, 0, 0, 0);
    if (rc) goto done;
  }
  int64_t ngroups = (n + 31) / 32, inter = 0;
#pragma omp parallel for schedule(dynamic, 1) reduction(+ : inter)
  for (int64_t g = 0; g < ngroups; ++g) {
    if (!want[g]) continue; /* no requested member: the group's walk is not needed */
    int64_t q0 = 32 * g, q1 = q0 + 32 < n ? q0 + 32 : n;
    int nm = (int)(q1 - q0);
    or_sum acc[32][3];
    memset(acc, 0, sizeof acc);
    int64_t stack[256];
    int top = 0;
    stack[top++] = 0;
    while (top > 0) {
      const or_tnode* nd = &t.v[stack[--top]];
      int open = 0;
      for (int k = 0; k < nm && !open; ++k) {
        int64_t i = ord[q0 + k];
        open = or_tree_opens(&u[3 * i], hu[i], nd, Lu, th2);
      }
      if (open && nd->nchild > 0) {
        for (int k = 0; k < nd->nchild; ++k) stack[top++] = nd->child0 + k;
        continue;
      }
      for (int k = 0; k < nm; ++k) {
        int64_t i = ord[q0 + k];
        double f[3];
        if (!open) {
          if (F->r3)
            or_r3_pair(x[i] - nd->com[0], y[i] - nd->com[1], z[i] - nd->com[2], h[i] + nd->hmax, f);
          else
            or_tree_pair(x[i] - nd->com[0], y[i] - nd->com[1], z[i] - nd->com[2], h[i] + nd->hmax, L, n_cut, tab,
                         tc, f);
          for (int a = 0; a < 3; ++a) or_add(&acc[k][a], G * nd->M * f[a]);
          ++inter;
        } else {
          for (int64_t p = nd->begin; p < nd->end; ++p) {
            int64_t j = ord[p];
            ++inter; /* member x entry, the member's own entry included */
            if (j == i) continue;
            if (F->r3)
              or_r3_pair(x[i] - x[j], y[i] - y[j], z[i] - z[j], h[i] + h[j], f);
            else
              or_tree_pair(x[i] - x[j], y[i] - y[j], z[i] - z[j], h[i] + h[j], L, n_cut, tab, tc, f);
            for (int a = 0; a < 3; ++a) or_add(&acc[k][a], G * m[j] * f[a]);
          }
        }
      }
    }
    for (int k = 0; k < nm; ++k) {
      int64_t o = slot[ord[q0 + k]];
      if (o < 0) continue;
      gx[o] = acc[k][0].s + acc[k][0].c;
      gy[o] = acc[k][1].s + acc[k][1].c;
      gz[o] = acc[k][2].s + acc[k][2].c;
    }
  }
  if (stats) {
    int64_t leaves = 0, depth = 0;
    for (int64_t k = 0; k < t.n; ++k) {
      if (t.v[k].nchild == 0) ++leaves;
      if (t.v[k].level > depth) depth = t.v[k].level;
    }
    stats[0] = t.n;
    stats[1] = leaves;
    stats[2] = depth;
    stats[3] = inter;
  }
done:
  free(u); free(hu); free(zt); free(ki); free(key); free(ord); free(slot); free(want); free(t.v);
  return rc;
}

int or_tree_field(int64_t n, const double* x, const double* y, const double* z, const double* m, const double* h,
                  double G, double L, double R_sim, int32_t n_cut, const double* tab, const or_table_cfg* tc,
                  double theta, int32_t leaf, double zeta, double phi, int64_t ni, const int64_t* idx, double* gx,
                  double* gy, double* gz, int64_t* stats) {
  or_tframe F;
  memset(&F, 0, sizeof F);
  F.S = 2.0 * fmax(L, 2.0 * R_sim);
  F.zeta = zeta;
  F.c = cos(phi);
  F.s = sin(phi);
  return or_tree_core(n, x, y, z, m, h, G, L, n_cut, tab, tc, theta, leaf, &F, ni, idx, gx, gy, gz, stats);
}

int or_tree_field_r3(int64_t n, const double* x, const double* y, const double* z, const double* m, const double* h,
                     double G, double R_sim, double theta, int32_t leaf, const double cen[3], const double axis[3],
                     double angle, int64_t ni, const int64_t* idx, double* gx, double* gy, double* gz,
                     int64_t* stats) {
  or_tframe F;
  memset(&F, 0, sizeof F);
  F.r3 = 1;
  F.S = 4.0 * R_sim;
  for (int a = 0; a < 3; ++a) F.cen[a] = cen[a];
  or_rotation(axis, angle, F.R);
  return or_tree_core(n, x, y, z, m, h, G, 1.0, 0, NULL, NULL, theta, leaf, &F, ni, idx, gx, gy, gz, stats);
}

/* Sorted order of the tree frame (for checks of the sort): ord[q] = particle at
 * key position q, key[q] its key. */
int or_tree_order(int64_t n, const double* x, const double* y, const double* z, double L, double R_sim,
                  double zeta, double phi, uint64_t* key, int64_t* ord) {
  double S = 2.0 * fmax(L, 2.0 * R_sim), invS = 1.0 / S, c = cos(phi), s = sin(phi), halfL = 0.5 * L;
  or_keyidx* ki = (or_keyidx*)malloc(sizeof(or_keyidx) * (size_t)n);
  if (!ki) return -2;
  for (int64_t i = 0; i < n; ++i) {
    double xr = fma(c, x[i], -(s * y[i])), yr = fma(s, x[i], c * y[i]), zr = z[i] + zeta;
    if (zr >= L) zr = zr - L;
    float v[3] = {(float)fma(xr, invS, 0.5), (float)fma(yr, invS, 0.5), (float)fma(zr - halfL, invS, 0.5)};
    uint32_t q[3];
    for (int a = 0; a < 3; ++a) {
      if (!(v[a] >= 0.0f && v[a] < 1.0f)) { free(ki); return -1; }
      q[a] = (uint32_t)(v[a] * 2097152.0f);
    }
    ki[i].key = (or_spread3(q[0]) << 2) | (or_spread3(q[1]) << 1) | or_spread3(q[2]);
    ki[i].idx = i;
  }
  qsort(ki, (size_t)n, sizeof(or_keyidx), or_keyidx_cmp);
  for (int64_t q = 0; q < n; ++q) {
    key[q] = ki[q].key;
    ord[q] = ki[q].idx;
  }
  free(ki);
  return 0;
}
