/*
 * FP64 CPU oracle for the S1xR2 (periodic-cylinder) StePS force and integrator.
 *
 * TEST INFRASTRUCTURE ONLY. This library exists to check the CUDA path. Only the
 * test-suite, the smoke check and the benchmark's CPU-baseline leg may load it.
 * It shares no code, header, table or constant with the CUDA library.
 *
 * Every routine is the plain definition from the paper (arXiv 2602.20787):
 *   - Eq. Force_spline_kernel (Sect. 2.1): cubic-spline softened force F(r,h).
 *   - Eq. ForceCylindrical (Sect. 2.1): windowed image sum along z.
 *   - Eq. ComovingEquationsOfMotionCylindrical (Sect. 2.1): pair term, 1/a^3,
 *     background term of eq. F_horiz, Hubble drag.
 *   - Eq. F_horiz (Sect. 2.1), re-derived (the printed form is garbled), with the
 *     limit eq. F_horiz_infty.
 *   - Eqs. Friedmann, DEdensity, CPLw0wa (Sect. 2.3) with RK4 (Sect. 2.3).
 *   - KDK leapfrog in cosmic time (end of Sect. 2.1).
 * The far-image surrogate (a 3->32->32->2 ReLU MLP) has its FP64 forward and
 * backward pass here too, for gradient checks.
 */
#ifndef STEPS_ORACLE_H
#define STEPS_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Cosmology of eqs. Friedmann / DEdensity / CPLw0wa. comoving == 0 means
 * static space: a = 1, H = 0 at all times. */
typedef struct {
  double H0, Omega_m, Omega_r, Omega_L, w0, wa;
  int32_t comoving;
} or_cosmo;

double or_spline_F(double r, double h);
double or_spline_F_over_r(double r, double h);
int or_image_force(double rx, double ry, double rz, double h, double L, int32_t n_cut, double out[3]);
void or_pair_field(int64_t n, const double* x, const double* y, const double* z, const double* m,
                   const double* h, double G, double L, int32_t n_cut, int64_t ni, const int64_t* idx,
                   double* gx, double* gy, double* gz);
double or_cylinder_field(double varrho, double R, double Lw, double G, double rho0);
void or_background_field(int64_t ni, const double* x, const double* y, double R, double Lw, double G,
                         double rho0, double* gx, double* gy);
double or_hubble(const or_cosmo* c, double a);
double or_a_of_t_step(const or_cosmo* c, double a, double dt);
void or_kdk_factors(const or_cosmo* c, double a, double dt, double* K1, double* D, double* K2,
                    double* a_next);
int or_kdk(int64_t n, double* x, double* y, double* z, double* px, double* py, double* pz,
           const double* m, const double* h, double G, double L, int32_t n_cut, double R_bg,
           double rho0, int32_t background, const or_cosmo* c, double* a, double* t, double dt,
           int32_t nsteps);
/* R^3 topology (eq. NewtonianForce, no images) and its radial background term. */
void or_pair_field_r3(int64_t n, const double* x, const double* y, const double* z, const double* m,
                      const double* h, double G, int64_t ni, const int64_t* idx, double* gx, double* gy,
                      double* gz);
void or_background_sphere(int64_t ni, const double* x, const double* y, const double* z, double G, double rho0,
                          double* gx, double* gy, double* gz);
/* or_kdk with a topology: 0 = S1xR2 (z wrapped into [0, L)), 1 = R^3 (background 0 or 3 = sphere). */
int or_kdk_topo(int64_t n, double* x, double* y, double* z, double* px, double* py, double* pz,
                const double* m, const double* h, double G, double L, int32_t n_cut, double R_bg,
                double rho0, int32_t background, int32_t topology, const or_cosmo* c, double* a, double* t,
                double dt, int32_t nsteps);
/* Sect. 1 diagnostics of a state at expansion factor a (p canonical, a^2 dx/dt):
 * out = (sum m p [3], L_z = sum m (x p_y - y p_x), sum m |dx/dt|^2 / 2, sum m). */
void or_diagnostics(int64_t n, const double* x, const double* y, const double* px, const double* py,
                    const double* pz, const double* m, double a, double out[6]);
void or_tail_sums(double dR, double dzw, double h, double L, int32_t n_cut, int32_t n0, double* SR,
                  double* Sz);
void or_mlp_forward(const double* w, const double* u, double* y);
/* Learned far-image surrogate (this project's definition; the paper has none):
 * tail = order-1 Euler-Maclaurin continuum base + envelope * (MLP(u) * sc + mu),
 * plus the exact spline correction of tail images inside the softening support. */
typedef struct {
  int32_t n_cut, n0;
  double dR_max;        /* input scaling of dR (units of L) */
  double out_mu[2], out_sc[2];
} or_surr_cfg;
void or_tail_base(double dR, double adz, int32_t n_cut, int32_t n0, double* BR, double* BZ);
void or_tail_envelope(double dR, double adz, int32_t n0, double* ER, double* EZ);
void or_surrogate_inputs(double dR, double adz, double h, int32_t n0, double dR_max, double u[3]);
void or_tail_surrogate(double dR, double dz, double h, const double* w, const or_surr_cfg* c, double* SR,
                       double* SZ);
void or_pair_field_surrogate(int64_t n, const double* x, const double* y, const double* z, const double* m,
                             const double* h, double G, double L, const double* w, const or_surr_cfg* c,
                             int64_t ni, const int64_t* idx, double* gx, double* gy, double* gz);
/* Ncut -> infinity: every periodic image (exact to |k| <= 512, continuum cells
 * beyond), the pair field with that window, and the tail base beyond |k| <= n0. */
void or_image_sums_inf(double dR, double dzw, double h, int32_t n0, double* SR, double* SZ);
void or_pair_field_inf(int64_t n, const double* x, const double* y, const double* z, const double* m,
                       const double* h, double G, double L, int64_t ni, const int64_t* idx, double* gx,
                       double* gy, double* gz);
void or_tail_base_inf(double dR, double adz, int32_t n0, double* BR, double* BZ);
/* Ewald summation of the infinite line (Sect. 2.3) with the re-derived Fourier
 * kernel: the sums of the images |k| > n0 (units of L, point masses), split
 * parameter alpha (1/L), real-space images |n| <= nmax, Fourier modes m <= mmax. */
void or_ewald_tail(double dR, double dzw, int32_t n0, double alpha, int32_t nmax, int32_t mmax, double* SR,
                   double* SZ);
/* Correction-table tail (the paper's Sect. 2.3 table restated for the windowed
 * sum beyond |k| <= n0): residual of the point-mass tail over the continuum base
 * in envelope units on a uniform (dR, |dz|) grid, read with cloud-in-cell
 * (bilinear) or triangular-shaped-cloud weights, the two reads Sect. 2.3 names.
 * n0 = 0 is the paper's table over the nearest image alone: it holds the tail
 * sums themselves (no base, unit envelope). */
#define OR_TABLE_CIC 0
#define OR_TABLE_TSC 1
typedef struct {
  int32_t n_cut, n0, nx, ny;   /* n_cut = 0: the infinite window */
  double dR_max;        /* last column; dR beyond it reads the last column */
  int32_t read, pad;    /* OR_TABLE_CIC or OR_TABLE_TSC */
} or_table_cfg;
void or_tail_residual(double dR, double adz, int32_t n_cut, int32_t n0, double r[2]);
void or_tail_table_build(const or_table_cfg* c, double* tab); /* tab[ny][nx][2] */
void or_tail_table_read(const double* tab, const or_table_cfg* c, double dR, double adz, double r[2]);
void or_tail_table(double dR, double dz, double h, const double* tab, const or_table_cfg* c, double* SR,
                   double* SZ);
void or_pair_field_table(int64_t n, const double* x, const double* y, const double* z, const double* m,
                         const double* h, double G, double L, const double* tab, const or_table_cfg* c,
                         int64_t ni, const int64_t* idx, double* gx, double* gy, double* gz);
/* Octree (Sect. 2.4): Barnes-Hut group walk in a shifted and rotated frame
 * (zeta, phi), opening angle theta, leaves of <= leaf particles; each
 * interaction is the pair term of the direct form (tab == NULL: the plain
 * window of n_cut; else near images plus the correction table tc). idx ==
 * NULL gives every particle (ni = n); else the ni listed ones, walking only
 * their groups. Returns 0, -1 when a particle lies outside the root cube, -2 on
 * allocation failure, -3 for a bad index. stats (may be NULL): nodes, leaves,
 * depth, interactions (member x list entry over the groups walked, a member's
 * own entry in its leaf included). */
int or_tree_field(int64_t n, const double* x, const double* y, const double* z, const double* m, const double* h,
                  double G, double L, double R_sim, int32_t n_cut, const double* tab, const or_table_cfg* tc,
                  double theta, int32_t leaf, double zeta, double phi, int64_t ni, const int64_t* idx, double* gx,
                  double* gy, double* gz, int64_t* stats);
/* The R^3 octree (Sect. 2.4): the domain centre moved to cen, the frame rotated
 * by angle about the unit axis, root side 4 R_sim centred there, no period; the
 * interactions are the pair force of eq. NewtonianForce. Otherwise as
 * or_tree_field. */
int or_tree_field_r3(int64_t n, const double* x, const double* y, const double* z, const double* m, const double* h,
                     double G, double R_sim, double theta, int32_t leaf, const double cen[3], const double axis[3],
                     double angle, int64_t ni, const int64_t* idx, double* gx, double* gy, double* gz,
                     int64_t* stats);
int or_tree_order(int64_t n, const double* x, const double* y, const double* z, double L, double R_sim,
                  double zeta, double phi, uint64_t* key, int64_t* ord);
double or_mlp_loss_grad(const double* w, int64_t ns, const double* u, const double* t, double* grad);
void or_adam_step(int64_t nw, double* w, const double* g, double* m1, double* m2, double lr,
                  double beta1, double beta2, double eps, int64_t step);
int32_t or_num_threads(void);

#ifdef __cplusplus
}
#endif
#endif
