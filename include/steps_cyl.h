/*
 * steps_cyl.h - C ABI of the GB300 (sm_103a) S1xR2 StePS hot path.
 *
 * What it computes (arXiv 2602.20787, Sect. 2.1 and 2.3):
 *   - the softened pair force of eq. Force_spline_kernel summed over the periodic
 *     images of eq. ForceCylindrical (window |r_z - n L| < Ncut L, n in [-Ncut, Ncut]),
 *     with pair softening h_i + h_j (eq. ComovingEquationsOfMotion);
 *   - the finite-cylinder background of eq. F_horiz (re-derived: the printed formula
 *     is garbled) or its infinite limit eq. F_horiz_infty;
 *   - the comoving equations of motion eq. ComovingEquationsOfMotionCylindrical,
 *     integrated with a kick-drift-kick leapfrog in cosmic time with a(t) from the
 *     Friedmann equation (eqs. Friedmann, DEdensity, CPLw0wa) by RK4.
 *
 * Conventions shared by every entry point
 *   - Units are the caller's; positions x, y are free, z must lie in [0, L).
 *   - Arrays are structure-of-arrays, one double per particle, contiguous.
 *   - A pointer argument may be host memory or device memory of the context's
 *     device; the library finds out with cudaPointerGetAttributes. The library
 *     copies what it needs and never keeps a caller pointer past the call.
 *   - Work is ordered on the context's stream (steps_cyl_params.stream, or the
 *     legacy default stream when NULL). A call that writes host memory returns
 *     after the data is there; a call that writes device memory returns once the
 *     work is enqueued, except steps_cyl_kdk_step which always synchronises to
 *     read the device error word.
 *   - Every call returns STEPS_OK (0) or a negative STEPS_E* code. The message of
 *     the last failure on the calling thread is steps_cyl_last_error().
 *   - A context is not thread-safe; distinct contexts are independent.
 */
#ifndef STEPS_CYL_H
#define STEPS_CYL_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------ */
#define STEPS_OK 0
#define STEPS_EINVAL (-1)               /* bad argument (N < 2, h <= 0, L <= 0, z outside [0,L), non-finite input) */
#define STEPS_ECUDA (-2)                /* a CUDA runtime call failed */
#define STEPS_ENOMEM (-3)               /* device allocation failed */
#define STEPS_EDEVICE (-4)              /* the device error word was set (non-finite force, particle beyond the background
                                         * table, particle outside the octree's root cube, octree walk stack overflow,
                                         * a pair sum beyond the range of the symmetric kernels' fixed-point sums) */
#define STEPS_ESURROGATE_REJECTED (-5)  /* surrogate error above its bound: the plain image sum was used instead */
#define STEPS_ENOSURROGATE (-6)         /* modelled tail requested but no accepted network / correction table is loaded */

/* ---- enumerations ------------------------------------------------------ */
#define STEPS_FP64 0        /* pair geometry and sums in FP64 */
#define STEPS_FP32_KAHAN 1  /* FP32 pair math on hi/lo split positions, Kahan-compensated j sum */
#define STEPS_FP32_PLAIN 2  /* FP32 pair math on hi/lo split positions, plain j sum */

#define STEPS_TAIL_FULL 0       /* every image of the window summed directly */
#define STEPS_TAIL_SURROGATE 1  /* images |k| <= n0 direct, far tail from the learned surrogate */
#define STEPS_TAIL_TABLE 2      /* images |k| <= n0 direct, far tail from the correction table */

#define STEPS_TABLE_READ_CIC 0  /* correction table read with cloud-in-cell (bilinear) weights */
#define STEPS_TABLE_READ_TSC 1  /* correction table read with triangular-shaped-cloud weights */

#define STEPS_BG_OFF 0       /* no background term */
#define STEPS_BG_FINITE 1    /* eq. F_horiz: cylinder of radius R_sim and height 2 Ncut L */
#define STEPS_BG_INFINITE 2  /* eq. F_horiz_infty inside R_sim, line-mass field outside */
#define STEPS_BG_SPHERE 3    /* R^3 topology: the radial term +(4 pi G / 3) rho_bar x of Sect. 2.1 */

#define STEPS_FORCE_DIRECT 0  /* the O(N^2) direct pair sum */
#define STEPS_FORCE_OCTREE 1  /* the octree of Sect. 2.4 (O(N log N)) */

#define STEPS_TOPO_S1R2 0  /* compact z axis of period L: eq. ForceCylindrical (the default) */
#define STEPS_TOPO_R3 1    /* no compact axis: the softened Newtonian pair force of eq. NewtonianForce,
                            * no images, z unbounded; background STEPS_BG_OFF or STEPS_BG_SPHERE */

typedef struct steps_cyl_ctx steps_cyl_ctx; /* opaque; owned by the library until steps_cyl_free */

typedef struct {
  double G;         /* gravitational constant (!= 0; G < 0 is the repulsive gravity of glass making, Sect. 3.1) */
  double L;         /* period L_z of the compact axis (> 0) */
  double R_sim;     /* radius of the simulated cylinder used by the background term (> 0) */
  double rho_bar;   /* comoving mean density of the background term; 0 means sum(m) / (pi R_sim^2 L), or
                     * sum(m) / (4 pi R_sim^3 / 3) in the R^3 topology */
  int32_t n_cut;    /* image cut-off Ncut of eq. ForceCylindrical, 1 <= n_cut <= 4096; 0 is the
                     * infinite window (Ncut -> infinity, Sect. 2.2): it has no plain image sum,
                     * needs STEPS_TAIL_TABLE at init (its correction table is built there; a
                     * surrogate trained to infinity may be selected later), an FP32 precision
                     * and STEPS_BG_INFINITE or STEPS_BG_OFF */
  int32_t n0;       /* near range of a modelled tail: images |k| <= n0 summed directly,
                     * 1 <= n0 < n_cut (1 <= n0 < 512 for the infinite window); the
                     * table tail also takes n0 = 0, the paper's table over the
                     * nearest image alone (steps_cyl_build_tail_table) */
  int32_t precision;  /* STEPS_FP64 | STEPS_FP32_KAHAN | STEPS_FP32_PLAIN */
  int32_t tail;       /* STEPS_TAIL_FULL | STEPS_TAIL_SURROGATE | STEPS_TAIL_TABLE */
  int32_t background; /* STEPS_BG_OFF | STEPS_BG_FINITE | STEPS_BG_INFINITE */
  int32_t comoving;   /* 0: static space (a = 1, H = 0); 1: expanding background */
  double H0, Omega_m, Omega_r, Omega_L, w0, wa; /* eqs. Friedmann, DEdensity, CPLw0wa; Omega_k = 1 - sum */
  double a_start;   /* scale factor at t_start (1 in static space) */
  double t_start;   /* cosmic time at the start */
  int32_t device;   /* CUDA device ordinal */
  int32_t reorder_every; /* particles are kept in a Morton order of (x, y) inside the library (results are
                          * returned in the caller's order); it is rebuilt at init, by set_state, and every
                          * reorder_every KDK steps (0: never during stepping; -1: keep the caller's order) */
  int32_t check_every;   /* with a modelled tail (surrogate or table): every check_every KDK steps its forces
                          * on a particle sample are compared with the plain image sum; above the bounds
                          * the context falls back to the plain sum (0: no periodic check) */
  int32_t check_particles; /* size of that sample (default 1024) */
  int32_t topology; /* STEPS_TOPO_S1R2 | STEPS_TOPO_R3 (R^3: n_cut is not used, tail must be STEPS_TAIL_FULL) */
  int32_t reserved; /* 0 */
  void* stream;     /* cudaStream_t to order work on; NULL = legacy default stream */
  int32_t force;    /* STEPS_FORCE_DIRECT | STEPS_FORCE_OCTREE. The octree (Sect. 2.4) needs an FP32
                     * precision and, in S1xR2, the infinite window (n_cut = 0, STEPS_TAIL_TABLE) */
  int32_t leaf_size;  /* octree: a node of at most this many particles is a leaf (1 .. 64) */
  double theta;       /* octree: opening angle Theta, 0 < theta <= 1 */
  uint64_t tree_seed; /* octree: seed of the random shift and rotation drawn at every force evaluation */
} steps_cyl_params;

/* Fill *p with defaults (direct force; octree leaf_size 16, theta 0.5, tree_seed 1):
 * G = L = 1, R_sim = 0.5 tan(0.45 pi), rho_bar = 0, n_cut = 16,
 * n0 = 4, FP32_KAHAN, TAIL_FULL, BG_FINITE, static space, H0 = 1, Omega_m = 0.3,
 * Omega_L = 0.7, w0 = -1, wa = 0, a_start = 1, t_start = 0, device 0, reorder_every = 32,
 * check_every = 50, check_particles = 1024, default stream. */
int steps_cyl_params_default(steps_cyl_params* p);

/* Create a context holding n particles (eq. ComovingEquationsOfMotionCylindrical state).
 * x, y, z: positions (z in [0, L)); vx, vy, vz: comoving velocities dx/dt; m: masses
 * (> 0); h: softening support radii (> 0; a pair uses h_i + h_j). All length n,
 * host or device. 2 <= n < 2^31. On success *out is a new context and the forces at
 * the initial positions are computed (they feed the first kick). */
int steps_cyl_init(steps_cyl_ctx** out, const steps_cyl_params* p, int64_t n, const double* x,
                   const double* y, const double* z, const double* vx, const double* vy,
                   const double* vz, const double* m, const double* h);

/* Accelerations at the current positions: the pair term of eq.
 * ComovingEquationsOfMotionCylindrical divided by a^3 plus the background term
 * (also divided by a^3), without the Hubble drag. ax, ay, az: length n, host or
 * device, written in full (a sharded context writes zeros outside its rows). */
int steps_cyl_forces(steps_cyl_ctx* ctx, double* ax, double* ay, double* az);

/* Same as steps_cyl_forces for the ni particles listed in idx (host or device
 * int64 array, values in [0, n)), each against all n particles. Output length ni. */
int steps_cyl_forces_subset(steps_cyl_ctx* ctx, int64_t ni, const int64_t* idx, double* ax,
                            double* ay, double* az);

/* Advance nsteps >= 0 KDK steps of constant cosmic-time length dt > 0: kick by
 * Int dt/a over the first half, drift by Int dt/a^2, new forces, kick by Int dt/a
 * over the second half (canonical momentum p = a^2 dx/dt; the Hubble drag is
 * exact in this form). z is wrapped into [0, L) after each drift. */
int steps_cyl_kdk_step(steps_cyl_ctx* ctx, double dt, int32_t nsteps);

/* Copy the state out: positions, comoving velocities dx/dt, and the scale factor
 * and time (any output pointer may be NULL to skip it). */
int steps_cyl_get_state(steps_cyl_ctx* ctx, double* x, double* y, double* z, double* vx,
                        double* vy, double* vz, double* a, double* t);

/* Replace positions and velocities (same n; masses and softenings unchanged).
 * The forces that feed the next kick are recomputed unless the new positions are
 * bitwise equal to the current ones (then the cached forces are still exact).
 * Pointers as in steps_cyl_init. Synchronises the context stream. */
int steps_cyl_set_state(steps_cyl_ctx* ctx, const double* x, const double* y, const double* z,
                        const double* vx, const double* vy, const double* vz);

/* Switch the pair-kernel precision (STEPS_FP64 / FP32_KAHAN / FP32_PLAIN) of an
 * existing context (STEPS_FP64 also selects STEPS_TAIL_FULL). Nothing is
 * computed here: the forces that feed the next kick are recomputed by the next
 * force evaluation or at the start of the next KDK step. */
int steps_cyl_set_precision(steps_cyl_ctx* ctx, int32_t precision);

/* Conserved quantities and energies (Sect. 1: P_z and L_z are conserved in
 * S1xR2). out[0..2] = sum m p (canonical momentum a^2 dx/dt), out[3] = L_z =
 * sum m (x p_y - y p_x), out[4] = sum m |dx/dt|^2 / 2, out[5] = a, out[6] = t,
 * out[7] = total mass. out: 8 doubles of host memory. */
int steps_cyl_diagnostics(steps_cyl_ctx* ctx, double out[8]);

/* Pair-images of the last force evaluation, counted as the paper's window
 * over every ordered pair (2 Ncut per pair, 2 Ncut - 1 when r_z = 0 mod L),
 * and the device time of its pair kernel in milliseconds (CUDA events on the
 * context stream). The symmetric kernels deliver these while evaluating each
 * unordered pair once; steps_cyl_last_eval gives the count they evaluated. */
int steps_cyl_last_timing(steps_cyl_ctx* ctx, double* pair_images, double* pair_ms);

/* The last direct force evaluation in more detail (out: 4 doubles, host):
 * out[0] = pair-images delivered (as steps_cyl_last_timing), out[1] = pairs the
 * pair kernel evaluated, out[2] = its device time in ms, out[3] = 1 when it was
 * a symmetric kernel, 2 when that symmetric kernel was a modelled tail's
 * straight-run form (learned tail or residual table of a finite window with
 * near range n0 = 4 and every h_i + h_j below L / 2; same values as the tiered
 * form). The FP32 direct forms of an S1xR2 context whose rows are
 * not shared with other ranks evaluate each unordered pair of particles once
 * and add it to both (Newton's third law; the window of eq. ForceCylindrical is
 * symmetric in i and j), so out[1] is n (n - 1) / 2 plus the pairs inside each
 * block of 128 rows, which are taken both ways; the row kernels evaluate
 * (rows) x (n - 1) ordered pairs. The octree reports its interactions in
 * steps_cyl_tree_stats instead. */
int steps_cyl_last_eval(steps_cyl_ctx* ctx, double out[4]);

/* ---- row sharding (one rank per GPU) ---------------------------------------
 * Sect. 2.4 runs the direct force on many GPUs with MPI. Here the rows i of the
 * pair sum are split across ranks: each rank's context holds the whole particle
 * set, evaluates the pair force of its own rows against every j, and kicks and
 * drifts only those rows. The one exchange per step is an all-gather of the
 * packed positions of every rank's rows, made by the caller (NCCL, gloo, ...)
 * between steps_cyl_shard_drift and steps_cyl_shard_kick.
 *
 * steps_cyl_shard makes a context (created by steps_cyl_init from the same full
 * state on every rank, with the same parameters) the shard `rank` of `world`.
 * The internal particle order, which every rank computed identically at init,
 * is frozen from then on. The rows are split into world balanced contiguous
 * ranges of 128-row blocks (world <= ceil(n / 128)). rows (3 int64, host)
 * receives the owned internal range [k0, k1) and chunk, the largest share: an
 * exchange buffer holds chunk rows of 8 floats (32 bytes) per rank.
 * Afterwards:
 *   - steps_cyl_forces, steps_cyl_get_state and steps_cyl_diagnostics cover the
 *     owned rows only: outputs in caller order hold zeros for the other rows
 *     (so a sum over ranks assembles the whole), and diagnostics sum the owned
 *     rows (sum them over ranks; out[5], out[6] are a and t);
 *   - steps_cyl_kdk_step, steps_cyl_forces_subset, steps_cyl_set_state,
 *     steps_cyl_checkpoint, steps_cyl_train_surrogate, steps_cyl_set_surrogate
 *     and steps_cyl_build_tail_table give STEPS_EINVAL: train or install a
 *     modelled tail before sharding; steps_cyl_set_tail and
 *     steps_cyl_set_precision still switch forms;
 *   - steps_cyl_check_surrogate checks a sample of the owned rows, and the
 *     periodic checks of steps_cyl_kdk_step do not run: the caller combines
 *     the ranks' checks (e.g. the largest error) and switches every rank alike.
 * STEPS_EINVAL for a context sharded already, an octree context, the FP64
 * precision (its kernel reads the FP64 positions of every j, and only the
 * packed FP32 words are exchanged; steps_cyl_set_precision refuses it later
 * too), or a bad rank/world; STEPS_ENOMEM/ECUDA leave the context whole and
 * unsharded. */
int steps_cyl_shard(steps_cyl_ctx* ctx, int32_t rank, int32_t world, int64_t* rows);

/* First half of a sharded KDK step of dt (the order of steps_cyl_kdk_step): the
 * kick and drift factors of the Friedmann integration, then on the owned rows
 * p += g K1, x += p D, z wrapped into [0, L), the FP32 positions repacked. The
 * owned packed rows are written to send (device memory of the context's
 * device, 16-byte aligned, chunk x 8 floats; rows past the share are zeros).
 * The caller then gathers every rank's send buffer, in rank order, into one
 * buffer of world x chunk x 8 floats. Stream-ordered; returns without waiting. */
int steps_cyl_shard_drift(steps_cyl_ctx* ctx, double dt, float* send);

/* Second half of the step: the gathered packed rows of every rank (recv,
 * device memory, 16-byte aligned, world x chunk x 8 floats, rank order) become
 * the j-set; the pair force of the owned rows against all n particles, the
 * background and the second kick p += g K2 follow, and a and t advance.
 * STEPS_EINVAL unless steps_cyl_shard_drift came first. Synchronises the stream
 * to read the device error word (STEPS_EDEVICE). */
int steps_cyl_shard_kick(steps_cyl_ctx* ctx, const float* recv);

/* The symmetric sharded step. The row step above evaluates each of a rank's
 * rows against every j, one ordered pair at a time. On one GPU the FP32 direct
 * forms evaluate each unordered pair once instead (steps_cyl_last_eval), and
 * the symmetric step does the same across ranks, with a second exchange:
 *   steps_cyl_shard_drift    (as above; then the caller all-gathers send)
 *   steps_cyl_shard_force    this rank's equal share of the unordered pairs,
 *                            both particles of each, into sums
 *   (the caller reduce-scatters sums: 64-bit integer sums over the ranks)
 *   steps_cyl_shard_finish   this rank's rows from its reduced sums: the
 *                            background and p += g K2; a and t advance.
 * Integer sums make the step deterministic for a given world size.
 *
 * steps_cyl_shard_mode: *symmetric = 1 when the sharded context offers this step
 * (world > 1, S1xR2, not FP64, and the fixed-point scale of steps_cyl_last_eval's
 * symmetric kernels is usable); *sums_len (may be NULL) = world x 3 x chunk, the
 * int64 length of the sums buffer (0 without the step). */
int steps_cyl_shard_mode(steps_cyl_ctx* ctx, int32_t* symmetric, int64_t* sums_len);

/* The gathered rows (recv, as for steps_cyl_shard_kick) become the j-set; this
 * rank's 1/world share of the unordered pairs is evaluated and every pair added
 * to both its particles in sums: device memory, 16-byte aligned, int64
 * [world][3][chunk] (rank-major: rank q's rows, component by component), in
 * units of 2^-S of the fixed-point scale; zeroed and written whole. A NCCL
 * reduce-scatter of sums with ncclInt64 and ncclSum hands rank q its slice
 * [3][chunk]. STEPS_EINVAL without a symmetric step or after anything but
 * steps_cyl_shard_drift. Stream-ordered; returns without waiting. */
int steps_cyl_shard_force(steps_cyl_ctx* ctx, const float* recv, int64_t* sums);

/* Finish the step from own: device memory, 16-byte aligned, int64 [3][chunk],
 * the sums of this rank's rows added over every rank. STEPS_EINVAL unless
 * steps_cyl_shard_force came first. Synchronises the stream to read the device
 * error word (STEPS_EDEVICE). */
int steps_cyl_shard_finish(steps_cyl_ctx* ctx, const int64_t* own);

/* ---- learned far-image surrogate ------------------------------------------
 * The paper sums every image of the window (eq. ForceCylindrical). The
 * surrogate tail form (STEPS_TAIL_SURROGATE) sums the near images |k| <= n0
 * exactly and replaces the far tail of each pair by
 *   B1 + E (MLP(u) sc + mu)      (z component times sign(dz)),
 * B1 = continuum integral of the image cells with the first Euler-Maclaurin end
 * correction, E = (e^3, e^(5/2)), e = 1 / (dR^2 + (n0 + 1/2 + |dz|)^2) in units of
 * L, and a 3 -> 32 -> 32 -> 2 ReLU network of
 * u = (2 min(dR, dR_max)/dR_max - 1, 4|dz| - 1, 2 min(h, n0 + 1/2)/(n0 + 1/2) - 1)
 * evaluated in FP16 with FP32 accumulation on the tensor cores. Tail images
 * inside the softening support are corrected to the exact spline.
 *
 * Parameter vector (STEPS_SURR_NPARAM floats): W1[32][3], b1[32], W2[32][32],
 * b2[32], W3[2][32], b3[2], then mu[2], sc[2], dR_max. */
#define STEPS_SURR_NW 1250
#define STEPS_SURR_NPARAM 1255

typedef struct {
  int64_t n_samples;    /* training + held-out samples (the last 1/16 are held out) */
  int32_t epochs;
  int32_t batch;        /* multiple of 64 */
  double lr;            /* peak Adam learning rate, cosine decay to 0 */
  double dR_max;        /* input scale in units of L; 0 = 2.2 x the largest particle radius / L */
  uint64_t seed;        /* sample draw, initial weights, shuffling */
  double err_median;    /* acceptance bounds on the relative total-force error against the */
  double err_p999;      /* plain image sum over a particle sample (median, 99.9th percentile) */
  int32_t check_particles;
  int32_t reserved;     /* must be 0 */
} steps_cyl_train_cfg;

/* Defaults: 2^20 samples, 60 epochs, batch 8192, lr 3e-3, dR_max 0, seed 1,
 * bounds 1e-5 / 1e-3, 1024 check particles. */
int steps_cyl_train_cfg_default(steps_cyl_train_cfg* cfg);

/* Exact far-image tail sums in FP64 (no context): for each of ns samples
 * (dR, dz, h) in units of L (row-major ns x 3, |dz| <= 1/2, h > 0; host or device)
 * out[2 s], out[2 s + 1] = SR, SZ of the window images |dz + k| < n_cut with
 * |k| > n0, SR = sum F(r,h)/r and SZ = sum (dz + k) F(r,h)/r (eq. Force_spline_kernel).
 * n_cut = 0: the infinite line, images |k| <= 512 one by one and the continuum
 * cells beyond with their near end's Euler-Maclaurin term.
 * Requires 0 <= n0 < n_cut <= 4096, or n_cut = 0 and 0 <= n0 < 512; STEPS_EINVAL
 * otherwise, before any CUDA call.
 * out: host or device, ns x 2. Synchronises the stream. */
int steps_cyl_tail_sums(int64_t ns, const double* samples, int32_t n_cut, int32_t n0, double* out,
                        void* stream);

/* One forward and backward pass of the network in FP32 over ns samples (no
 * context): w (STEPS_SURR_NW floats), u (ns x 3), t (ns x 2) targets; *loss =
 * 1/(2 ns) sum |y - t|^2 and grad (STEPS_SURR_NW floats) its gradient. Host or
 * device pointers. Synchronises the stream. */
int steps_cyl_mlp_loss_grad(int64_t ns, const float* w, const float* u, const float* t, float* loss,
                            float* grad, void* stream);

/* Train the surrogate of a context on the GPU (its n_cut and n0): draw the
 * samples, compute exact FP64 targets, train with Adam, round to FP16, and
 * check the result against the plain image sum on cfg->check_particles
 * particles. For the infinite window (n_cut = 0) the targets are the infinite
 * line over the infinite base, and the check (here, in steps_cyl_set_surrogate,
 * steps_cyl_check_surrogate and the KDK's periodic checks) is against the
 * correction-table form built at init; a network dropped by a periodic check
 * hands the tail back to that table. report (8 doubles, may be NULL): final training loss, held-out
 * RMS error (normalised units), check median, check 99.9th percentile,
 * accepted (1/0), training ms, mu[0], sc[0]. Returns STEPS_OK when accepted
 * (the context may then use STEPS_TAIL_SURROGATE) or STEPS_ESURROGATE_REJECTED. */
int steps_cyl_train_surrogate(steps_cyl_ctx* ctx, const steps_cyl_train_cfg* cfg, double* report);

/* Load surrogate parameters (STEPS_SURR_NPARAM floats, host or device) and check
 * them as steps_cyl_train_surrogate does (bounds from the arguments; report: 4
 * doubles = check median, check 99.9th percentile, accepted, 0; may be NULL).
 * STEPS_ESURROGATE_REJECTED when the check fails (the parameters are dropped). */
int steps_cyl_set_surrogate(steps_cyl_ctx* ctx, const float* params, double err_median, double err_p999,
                            double* report);

/* Copy out the context's surrogate parameters (STEPS_SURR_NPARAM floats, host).
 * STEPS_ENOSURROGATE when none is loaded. */
int steps_cyl_get_surrogate(steps_cyl_ctx* ctx, float* params);

/* The network's tensor-core operands exactly as the surrogate kernels stage them
 * in shared memory, for checking the fragment layout on a host without a GPU
 * (no context, no CUDA call). The paper has no counterpart: the network is this
 * project's. params: STEPS_SURR_NPARAM floats (host) in the layout above.
 * lanes (host, 32 x STEPS_SURR_LANE_WORDS words, caller-owned) receives lane
 * L = 4g + t's record at lanes[L * STEPS_SURR_LANE_WORDS]:
 *   words 0-3   the first layer's B operand of mma.m16n8k8 (f16x2), n-block nb:
 *               rows 2t, 2t + 1 of column 8 nb + g of the 8 x 32 matrix whose
 *               rows are the weights of u0, u1, u2, then b1 (the input vector
 *               carries a constant 1 as its fourth component), then zeros;
 *   words 4-19  the hidden layer's B operands of mma.m16n8k16 (f16x2), [nb][kb]
 *               {rows 16 kb + 2t, +1 | 16 kb + 2t + 8, +9} of column 8 nb + g;
 *   words 20-23 the output layer's B operands for the even m-tile, [kb]: column
 *               g carries output g & 1 for g < 4, zero for g >= 4;
 *   words 24-27 the same for the odd m-tile (columns g >= 4);
 *   words 28-43 the hidden bias b2 as FP32 C operands, [nb]: columns 8 nb + 2t,
 *               8 nb + 2t + 1 for rows g and g + 8.
 * shift (host, 2 floats) receives the output shift mu + sc b3 the kernels add,
 * so that the tail is B1 + E (y sc + shift) with y the network without b3.
 * STEPS_EINVAL for a NULL pointer. */
#define STEPS_SURR_LANE_WORDS 44
int steps_cyl_surrogate_lanes(const float* params, uint32_t* lanes, float* shift);

/* Select the tail form: STEPS_TAIL_FULL, STEPS_TAIL_SURROGATE or
 * STEPS_TAIL_TABLE (a modelled tail requires an accepted network / table and an
 * FP32 precision; the infinite window refuses STEPS_TAIL_FULL). As with
 * steps_cyl_set_precision the cached forces are refreshed by the next force
 * evaluation or KDK step. */
int steps_cyl_set_tail(steps_cyl_ctx* ctx, int32_t tail);

/* ---- correction-table tail -----------------------------------------------
 * Sect. 2.3, eq. S1R2EwaldCorrectionTable: the paper tabulates the force of the
 * periodic images beyond the nearest on an equally spaced (rho, z) grid and adds
 * it, read with cloud-in-cell or triangular-shaped-cloud interpolation, to the
 * nearest-image force. Here
 * the table holds the images beyond the near range |k| <= n0 of the context's
 * window (eq. ForceCylindrical), for point masses, as the residual of that tail
 * over the continuum base in envelope units (the quantity the surrogate
 * learns), at nodes dR_i = i dR_max / (nx - 1), |dz|_j = j / (2 (ny - 1)) in
 * units of L; dR beyond dR_max reads the last column. It is computed in FP64 on
 * the GPU, stored in FP32 and read with the texture unit's bilinear filter
 * (CIC, the default), or with TSC weights: in node units x, the nearest node i
 * and d = x - i weigh nodes i - 1, i, i + 1 by (1/2 - d)^2 / 2, 3/4 - d^2,
 * (1/2 + d)^2 / 2 per axis (four bilinear fetches), a node beyond the edge
 * taking the edge value. TSC smooths the table by a quarter of a cell squared
 * times its curvature, so at the same grid it is less accurate than CIC. The
 * table form (STEPS_TAIL_TABLE) sums the near images exactly, adds
 * base + envelope x table, and corrects tail images inside the softening support
 * exactly, as the surrogate form does. With n_cut = 0 (the infinite window) the
 * table holds the whole image line beyond n0, summed exactly to |k| = 512 and
 * by Euler-Maclaurin beyond, over the base of the infinite window; no plain sum
 * exists to check it against, so it is kept without a check.
 * With n0 = 0 the table is the paper's own, over the nearest image alone
 * (D = F_S1xR2 - F_R3 of the nearest image): the continuum base would reach the
 * pair itself at |dz| = 1/2, so the nodes hold the tail sums themselves (no
 * base, unit envelope). Its interpolation error is far larger than the
 * residual's (about 1.4e-4 of the force at the median on a 144 x 128 grid,
 * against 4e-10 with n0 = 4), so the 1e-5 check rejects it at such grids. The
 * learned tail needs n0 >= 1. */

/* Build the context's table (its n_cut and n0; 0 <= n0 < n_cut, or 0 <= n0 < 512
 * for the infinite window; FP32 precision) and, for a finite window, compare the table form with the plain image sum on
 * check_particles particles; keep it when median <= err_median and 99.9th
 * percentile <= err_p999 of the relative total-force error. nx in [2, 4096], ny
 * in [2, 1024]; dR_max = 0 picks 2.2 x the largest particle radius / L. report
 * (4 doubles, may be NULL): check median, 99.9th percentile, accepted (1/0),
 * build ms. STEPS_ESURROGATE_REJECTED when the check fails (the table is not
 * used). The context may then select STEPS_TAIL_TABLE. */
int steps_cyl_build_tail_table(steps_cyl_ctx* ctx, int32_t nx, int32_t ny, double dR_max, double err_median,
                               double err_p999, int32_t check_particles, double* report);

/* The infinite window's table (n_cut = 0) from the Ewald summation of the line
 * (Sect. 2.3, eqs. cylindricalEwaldSplit, EwaldRealSum, EwaldRecSum and the
 * m = 0 term) instead of the direct sum: in FP64 on the GPU, the real-space
 * images |k| <= nmax screened by erfc at split parameter alpha (units 1/L; the
 * near images |k| <= n0 keep only their smooth long-range part, so that they
 * are left out of the tail), Fourier modes k = 2 pi m, 1 <= m <= mmax, and the
 * m = 0 line term. The Fourier kernel is the incomplete Bessel integral
 * Int_0^{alpha^2} exp(-rho^2 t - k^2 / (4 t)) dt / t, which tends to
 * 2 K0(k rho) as alpha grows, as the kernel of a line must; the printed
 * eq. Bkernel is the doubly periodic slab's kernel (its limit is 2 exp(-k rho)),
 * so the paper's formula is read as this integral. nmax = 5, mmax = 12 at
 * alpha = 1 is the paper's single-precision setting. Nodes, layout and read as
 * for steps_cyl_build_tail_table; the direct construction runs beside it for
 * the report (4 doubles, may be NULL): the largest node difference and the
 * largest node magnitude (envelope units), Ewald build ms, direct build ms. The
 * Ewald nodes are installed. STEPS_EINVAL for a finite window, FP64 precision,
 * a sharded context, alpha outside [0.25, 8], nmax < n0 or above 64, mmax
 * outside [0, 64], or the nx, ny and dR_max bounds above. A checkpoint restores
 * the table through the direct construction. */
int steps_cyl_build_tail_table_ewald(steps_cyl_ctx* ctx, int32_t nx, int32_t ny, double dR_max, double alpha,
                                     int32_t nmax, int32_t mmax, double* report);

/* Choose the read of the correction table: STEPS_TABLE_READ_CIC (the default)
 * or STEPS_TABLE_READ_TSC. It applies from the next steps_cyl_build_tail_table
 * or steps_cyl_build_tail_table_ewald, whose check (finite window) then tests
 * the table form in that read; a table already built keeps the read it was
 * built with. A checkpoint records the read of its table. STEPS_EINVAL for any
 * other value. */
int steps_cyl_set_table_read(steps_cyl_ctx* ctx, int32_t read);

/* Copy out the context's table: out = ny x nx x 2 floats (host; may be NULL to
 * read only the sizes), its nx, ny and dR_max (each may be NULL).
 * STEPS_ENOSURROGATE when no table was built. */
int steps_cyl_get_tail_table(steps_cyl_ctx* ctx, float* out, int32_t* nx, int32_t* ny, double* dR_max);

/* ---- octree (Sect. 2.4) ------------------------------------------------------
 * A Barnes-Hut tree drawn at every force evaluation in a random frame. S1xR2: a
 * cube of side S = 2 max(L, 2 R_sim), shifted by zeta along the axis and
 * rotated by phi about it (x' = cos phi x - sin phi y, y' = sin phi x +
 * cos phi y, z' = z + zeta mod L). R^3: a cube of side 4 R_sim centred at a
 * point within R_sim / 2 of the origin, rotated by an angle about a unit axis
 * (Rodrigues), no period. Particles are grouped by 32 in Morton order
 * of the frame; a group opens a node when any member sees it under an angle
 * s / d >= theta or closer than the softening allows; accepted nodes act as
 * point masses at their centre of mass. Every interaction is the pair force of
 * the direct form: in S1xR2 the infinite window (near images exact, the rest from
 * the correction table), in R^3 eq. NewtonianForce. An optional radial correction
 * (Sect. 2.4) subtracts the mean radial force error measured by
 * steps_cyl_tree_calibrate (radius: cylindrical in S1xR2, spherical in R^3). */

/* Fix the frame of the following force evaluations (S1xR2: zeta in [0, L), phi in
 * radians); zeta < 0 returns to a random frame per evaluation. */
int steps_cyl_tree_frame(steps_cyl_ctx* ctx, double zeta, double phi);

/* R^3: fix the frame to frame[7] = (centre x, y, z within R_sim / 2 of the origin,
 * unit rotation axis x, y, z, angle in radians); NULL returns to random frames. */
int steps_cyl_tree_frame_r3(steps_cyl_ctx* ctx, const double* frame);

/* Statistics of the last octree evaluation: out[0] nodes, out[1] depth,
 * out[2] pair interactions (member x entry), out[3] build ms, out[4] walk ms,
 * out[5] evaluations so far. STEPS_EINVAL unless the context uses the octree. */
int steps_cyl_tree_stats(steps_cyl_ctx* ctx, double* out);

/* Radial calibration of Sect. 2.4: for n_frames frames (frames: 2 n_frames
 * doubles (zeta, phi) in S1xR2, 7 n_frames doubles (centre, axis, angle) in R^3,
 * or NULL to draw them) compare the octree's pair force with the direct pair
 * force (S1xR2: the table form in FP32; R^3: FP64) on n_sample particles
 * (sample: caller indices, or NULL to draw them) and average the radial
 * component of the difference in n_bins bins of the radius over [0, rmax], rmax
 * the largest particle radius now.
 * Empty bins hold 0. The table is then subtracted from the octree force at
 * every evaluation (interpolated linearly between bin centres, held beyond
 * them). n_frames = 0 removes the correction. table (n_bins doubles, may be
 * NULL) and rmax (may be NULL) receive the result. */
int steps_cyl_tree_calibrate(steps_cyl_ctx* ctx, int32_t n_frames, int32_t n_bins, int32_t n_sample,
                             const double* frames, const int64_t* sample, double* table, double* rmax);

/* Install a radial correction table measured elsewhere (n_bins doubles, host, in the
 * units steps_cyl_tree_calibrate returns: comoving a^3 g; bins over [0, rmax]), e.g.
 * the initial load's calibration in a later context. n_bins in [1, 4096], rmax > 0. */
int steps_cyl_tree_set_radial(steps_cyl_ctx* ctx, const double* table, int32_t n_bins, double rmax);

/* As steps_cyl_check_surrogate for a modelled tail (STEPS_TAIL_SURROGATE or
 * STEPS_TAIL_TABLE), which must be loaded and accepted. STEPS_EINVAL for the
 * infinite window (no plain image sum exists). */
int steps_cyl_check_tail(steps_cyl_ctx* ctx, int32_t tail, int32_t check_particles, double* report);

/* Compare the surrogate form with the plain image sum now on check_particles
 * particles (deterministic sample): report (4 doubles) = median and 99.9th
 * percentile of the relative total-force error, and the two forms' pair-kernel
 * times in ms on that sample. */
int steps_cyl_check_surrogate(steps_cyl_ctx* ctx, int32_t check_particles, double* report);

/* ---- allocation-free pair accelerations ----------------------------------
 * This entry point has no counterpart in the paper. It serves callers that may
 * not allocate device memory: a host whose device memory is owned and budgeted
 * by another allocator (a caching allocator or an arena reserved at start-up), a
 * loop that must not take cudaMalloc's implicit device-wide synchronisation, or
 * a plug-in that may allocate only while it initialises. Its result is what
 * steps_cyl_forces returns for a context with background STEPS_BG_OFF in static
 * space (a = 1), computed with the same kernels, and it calls no cudaMalloc,
 * cudaFree or allocating library routine. Its scratch (packed positions and the
 * work split's partial sums) is one file-scope device array of
 * STEPS_NOALLOC_SCRATCH_BYTES bytes that every device loading this library
 * holds until the process exits.
 *   - n: 2 <= n <= STEPS_NOALLOC_MAX_N, else STEPS_EINVAL (nothing is launched).
 *   - x, y, z, m, h (inputs) and ax, ay, az (outputs): device (or managed)
 *     memory of the calling thread's current device, n doubles each; z in
 *     [0, L); m, h > 0. A host pointer, pinned or not, or another device's
 *     memory gives STEPS_EINVAL before anything is launched (checked with
 *     cudaPointerGetAttributes; the lengths cannot be checked here).
 *   - precision: STEPS_FP32_KAHAN or STEPS_FP32_PLAIN; n_cut in [1, 4096];
 *     G, L > 0. stream: cudaStream_t to enqueue on (NULL = legacy default).
 *   - The call returns once the work is enqueued and never synchronises, so it
 *     keeps no device error word: non-finite results are not reported (check
 *     the outputs). STEPS_ECUDA when a runtime call or a launch of this call
 *     fails; an error left pending by the caller's earlier work is neither
 *     cleared nor reported as this call's.
 *   - The first call on a device looks up the array's device address
 *     (cudaGetSymbolAddress, with that device current); make that first call
 *     before any stream capture.
 *   - Every call uses the same array and leaves its contents behind: calls whose
 *     work overlaps on the GPU (two streams, two threads) race and give wrong
 *     results, so serialise them. */
#define STEPS_NOALLOC_MAX_N 65536
#define STEPS_NOALLOC_MAX_CTAS 2048
#define STEPS_NOALLOC_SCRATCH_BYTES 9961472
int steps_cyl_pair_accel_noalloc(int64_t n, const double* x, const double* y, const double* z,
                                 const double* m, const double* h, double G, double L,
                                 int32_t n_cut, int32_t precision, double* ax, double* ay,
                                 double* az, void* stream);

/* Write the complete state of a context to a file: parameters, a and t, the
 * background table, positions, momenta, masses, softenings and the cached forces
 * in the library's internal particle order with its permutation, the re-order
 * and check counters and any accepted surrogate. Synchronises the stream. */
int steps_cyl_checkpoint(steps_cyl_ctx* ctx, const char* path);

/* Create a context from a checkpoint file on the given device and stream. The
 * resumed context continues bit-identically to the one that wrote the file.
 * STEPS_EINVAL for a missing, foreign or truncated file, and for a corrupt one.
 * That covers a file whose size differs from what its header implies, a
 * permutation that is not one of [0, n), and a finite-cylinder background
 * without its table. It also covers a non-finite or non-positive a, a
 * non-finite t or rho0, and a fixed octree frame that steps_cyl_tree_frame
 * would refuse. These checks, except the frame's, run before any CUDA call. */
int steps_cyl_resume(steps_cyl_ctx** out, const char* path, int32_t device, void* stream);

/* Release the context and its device memory. NULL is accepted. */
int steps_cyl_free(steps_cyl_ctx* ctx);

/* Static description of a status code; never NULL. */
const char* steps_cyl_strerror(int code);

/* Message of the last failure on the calling thread ("" when none). */
const char* steps_cyl_last_error(void);

#ifdef __cplusplus
}
#endif
#endif
