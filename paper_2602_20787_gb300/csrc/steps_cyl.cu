// C ABI of the S1xR2 StePS hot path (arXiv 2602.20787) on GB300 / sm_103a.
// Declarations and the contract of every entry point are in include/steps_cyl.h.
//
// Host side of the library: context, argument checks, the FP64 Friedmann/RK4
// schedule of the kick and drift factors (Sect. 2.3), the tabulated finite-height
// part of the background term (eq. F_horiz), and the launch sequence of a force
// evaluation and of a KDK step. All particle work runs in the kernels of
// pair_fp32.cuh and nbody_kernels.cuh.
//
// Particle order. Inside a context the particles are kept in an internal order
// along a Morton (Z-order) curve of (x, y), so that the 32 i-particles of a warp
// are close in the transverse plane: their pairs with a given j are then
// softened together or not at all, which keeps the warp-uniform spline bound of
// the pair kernel small. perm[k] is the caller's index of internal particle k;
// every input is gathered through perm and every output scattered back, so the
// caller only ever sees its own order. The order is rebuilt at init, when
// set_state moves particles, and every reorder_every KDK steps.
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "steps_cyl.h"
#include "nbody_kernels.cuh"
#include "surrogate_pair.cuh"
#include "surrogate_train.cuh"
#include "tail_table.cuh"
#include "octree.cuh"
#include "r3_pair.cuh"
#include "pair_sym.cuh"

using namespace steps;

// CTAs of the pair kernel per resident slot (build-time tuning knob): more CTAs
// than slots lets the block scheduler even out CTAs whose work differs.
#ifndef STEPS_CTA_MULT
#define STEPS_CTA_MULT 32
#endif

namespace {

thread_local std::string g_last_error;

// A named host range over one phase of an evaluation or a step, for profilers
// that record NVTX ranges; without one attached the calls do nothing.
struct Range {
  explicit Range(const char* name) { nvtxRangePushA(name); }
  ~Range() { nvtxRangePop(); }
  Range(const Range&) = delete;
  Range& operator=(const Range&) = delete;
};

int fail(int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_last_error = buf;
  return code;
}

#define CK(call)                                                                        \
  do {                                                                                  \
    cudaError_t e_ = (call);                                                            \
    if (e_ != cudaSuccess) return fail(STEPS_ECUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
  } while (0)

#define CKLAUNCH(what)                                                                  \
  do {                                                                                  \
    cudaError_t e_ = cudaGetLastError();                                                \
    if (e_ != cudaSuccess) return fail(STEPS_ECUDA, "launch %s: %s", what, cudaGetErrorString(e_)); \
  } while (0)

// ---------------------------------------------------------------------------
// Background cosmology: eqs. Friedmann, DEdensity (closed form for the CPL w(a)
// of eq. CPLw0wa) and the RK4 integration of a(t) (Sect. 2.3). The kick and drift
// factors of the KDK step in canonical momentum p = a^2 dx/dt are
//   K1 = Int_{t}^{t+dt/2} dt'/a,  K2 = Int_{t+dt/2}^{t+dt} dt'/a,  D = Int_t^{t+dt} dt'/a^2,
// integrated together with a by classical RK4 over each half step.
// ---------------------------------------------------------------------------
struct Cosmology {
  double H0, Om, Or, OL, w0, wa;
  bool comoving;

  double E2(double a) const {
    const double ok = 1.0 - Om - Or - OL;
    const double de = OL * std::pow(a, -3.0 * (1.0 + w0 + wa)) * std::exp(3.0 * wa * (a - 1.0));
    return Or / (a * a * a * a) + Om / (a * a * a) + ok / (a * a) + de;
  }
  double H(double a) const { return H0 * std::sqrt(E2(a)); }
};

struct Factors {
  double K1, D, K2, a_next;
};

// derivative of (a, Int dt/a, Int dt/a^2) with respect to t
static inline void friedmann_rhs(const Cosmology& c, const double y[3], double f[3]) {
  f[0] = y[0] * c.H(y[0]);
  f[1] = 1.0 / y[0];
  f[2] = 1.0 / (y[0] * y[0]);
}

static void rk4_half(const Cosmology& c, double a, double dt, double out[3]) {
  double y[3] = {a, 0.0, 0.0}, k1[3], k2[3], k3[3], k4[3], tmp[3];
  friedmann_rhs(c, y, k1);
  for (int q = 0; q < 3; ++q) tmp[q] = y[q] + 0.5 * dt * k1[q];
  friedmann_rhs(c, tmp, k2);
  for (int q = 0; q < 3; ++q) tmp[q] = y[q] + 0.5 * dt * k2[q];
  friedmann_rhs(c, tmp, k3);
  for (int q = 0; q < 3; ++q) tmp[q] = y[q] + dt * k3[q];
  friedmann_rhs(c, tmp, k4);
  for (int q = 0; q < 3; ++q) out[q] = y[q] + dt * (k1[q] + 2.0 * (k2[q] + k3[q]) + k4[q]) / 6.0;
}

static Factors kdk_factors(const Cosmology& c, double a, double dt) {
  if (!c.comoving) return Factors{0.5 * dt, dt, 0.5 * dt, 1.0};
  double first[3], second[3];
  rk4_half(c, a, 0.5 * dt, first);
  rk4_half(c, first[0], 0.5 * dt, second);
  return Factors{first[1], first[2] + second[2], second[1], second[0]};
}

// ---------------------------------------------------------------------------
// Finite-height part of the background (eq. F_horiz, re-derived):
//   F_h(rho) = F_inf(rho) + dF(rho),
//   dF(rho) = 4 G rho0 Int_0^R ln((sqrt(Lw^2+A)+Lw)/(sqrt(Lw^2+B)+Lw)) dY,
//   A, B = R^2 + rho^2 +- 2 rho sqrt(R^2 - Y^2),  Lw = Ncut L.
// With Y = R sin(theta) the integrand is analytic on [0, pi/2] (Lw > 0 keeps the
// logarithm away from zero), so a composite Gauss-Legendre rule converges
// geometrically. Nodes and weights come from Newton's method on P_n.
// ---------------------------------------------------------------------------
static void gauss_legendre(int n, std::vector<double>& x, std::vector<double>& w) {
  x.assign(n, 0.0);
  w.assign(n, 0.0);
  for (int i = 0; i < n; ++i) {
    double z = std::cos(M_PI * (i + 0.75) / (n + 0.5));
    for (int it = 0; it < 100; ++it) {
      double p0 = 1.0, p1 = z;
      for (int k = 2; k <= n; ++k) {
        const double pk = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
        p0 = p1;
        p1 = pk;
      }
      const double dp = n * (z * p1 - p0) / (z * z - 1.0);
      const double dz = p1 / dp;
      z -= dz;
      if (std::fabs(dz) < 1e-16) {
        double q0 = 1.0, q1 = z;
        for (int k = 2; k <= n; ++k) {
          const double qk = ((2.0 * k - 1.0) * z * q1 - (k - 1.0) * q0) / k;
          q0 = q1;
          q1 = qk;
        }
        const double dq = n * (z * q1 - q0) / (z * z - 1.0);
        x[i] = z;
        w[i] = 2.0 / ((1.0 - z * z) * dq * dq);
        break;
      }
    }
  }
}

static double finite_height_dF(double rho, double R, double Lw, double G, double rho0,
                               const std::vector<double>& gx, const std::vector<double>& gw, int panels) {
  const double a = 0.0, b = 0.5 * M_PI, hp = (b - a) / panels;
  double acc = 0.0;
  for (int p = 0; p < panels; ++p) {
    const double mid = a + (p + 0.5) * hp, half = 0.5 * hp;
    double s = 0.0;
    for (size_t k = 0; k < gx.size(); ++k) {
      const double th = mid + half * gx[k];
      const double sn = std::sin(0.5 * th);
      const double q = 4.0 * rho * R * sn * sn;
      const double A = (R + rho) * (R + rho) - q;
      const double B = (R - rho) * (R - rho) + q;
      const double lg = std::log((std::sqrt(Lw * Lw + A) + Lw) / (std::sqrt(Lw * Lw + B) + Lw));
      s += gw[k] * lg * R * std::cos(th);
    }
    acc += s * half;
  }
  return 4.0 * G * rho0 * acc;
}

bool is_host_ptr(const void* p) {
  if (!p) return false;
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return true;
  }
  return at.type != cudaMemoryTypeDevice && at.type != cudaMemoryTypeManaged;
}

int grid_for(int n, int threads) {
  long long g = ((long long)n + threads - 1) / threads;
  return (int)std::max(1LL, std::min(g, 152LL * 32));
}

}  // namespace

// ---------------------------------------------------------------------------
// One octree frame (Sect. 2.4): S1xR2 uses (zeta, phi); R^3 the domain centre,
// the rotation axis (unit) and angle.
struct TreeDraw {
  double zeta, phi;
  double cen[3], axis[3], angle;
};

struct steps_cyl_ctx {
  steps_cyl_params p{};
  int n = 0;
  int dev = 0;
  cudaStream_t st = nullptr;
  Cosmology cosmo{};
  double a = 1.0, t = 0.0, rho0 = 0.0, invL = 1.0;
  // device state (FP64 SoA, internal order)
  double* state = nullptr;  // one allocation for the 11 arrays below
  double *x, *y, *z, *px, *py, *pz, *m, *h, *gx, *gy, *gz;
  float4* jA = nullptr;
  float4* jB = nullptr;
  double* part = nullptr;   // stream-K partials or direct FP64 sums; also a permutation temporary
  size_t part_elems = 0;
  double* stage = nullptr;  // 3 n doubles: inputs and outputs in the caller's order
  double* red = nullptr;    // reduction scratch
  int* perm = nullptr;      // internal -> caller index (device)
  int* iperm = nullptr;     // caller -> internal index (device)
  int* ord = nullptr;       // re-ordering of internal indices (device)
  std::vector<int> perm_h;  // host copy of perm
  int64_t* idx = nullptr;   // subset indices (grown on demand)
  int idx_cap = 0;
  double* sub = nullptr;    // subset sums (3 * idx_cap)
  int* err = nullptr;
  double* bgtab = nullptr;
  int bgK = 0;
  double bg_dr = 0.0;
  int C = 0, NT = 0, NB = 0;
  long long U = 0;
  // Rows evaluated by the pair kernels: i-blocks [b0, b0 + nbo), internal rows
  // [k0, k1). All of them unless the rows are sharded (steps_cyl_shard); U and
  // the CTA counts C, SC, TC are those of this range, capped at Ccap etc.
  int b0 = 0, nbo = 0, k0 = 0, k1 = 0;
  int Ccap = 0, SCcap = 0, TCcap = 0;
  // symmetric (Newton's third law) evaluation into fixed-point accumulators
  unsigned long long* facc = nullptr;  // [3][n]
  double fix_scale = 0.0;              // 2^S
  double h_max = 0.0;                  // the largest softening (set with fix_scale)
  bool fix_ready = false, fix_ok = false;
  long long Usym = 0;
  int SYC = 0, SYSC = 0, SYTC = 0;     // CTAs of the symmetric plain / surrogate / table kernels
  // row sharding
  bool shard = false;
  int shard_rank = 0, shard_world = 1, chunk = 0;
  int* shard_off = nullptr;       // device: world + 1 row offsets
  bool drifted = false;           // steps_cyl_shard_drift done, steps_cyl_shard_kick pending
  bool shard_sym = false;         // the symmetric two-exchange step is available
  bool forced = false;            // steps_cyl_shard_force done, steps_cyl_shard_finish pending
  double pend_K2 = 0.0, pend_a = 0.0, pend_dt = 0.0;
  int steps_since_order = 0;
  bool forces_stale = false;       // g must be recomputed before the next kick
  // learned far-image surrogate
  SurrLane* surr_lanes = nullptr;  // per-lane MLP fragments (device, 32 entries)
  SurrConst surr{};
  std::vector<float> surr_params;  // STEPS_SURR_NPARAM floats of the accepted network
  bool surr_ok = false;            // an accepted network is loaded
  int steps_since_check = 0;
  double surr_bound_med = 1e-5, surr_bound_p999 = 1e-3;
  int SC = 0;                      // CTAs of the surrogate pair kernel
  // correction-table tail
  cudaArray_t tab_arr = nullptr;
  TableTail tab{};                 // texture of the residual table
  SurrConst tab_const{};           // mu = 0, sc = 1, the table's dR_max
  int tab_nx = 0, tab_ny = 0;
  int tab_read_next = STEPS_TABLE_READ_CIC;  // the read of the next table build (tab.read: the built one's)
  double tab_dR_max = 0.0;
  bool tab_ok = false;             // an accepted table is loaded
  double tab_bound_med = 1e-5, tab_bound_p999 = 1e-3;
  int TC = 0;                      // CTAs of the table pair kernel
  double* chk = nullptr;           // check buffers (grown on demand)
  size_t chk_elems = 0;
  // octree (force == STEPS_FORCE_OCTREE)
  struct Tree {
    uint64_t* key[2] = {nullptr, nullptr};  // radix-sort ping-pong: keys and internal indices
    int* val[2] = {nullptr, nullptr};
    unsigned *hist = nullptr, *offs = nullptr;
    float4 *u4 = nullptr, *u4s = nullptr;   // tree-frame coordinates (internal / key order)
    double* zt = nullptr;                   // z in the tree frame (internal order)
    float4 *sA = nullptr, *sB = nullptr;    // packed particles in key order
    int node_cap = 0, slot_cap = 0;
    int4* link = nullptr;
    float4* geo = nullptr;
    float* hmf = nullptr;
    uint64_t* pre = nullptr;
    double4_32a* mom = nullptr;
    double* hmx = nullptr;
    float4 *nA = nullptr, *nB = nullptr;
    int *active[2] = {nullptr, nullptr};
    int *cnt = nullptr, *beg = nullptr, *pos = nullptr, *totals = nullptr;
    int* totals_h = nullptr;                // pinned
    unsigned long long* inter = nullptr;
    int nodes = 0, depth = 0;
    double interactions = 0.0, build_ms = 0.0, walk_ms = 0.0;
    bool ready = false;                     // every per-particle buffer above is allocated
    bool fixed = false;
    TreeDraw fd{};                          // the fixed frame
    uint64_t evals = 0;
    double* rad = nullptr;                  // radial correction table (device)
    int rad_nb = 0;
    double rad_rmax = 0.0;
    std::vector<double> rad_h;
    cudaEvent_t t0 = nullptr, t1 = nullptr, t2 = nullptr;
  } tr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  double last_images = 0.0;
  double last_pairs = 0.0;   // pairs the last pair kernel evaluated
  bool last_sym = false;     // ... with the symmetric kernels
  bool last_straight = false;  // ... taking the straight run of the modelled tails
  bool timed = false;
};

namespace {

BgParams bg_params(const steps_cyl_ctx* c) {
  BgParams b;
  b.mode = c->p.background;
  b.two_pi_G_rho0 = 2.0 * M_PI * c->p.G * c->rho0;
  b.R = c->p.R_sim;
  b.tab = c->bgtab;
  b.K = c->bgK;
  b.inv_dr = c->bg_dr > 0 ? 1.0 / c->bg_dr : 0.0;
  return b;
}

bool is_r3(const steps_cyl_ctx* c) { return c->p.topology == STEPS_TOPO_R3; }
// Images per pair: the window's 2 Ncut (S1xR2), the one image of R^3.
bool is_inf(const steps_cyl_ctx* c) { return c->p.n_cut == 0; }  // Ncut -> infinity
// Images per pair: the window's 2 Ncut (S1xR2), the one image of R^3, and the
// 2 n0 + 1 exact images of the infinite window (its tail is the table's).
double images_per_pair(const steps_cyl_ctx* c) {
  return is_r3(c) ? 1.0 : is_inf(c) ? 2.0 * c->p.n0 + 1.0 : 2.0 * c->p.n_cut;
}
int n_cut_eff(const steps_cyl_ctx* c) { return is_r3(c) ? 1 : c->p.n_cut; }

int check_params(const steps_cyl_params* p) {
  if (!p) return fail(STEPS_EINVAL, "params is NULL");
  if (!(p->G != 0) || !std::isfinite(p->G)) return fail(STEPS_EINVAL, "G must be finite and != 0");
  if (p->topology != STEPS_TOPO_S1R2 && p->topology != STEPS_TOPO_R3) return fail(STEPS_EINVAL, "bad topology");
  if (p->reserved != 0) return fail(STEPS_EINVAL, "reserved must be 0");
  if (p->topology == STEPS_TOPO_R3 && p->tail != STEPS_TAIL_FULL)
    return fail(STEPS_EINVAL, "the R^3 topology has no image tail (tail must be STEPS_TAIL_FULL)");
  if (p->topology == STEPS_TOPO_R3 && p->background != STEPS_BG_OFF && p->background != STEPS_BG_SPHERE)
    return fail(STEPS_EINVAL, "the R^3 topology takes STEPS_BG_OFF or STEPS_BG_SPHERE");
  if (p->topology == STEPS_TOPO_S1R2 && p->background == STEPS_BG_SPHERE)
    return fail(STEPS_EINVAL, "STEPS_BG_SPHERE belongs to the R^3 topology");
  if (!(p->L > 0) || !std::isfinite(p->L)) return fail(STEPS_EINVAL, "L must be finite and > 0");
  if (!(p->R_sim > 0) || !std::isfinite(p->R_sim)) return fail(STEPS_EINVAL, "R_sim must be finite and > 0");
  if (!(p->rho_bar >= 0) || !std::isfinite(p->rho_bar)) return fail(STEPS_EINVAL, "rho_bar must be >= 0");
  if (p->n_cut < 0 || p->n_cut > 4096) return fail(STEPS_EINVAL, "n_cut must be in [0, 4096] (0: infinite window)");
  if (p->n_cut == 0) {  // Ncut -> infinity: a modelled tail carries the whole line beyond n0
    if (p->topology != STEPS_TOPO_S1R2) return fail(STEPS_EINVAL, "the infinite window belongs to S1xR2");
    if (p->tail == STEPS_TAIL_FULL) return fail(STEPS_EINVAL, "the infinite window needs a modelled tail");
    if (p->precision == STEPS_FP64) return fail(STEPS_EINVAL, "the infinite window needs an FP32 precision");
    if (p->background != STEPS_BG_OFF && p->background != STEPS_BG_INFINITE)
      return fail(STEPS_EINVAL, "the infinite window takes STEPS_BG_INFINITE or STEPS_BG_OFF");
    // the tail sums images |k| <= kKInf one by one and the line ends beyond, so the
    // near range must end inside that range
    if (p->n0 < 0 || p->n0 >= kKInf) return fail(STEPS_EINVAL, "n0 must be in [0, %d) for the infinite window", kKInf);
    if (p->n0 == 0 && p->tail != STEPS_TAIL_TABLE)
      return fail(STEPS_EINVAL, "n0 = 0 (the table over the nearest image) needs STEPS_TAIL_TABLE");
  }
  if (p->precision < STEPS_FP64 || p->precision > STEPS_FP32_PLAIN) return fail(STEPS_EINVAL, "bad precision");
  if (p->force != STEPS_FORCE_DIRECT && p->force != STEPS_FORCE_OCTREE) return fail(STEPS_EINVAL, "bad force method");
  if (p->force == STEPS_FORCE_OCTREE) {
    // the octree's node interactions are smooth only for the infinite window: with a finite
    // window the image set of a pair jumps at the window's edge, which no node moment follows
    if (p->topology == STEPS_TOPO_S1R2 && (p->n_cut != 0 || p->tail != STEPS_TAIL_TABLE))
      return fail(STEPS_EINVAL, "the octree needs the infinite window (n_cut = 0) with STEPS_TAIL_TABLE");
    if (p->precision == STEPS_FP64) return fail(STEPS_EINVAL, "the octree needs an FP32 precision");
    if (p->leaf_size < 1 || p->leaf_size > 64) return fail(STEPS_EINVAL, "leaf_size must be in [1, 64]");
    if (!(p->theta > 0.0 && p->theta <= 1.0)) return fail(STEPS_EINVAL, "theta must be in (0, 1]");
  }
  if (p->tail != STEPS_TAIL_FULL && p->tail != STEPS_TAIL_SURROGATE && p->tail != STEPS_TAIL_TABLE)
    return fail(STEPS_EINVAL, "bad tail mode");
  if (p->n0 < 0) return fail(STEPS_EINVAL, "n0 must be >= 0");
  if (p->tail == STEPS_TAIL_SURROGATE && p->n_cut > 0 && (p->n0 < 1 || p->n0 >= p->n_cut))
    return fail(STEPS_EINVAL, "the learned tail needs n0 in [1, n_cut)");
  if (p->tail == STEPS_TAIL_TABLE && p->n_cut > 0 && p->n0 >= p->n_cut)
    return fail(STEPS_EINVAL, "the table tail needs n0 in [0, n_cut)");
  if (p->background < STEPS_BG_OFF || p->background > STEPS_BG_SPHERE) return fail(STEPS_EINVAL, "bad background");
  if (p->comoving) {
    if (!(p->H0 > 0) || !(p->a_start > 0)) return fail(STEPS_EINVAL, "comoving runs need H0 > 0 and a_start > 0");
  }
  if (p->reorder_every < -1) return fail(STEPS_EINVAL, "reorder_every must be >= -1");
  if (p->check_every < 0 || p->check_particles < 0) return fail(STEPS_EINVAL, "check_every and check_particles must be >= 0");
  return STEPS_OK;
}

// Device-side check of the state: finite values, m > 0, h > 0, 0 <= z < L.
__global__ void validate_kernel(const double* __restrict__ x, const double* __restrict__ y,
                                const double* __restrict__ z, const double* __restrict__ px,
                                const double* __restrict__ py, const double* __restrict__ pz,
                                const double* __restrict__ m, const double* __restrict__ h, int n, double L,
                                int* __restrict__ bad) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    int b = 0;
    if (!isfinite(x[i]) || !isfinite(y[i]) || !isfinite(z[i]) || !isfinite(px[i]) || !isfinite(py[i]) ||
        !isfinite(pz[i]))
      b |= 1;
    if (!(m[i] > 0.0) || !isfinite(m[i])) b |= 2;
    if (!(h[i] > 0.0) || !isfinite(h[i])) b |= 4;
    if (L > 0.0 && !(z[i] >= 0.0 && z[i] < L)) b |= 8;  // S1xR2 only (L = 0: no period)
    if (b) atomicOr(bad, b);
  }
}

// Sets *changed when any staged position (caller order) differs bitwise from the
// current one (internal order).
__global__ void positions_changed_kernel(const double* __restrict__ x, const double* __restrict__ y,
                                         const double* __restrict__ z, const double* __restrict__ nx,
                                         const double* __restrict__ ny, const double* __restrict__ nz,
                                         const int* __restrict__ perm, int n, int* __restrict__ changed) {
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
    const int i = perm[k];
    if (__double_as_longlong(x[k]) != __double_as_longlong(nx[i]) ||
        __double_as_longlong(y[k]) != __double_as_longlong(ny[i]) ||
        __double_as_longlong(z[k]) != __double_as_longlong(nz[i])) {
      atomicOr(changed, 32);
    }
  }
}

__global__ void max_rho_kernel(const double* __restrict__ x, const double* __restrict__ y, int n,
                               unsigned long long* __restrict__ out) {
  double r = 0.0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    r = fmax(r, sqrt(x[i] * x[i] + y[i] * y[i]));
  // non-negative doubles order like their bit patterns
  atomicMax(out, (unsigned long long)__double_as_longlong(r));
}

// dst[k] = s * src[map[k]]
__global__ void gather_kernel(const double* __restrict__ src, const int* __restrict__ map, int n, double s,
                              double* __restrict__ dst) {
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) dst[k] = s * src[map[k]];
}

// dst[map[k]] = s * src[k]
__global__ void scatter_kernel(const double* __restrict__ src, const int* __restrict__ map, int n, double s,
                               double* __restrict__ dst) {
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) dst[map[k]] = s * src[k];
}

// dst[map[k]] = s * src[k] for k in [k0, k1), 0 for the other k
__global__ void scatter_rows_kernel(const double* __restrict__ src, const int* __restrict__ map, int n, double s,
                                    int k0, int k1, double* __restrict__ dst) {
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x)
    dst[map[k]] = (k >= k0 && k < k1) ? s * src[k] : 0.0;
}

__global__ void gather3_kernel(const double* __restrict__ ax, const double* __restrict__ ay,
                               const double* __restrict__ az, const int64_t* __restrict__ idx, int ni, double s,
                               double* __restrict__ ox, double* __restrict__ oy, double* __restrict__ oz) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q < ni) {
    const int64_t i = idx[q];
    ox[q] = s * ax[i]; oy[q] = s * ay[i]; oz[q] = s * az[i];
  }
}

// caller indices -> internal indices, flagging out-of-range entries
__global__ void map_idx_kernel(int64_t* __restrict__ idx, int ni, int n, const int* __restrict__ iperm,
                               int* __restrict__ bad) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q < ni) {
    const int64_t i = idx[q];
    if (i < 0 || i >= n) {
      atomicOr(bad, 16);
      idx[q] = 0;
    } else {
      idx[q] = iperm[i];
    }
  }
}

int read_and_clear_err(steps_cyl_ctx* c, int* out) {
  int h = 0;
  CK(cudaMemcpyAsync(&h, c->err, sizeof(int), cudaMemcpyDeviceToHost, c->st));
  CK(cudaStreamSynchronize(c->st));
  CK(cudaMemsetAsync(c->err, 0, sizeof(int), c->st));
#if STEPS_DEBUG_INDEX
  unsigned int ix = 0;
  CK(cudaMemcpyFromSymbolAsync(&ix, g_index_err, sizeof ix, 0, cudaMemcpyDeviceToHost, c->st));
  CK(cudaStreamSynchronize(c->st));
  if (ix) {
    const unsigned int zero = 0;
    CK(cudaMemcpyToSymbolAsync(g_index_err, &zero, sizeof zero, 0, cudaMemcpyHostToDevice, c->st));
    h |= kErrIndex;
  }
#endif
  *out = h;
  return STEPS_OK;
}

int device_error(int e) {
  return fail(STEPS_EDEVICE, "device error word 0x%x (%s%s%s%s%s%s%s)", e, (e & kErrNonFinite) ? "non-finite value " : "",
              (e & kErrBgRange) ? "particle beyond background table " : "", (e & kErrZRange) ? "z range " : "",
              (e & kErrTreeRange) ? "particle outside the octree root " : "",
              (e & kErrTreeStack) ? "octree walk stack overflow " : "",
              (e & kErrFixRange) ? "pair sum beyond the fixed-point range " : "",
              (e & kErrIndex) ? "index outside its buffer (index-checked build)" : "");
}

// Calls that need every row of the context current refuse a sharded context.
int refuse_sharded(const steps_cyl_ctx* c, const char* what) {
  return fail(STEPS_EINVAL, "%s: the context's rows are sharded (use steps_cyl_shard_drift / steps_cyl_shard_kick)",
              what);
}

// Morton (Z-order) rank of (x, y): stable sort of 2 x 16-bit interleaved cell
// codes over the bounding box. Returns order[k] = index of the k-th particle.
void morton_order(const std::vector<double>& x, const std::vector<double>& y, std::vector<int>& order) {
  const size_t n = x.size();
  double x0 = x[0], x1 = x[0], y0 = y[0], y1 = y[0];
  for (size_t i = 1; i < n; ++i) {
    x0 = std::min(x0, x[i]); x1 = std::max(x1, x[i]);
    y0 = std::min(y0, y[i]); y1 = std::max(y1, y[i]);
  }
  const double span = std::max({x1 - x0, y1 - y0, 1e-300});
  auto spread = [](uint32_t v) {
    v = (v | (v << 8)) & 0x00FF00FFu;
    v = (v | (v << 4)) & 0x0F0F0F0Fu;
    v = (v | (v << 2)) & 0x33333333u;
    v = (v | (v << 1)) & 0x55555555u;
    return v;
  };
  std::vector<uint32_t> key(n);
  for (size_t i = 0; i < n; ++i) {
    const double fx = (x[i] - x0) / span, fy = (y[i] - y0) / span;
    const uint32_t qx = (uint32_t)std::min(65535.0, std::max(0.0, std::floor(fx * 65536.0)));
    const uint32_t qy = (uint32_t)std::min(65535.0, std::max(0.0, std::floor(fy * 65536.0)));
    key[i] = spread(qx) | (spread(qy) << 1);
  }
  order.resize(n);
  for (size_t i = 0; i < n; ++i) order[i] = (int)i;
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return key[a] < key[b]; });
}

int upload_perm(steps_cyl_ctx* c) {
  std::vector<int> inv(c->n);
  for (int k = 0; k < c->n; ++k) inv[c->perm_h[k]] = k;
  CK(cudaMemcpyAsync(c->perm, c->perm_h.data(), sizeof(int) * c->n, cudaMemcpyHostToDevice, c->st));
  CK(cudaMemcpyAsync(c->iperm, inv.data(), sizeof(int) * c->n, cudaMemcpyHostToDevice, c->st));
  CK(cudaStreamSynchronize(c->st));  // the host vectors go out of scope
  return STEPS_OK;
}

// New caller->internal map from staged positions (caller order): the Morton
// order, or the caller's order when reorder_every == -1. With carry set, the
// per-particle arrays that are not re-uploaded (m, h) are moved from the old
// internal order to the new one.
int order_from_stage(steps_cyl_ctx* c, const double* sx, const double* sy, bool carry) {
  std::vector<int> np(c->n);
  if (c->p.reorder_every < 0) {
    for (int k = 0; k < c->n; ++k) np[k] = k;
  } else {
    std::vector<double> hx(c->n), hy(c->n);
    CK(cudaMemcpyAsync(hx.data(), sx, sizeof(double) * c->n, cudaMemcpyDeviceToHost, c->st));
    CK(cudaMemcpyAsync(hy.data(), sy, sizeof(double) * c->n, cudaMemcpyDeviceToHost, c->st));
    CK(cudaStreamSynchronize(c->st));
    morton_order(hx, hy, np);
  }
  if (carry) {
    std::vector<int> inv_old(c->n), o(c->n);
    for (int k = 0; k < c->n; ++k) inv_old[c->perm_h[k]] = k;
    for (int k = 0; k < c->n; ++k) o[k] = inv_old[np[k]];  // old internal index of new internal k
    CK(cudaMemcpyAsync(c->ord, o.data(), sizeof(int) * c->n, cudaMemcpyHostToDevice, c->st));
    double* tmp = c->part;
    for (double* arr : {c->m, c->h}) {
      gather_kernel<<<grid_for(c->n, 256), 256, 0, c->st>>>(arr, c->ord, c->n, 1.0, tmp);
      CK(cudaMemcpyAsync(arr, tmp, sizeof(double) * c->n, cudaMemcpyDeviceToDevice, c->st));
    }
    CKLAUNCH("carry");
    CK(cudaStreamSynchronize(c->st));  // o goes out of scope
  }
  c->perm_h.swap(np);
  c->steps_since_order = 0;
  return upload_perm(c);
}

int build_background(steps_cyl_ctx* c) {
  if (c->p.background != STEPS_BG_FINITE) return STEPS_OK;
  unsigned long long* dmax = nullptr;
  CK(cudaMallocAsync(&dmax, sizeof(unsigned long long), c->st));
  CK(cudaMemsetAsync(dmax, 0, sizeof(unsigned long long), c->st));
  max_rho_kernel<<<grid_for(c->n, 256), 256, 0, c->st>>>(c->x, c->y, c->n, dmax);
  CKLAUNCH("max_rho");
  unsigned long long hb = 0;
  CK(cudaMemcpyAsync(&hb, dmax, sizeof hb, cudaMemcpyDeviceToHost, c->st));
  CK(cudaStreamSynchronize(c->st));
  CK(cudaFreeAsync(dmax, c->st));
  double rmax_p;
  std::memcpy(&rmax_p, &hb, sizeof rmax_p);
  const double rmax = std::max(4.0 * c->p.R_sim, 2.0 * rmax_p);
  const int K = 4096;
  c->bgK = K;
  c->bg_dr = rmax / K;
  std::vector<double> gx, gw, tab(K + 4);
  gauss_legendre(16, gx, gw);
  const double Lw = c->p.n_cut * c->p.L;
  for (int k = -1; k <= K + 2; ++k)
    tab[k + 1] = finite_height_dF(k * c->bg_dr, c->p.R_sim, Lw, c->p.G, c->rho0, gx, gw, 16);
  CK(cudaMalloc(&c->bgtab, sizeof(double) * (K + 4)));
  CK(cudaMemcpyAsync(c->bgtab, tab.data(), sizeof(double) * (K + 4), cudaMemcpyHostToDevice, c->st));
  CK(cudaStreamSynchronize(c->st));
  return STEPS_OK;
}

// FP64 pair sums of the listed particles (all when idx == nullptr) into
// out[3][ni], with the j-range split across CTAs so that short lists fill the GPU.
int launch_fp64(steps_cyl_ctx* c, const int64_t* idx, int ni, double* out) {
  int sms = 0;
  CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c->dev));
  const int gx = (ni + 127) / 128;
  const int want = std::max(1, std::min(c->NT, (sms * 8 + gx - 1) / gx));
  const int tpc = (c->NT + want - 1) / want;
  const int JC = (c->NT + tpc - 1) / tpc;
  if (c->chk_elems < (size_t)JC * 3 * ni) {
    cudaFree(c->chk);
    c->chk = nullptr;
    c->chk_elems = 0;
    CK(cudaMalloc(&c->chk, sizeof(double) * (size_t)JC * 3 * ni));
    c->chk_elems = (size_t)JC * 3 * ni;
  }
  pair_fp64_kernel<<<dim3(gx, JC), 128, 0, c->st>>>(c->x, c->y, c->z, c->m, c->h, c->n, idx, ni, c->invL, n_cut_eff(c),
                                                    tpc, c->chk, is_r3(c) ? 1 : 0);
  CKLAUNCH("pair_fp64");
  chunk_sum_kernel<<<(ni + 255) / 256, 256, 0, c->st>>>(c->chk, ni, JC, out);
  CKLAUNCH("chunk_sum");
  return STEPS_OK;
}

struct SplitMix {
  uint64_t s;
  explicit SplitMix(uint64_t seed) : s(seed) {}
  uint64_t next() {
    uint64_t z = (s += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
  }
  double uniform() { return (double)(next() >> 11) * (1.0 / 9007199254740992.0); }  // [0, 1)
};

// ---------------------------------------------------------------------------
// Octree (Sect. 2.4): buffers, build, walk (kernels in octree.cuh).
// ---------------------------------------------------------------------------
#define CKT(call)                                                                              \
  do {                                                                                         \
    cudaError_t e_ = (call);                                                                   \
    if (e_ != cudaSuccess)                                                                     \
      return fail(e_ == cudaErrorMemoryAllocation ? STEPS_ENOMEM : STEPS_ECUDA, "%s: %s", #call, \
                  cudaGetErrorString(e_));                                                     \
  } while (0)

bool is_tree(const steps_cyl_ctx* c) { return c->p.force == STEPS_FORCE_OCTREE; }

int tree_alloc(steps_cyl_ctx* c) {
  auto& T = c->tr;
  if (T.ready) return STEPS_OK;
  // a failure part-way leaves ready false; the buffers already made are freed with the context
  // or replaced on the next attempt
  const size_t n = (size_t)c->n;
  const int ntiles = (c->n + kSortTile - 1) / kSortTile;
  {
    void* old[] = {T.key[0], T.key[1], T.val[0], T.val[1], T.hist, T.offs, T.u4, T.u4s, T.zt, T.sA, T.sB,
                   T.totals, T.inter};
    for (void* q : old) cudaFree(q);
    T.key[0] = T.key[1] = nullptr;
    T.val[0] = T.val[1] = nullptr;
    T.hist = T.offs = nullptr;
    T.u4 = T.u4s = T.sA = T.sB = nullptr;
    T.zt = nullptr;
    T.totals = nullptr;
    T.inter = nullptr;
    if (T.totals_h) cudaFreeHost(T.totals_h);
    T.totals_h = nullptr;
    for (cudaEvent_t* e : {&T.t0, &T.t1, &T.t2})
      if (*e) {
        cudaEventDestroy(*e);
        *e = nullptr;
      }
  }
  for (int k = 0; k < 2; ++k) {
    CKT(cudaMalloc(&T.key[k], sizeof(uint64_t) * n));
    CKT(cudaMalloc(&T.val[k], sizeof(int) * n));
  }
  CKT(cudaMalloc(&T.hist, sizeof(unsigned) * 256 * (size_t)ntiles));
  CKT(cudaMalloc(&T.offs, sizeof(unsigned) * 256 * (size_t)ntiles));
  CKT(cudaMalloc(&T.u4, sizeof(float4) * n));
  CKT(cudaMalloc(&T.u4s, sizeof(float4) * n));
  CKT(cudaMalloc(&T.zt, sizeof(double) * n));
  CKT(cudaMalloc(&T.sA, sizeof(float4) * n));
  CKT(cudaMalloc(&T.sB, sizeof(float4) * n));
  CKT(cudaMalloc(&T.totals, sizeof(int) * 2));
  CKT(cudaMallocHost(&T.totals_h, sizeof(int) * 2));
  CKT(cudaMalloc(&T.inter, sizeof(unsigned long long)));
  CKT(cudaEventCreate(&T.t0));
  CKT(cudaEventCreate(&T.t1));
  CKT(cudaEventCreate(&T.t2));
  T.ready = true;
  return STEPS_OK;
}

// Grow the node arrays to hold `need` nodes, keeping the first `keep`.
int tree_grow_nodes(steps_cyl_ctx* c, int need, int keep) {
  auto& T = c->tr;
  if (need <= T.node_cap) return STEPS_OK;
  const int cap = std::max(need, T.node_cap * 2);
  auto grow = [&](auto*& ptr, size_t elem) -> int {
    void* q = nullptr;
    CKT(cudaMalloc(&q, elem * (size_t)cap));
    if (ptr && keep > 0) CKT(cudaMemcpyAsync(q, ptr, elem * (size_t)keep, cudaMemcpyDeviceToDevice, c->st));
    CKT(cudaStreamSynchronize(c->st));
    cudaFree(ptr);
    ptr = static_cast<std::remove_reference_t<decltype(ptr)>>(q);
    return STEPS_OK;
  };
  int rc;
  if ((rc = grow(T.link, sizeof(int4))) || (rc = grow(T.geo, sizeof(float4))) || (rc = grow(T.hmf, sizeof(float))) ||
      (rc = grow(T.pre, sizeof(uint64_t))) || (rc = grow(T.mom, sizeof(double4_32a))) ||
      (rc = grow(T.hmx, sizeof(double))) || (rc = grow(T.nA, sizeof(float4))) || (rc = grow(T.nB, sizeof(float4))))
    return rc;
  T.node_cap = cap;
  return STEPS_OK;
}

int tree_grow_slots(steps_cyl_ctx* c, int need) {
  auto& T = c->tr;
  if (need <= T.slot_cap) return STEPS_OK;
  const int cap = std::max(need, 2 * T.slot_cap);
  int* ptrs[5] = {T.active[0], T.active[1], T.cnt, T.beg, T.pos};
  for (int* q : ptrs) cudaFree(q);
  T.active[0] = T.active[1] = T.cnt = T.beg = T.pos = nullptr;
  T.slot_cap = 0;  // set again only once every array exists
  // active lists hold node ids (<= cap / 8 per level), the others one entry per child slot
  CKT(cudaMalloc(&T.active[0], sizeof(int) * (size_t)cap));
  CKT(cudaMalloc(&T.active[1], sizeof(int) * (size_t)cap));
  CKT(cudaMalloc(&T.cnt, sizeof(int) * (size_t)cap));
  CKT(cudaMalloc(&T.beg, sizeof(int) * (size_t)cap));
  CKT(cudaMalloc(&T.pos, sizeof(int) * (size_t)cap));
  T.slot_cap = cap;
  return STEPS_OK;
}

TreeFrame tree_frame_of(const steps_cyl_ctx* c, double zeta, double phi) {
  TreeFrame F;
  const double S = 2.0 * std::max(c->p.L, 2.0 * c->p.R_sim);
  F.c = std::cos(phi);
  F.s = std::sin(phi);
  F.zeta = zeta;
  F.L = c->p.L;
  F.halfL = 0.5 * c->p.L;
  F.invS = 1.0 / S;
  return F;
}

// Rotation by angle about the unit axis (Rodrigues), each entry with the
// explicit fma/mul sequence written here, so that any reproduction of the frame
// gets the same bits.
void tree_rotation(const double ax[3], double angle, double R[9]) {
  const double cs = std::cos(angle), sn = std::sin(angle), t = 1.0 - cs;
  const double tx = t * ax[0], ty = t * ax[1], tz = t * ax[2];
  const double sx = sn * ax[0], sy = sn * ax[1], sz = sn * ax[2];
  R[0] = std::fma(tx, ax[0], cs);
  R[1] = std::fma(tx, ax[1], -sz);
  R[2] = std::fma(tx, ax[2], sy);
  R[3] = std::fma(ty, ax[0], sz);
  R[4] = std::fma(ty, ax[1], cs);
  R[5] = std::fma(ty, ax[2], -sx);
  R[6] = std::fma(tz, ax[0], -sy);
  R[7] = std::fma(tz, ax[1], sx);
  R[8] = std::fma(tz, ax[2], cs);
}

// Sort, build and moments of the tree in frame f.
int tree_build(steps_cyl_ctx* c, const TreeDraw& f) {
  Range range("steps_cyl.tree_build");
  auto& T = c->tr;
  int rc;
  if ((rc = tree_alloc(c))) return rc;
  const int n = c->n;
  const double zeta = is_r3(c) ? 0.0 : f.zeta;
  if (is_r3(c)) {
    TreeFrame3 F;
    for (int a = 0; a < 3; ++a) F.cen[a] = f.cen[a];
    tree_rotation(f.axis, f.angle, F.R);
    F.invS = 1.0 / (4.0 * c->p.R_sim);
    tree_frame_r3_kernel<<<grid_for(n, 256), 256, 0, c->st>>>(c->x, c->y, c->z, c->h, c->perm, n, F, T.u4, T.zt,
                                                              T.key[0], T.val[0], c->err);
  } else {
    const TreeFrame F = tree_frame_of(c, f.zeta, f.phi);
    tree_frame_kernel<<<grid_for(n, 256), 256, 0, c->st>>>(c->x, c->y, c->z, c->h, c->perm, n, F, T.u4, T.zt,
                                                           T.key[0], T.val[0], c->err);
  }
  CKLAUNCH("tree_frame");
  const int ntiles = (n + kSortTile - 1) / kSortTile;
  for (int pass = 0; pass < 8; ++pass) {  // 8 digits of 8 bits; the result returns to buffer 0
    const int a = pass & 1, b = a ^ 1;
    radix_hist_kernel<<<ntiles, kSortThreads, 0, c->st>>>(T.key[a], n, 8 * pass, ntiles, T.hist);
    scan_exclusive_kernel<<<1, 1024, 0, c->st>>>(T.hist, T.offs, 256 * ntiles, nullptr);
    radix_scatter_kernel<<<ntiles, kSortThreads, 0, c->st>>>(T.key[a], T.val[a], n, 8 * pass, ntiles, T.offs,
                                                             T.key[b], T.val[b]);
  }
  CKLAUNCH("tree_sort");
  const uint64_t* key = T.key[0];
  const int* sidx = T.val[0];
  tree_gather_kernel<<<grid_for(n, 256), 256, 0, c->st>>>(c->jA, c->jB, T.u4, sidx, n, T.sA, T.sB, T.u4s);
  CKLAUNCH("tree_gather");
  // root
  const int leaf = c->p.leaf_size;
  if ((rc = tree_grow_nodes(c, std::max(1024, 2 * n / std::max(leaf, 1) + 64), 0))) return rc;
  if ((rc = tree_grow_slots(c, std::max(1024, 8 * (n / (leaf + 1) + 8))))) return rc;
  {
    const int4 l0 = make_int4(-1, 0, 0, n);
    const float4 g0 = make_float4(0.5f, 0.5f, 0.5f, 1.0f);
    const uint64_t p0 = 0;
    const int a0 = 0;
    CKT(cudaMemcpyAsync(T.link, &l0, sizeof l0, cudaMemcpyHostToDevice, c->st));
    CKT(cudaMemcpyAsync(T.geo, &g0, sizeof g0, cudaMemcpyHostToDevice, c->st));
    CKT(cudaMemcpyAsync(T.pre, &p0, sizeof p0, cudaMemcpyHostToDevice, c->st));
    CKT(cudaMemcpyAsync(T.active[0], &a0, sizeof a0, cudaMemcpyHostToDevice, c->st));
  }
  std::vector<int> lstart = {0, 1};
  int nn = 1, n_active = n > leaf ? 1 : 0, cur = 0;
  for (int level = 0; n_active > 0 && level < kTreeDepth; ++level) {
    if ((rc = tree_grow_nodes(c, nn + 8 * n_active, nn))) return rc;
    // active nodes hold > leaf particles each, so 8 n_active <= 8 (n / (leaf + 1)), the size taken above
    if (8 * n_active > T.slot_cap) return fail(STEPS_ECUDA, "octree build: child slots exceed their bound");
    tree_children_kernel<<<(8 * n_active + 255) / 256, 256, 0, c->st>>>(T.active[cur], n_active, level, key, T.link,
                                                                       T.pre, T.cnt, T.beg);
    tree_link_kernel<<<1, 1024, 0, c->st>>>(T.active[cur], n_active, level, leaf, nn, T.cnt, T.beg, T.pos, T.link,
                                            T.geo, T.pre, T.active[cur ^ 1], T.totals);
    CKLAUNCH("tree_level");
    CKT(cudaMemcpyAsync(T.totals_h, T.totals, sizeof(int) * 2, cudaMemcpyDeviceToHost, c->st));
    CKT(cudaStreamSynchronize(c->st));
    nn += T.totals_h[0];
    lstart.push_back(nn);
    n_active = T.totals_h[1];
    cur ^= 1;
  }
  T.nodes = nn;
  T.depth = (int)lstart.size() - 2;
  for (int l = (int)lstart.size() - 2; l >= 0; --l) {
    const int a = lstart[l], b = lstart[l + 1];
    if (b <= a) continue;
    tree_moments_kernel<<<(b - a + 255) / 256, 256, 0, c->st>>>(a, b, T.link, sidx, c->x, c->y, T.zt, c->m, c->h,
                                                               T.u4, T.mom, T.hmx, T.hmf);
  }
  tree_pack_kernel<<<grid_for(nn, 256), 256, 0, c->st>>>(nn, T.mom, T.hmx, zeta, c->p.L, c->invL, is_r3(c) ? 0 : 1,
                                                         T.nA, T.nB);
  CKLAUNCH("tree_moments");
  return STEPS_OK;
}

// The walk: pair sums [3][n] (internal order) into out.
int tree_walk(steps_cyl_ctx* c, double* out) {
  Range range("steps_cyl.tree_walk");
  auto& T = c->tr;
  TreeCrit C;
  const double S = 2.0 * std::max(c->p.L, 2.0 * c->p.R_sim);
  C.Lu = is_r3(c) ? INFINITY : (float)(c->p.L / S);  // R^3: no period, the wrap never applies
  C.hLu = 0.5f * C.Lu;
  C.th2 = (float)(c->p.theta * c->p.theta);
  const int groups = (c->n + 31) / 32;
  const int blocks = (groups + kWalkWarps - 1) / kWalkWarps;
  CKT(cudaMemsetAsync(T.inter, 0, sizeof(unsigned long long), c->st));
  const bool kahan = c->p.precision == STEPS_FP32_KAHAN;
  if (is_r3(c) && kahan)
    tree_walk_kernel<true, true><<<blocks, kWalkWarps * 32, 0, c->st>>>(T.sA, T.sB, T.u4s, T.val[0], c->n, T.link,
                                                                        T.geo, T.hmf, T.nA, T.nB, C, c->tab,
                                                                        c->tab_const, out, T.inter, c->err);
  else if (is_r3(c))
    tree_walk_kernel<false, true><<<blocks, kWalkWarps * 32, 0, c->st>>>(T.sA, T.sB, T.u4s, T.val[0], c->n, T.link,
                                                                         T.geo, T.hmf, T.nA, T.nB, C, c->tab,
                                                                         c->tab_const, out, T.inter, c->err);
  else if (kahan)
    tree_walk_kernel<true><<<blocks, kWalkWarps * 32, 0, c->st>>>(T.sA, T.sB, T.u4s, T.val[0], c->n, T.link, T.geo,
                                                                  T.hmf, T.nA, T.nB, C, c->tab, c->tab_const, out,
                                                                  T.inter, c->err);
  else
    tree_walk_kernel<false><<<blocks, kWalkWarps * 32, 0, c->st>>>(T.sA, T.sB, T.u4s, T.val[0], c->n, T.link, T.geo,
                                                                   T.hmf, T.nA, T.nB, C, c->tab, c->tab_const, out,
                                                                   T.inter, c->err);
  CKLAUNCH("tree_walk");
  return STEPS_OK;
}

// A frame drawn from a generator: S1xR2, a shift uniform in [0, L) and an angle
// uniform in [0, 2 pi); R^3, a rotation axis uniform on the sphere, an angle
// uniform in [0, 2 pi) and a domain centre uniform in the ball of radius R_sim / 2.
TreeDraw tree_draw(const steps_cyl_ctx* c, SplitMix& r) {
  TreeDraw f{};
  if (!is_r3(c)) {
    f.zeta = r.uniform() * c->p.L;
    f.phi = 2.0 * M_PI * r.uniform();
    return f;
  }
  const double za = 2.0 * r.uniform() - 1.0, pa = 2.0 * M_PI * r.uniform(), sa = std::sqrt(std::max(0.0, 1.0 - za * za));
  f.axis[0] = sa * std::cos(pa);
  f.axis[1] = sa * std::sin(pa);
  f.axis[2] = za;
  f.angle = 2.0 * M_PI * r.uniform();
  const double rc = 0.5 * c->p.R_sim * std::cbrt(r.uniform());
  const double zc = 2.0 * r.uniform() - 1.0, pc = 2.0 * M_PI * r.uniform(), sc = std::sqrt(std::max(0.0, 1.0 - zc * zc));
  f.cen[0] = rc * sc * std::cos(pc);
  f.cen[1] = rc * sc * std::sin(pc);
  f.cen[2] = rc * zc;
  return f;
}

// The frame of the next evaluation: the fixed one, or drawn from the seed and
// the evaluation counter.
TreeDraw tree_next_frame(steps_cyl_ctx* c) {
  auto& T = c->tr;
  TreeDraw f;
  if (T.fixed) {
    f = T.fd;
  } else {
    SplitMix r(c->p.tree_seed * 0x9E3779B97F4A7C15ull + T.evals);
    f = tree_draw(c, r);
  }
  ++T.evals;
  return f;
}

// One octree pair evaluation into c->part ([3][n]), timed in phases.
int tree_forces(steps_cyl_ctx* c, double* out) {
  auto& T = c->tr;
  const TreeDraw f = tree_next_frame(c);
  int rc;
  if ((rc = tree_alloc(c))) return rc;
  CKT(cudaEventRecord(T.t0, c->st));
  if ((rc = tree_build(c, f))) return rc;
  CKT(cudaEventRecord(T.t1, c->st));
  if ((rc = tree_walk(c, out))) return rc;
  CKT(cudaEventRecord(T.t2, c->st));
  unsigned long long inter = 0;
  CKT(cudaMemcpyAsync(&inter, T.inter, sizeof inter, cudaMemcpyDeviceToHost, c->st));
  CKT(cudaStreamSynchronize(c->st));
  float b = 0.f, w = 0.f;
  CKT(cudaEventElapsedTime(&b, T.t0, T.t1));
  CKT(cudaEventElapsedTime(&w, T.t1, T.t2));
  T.build_ms = b;
  T.walk_ms = w;
  T.interactions = (double)inter;
  return STEPS_OK;
}

RadialCorr radial_corr(const steps_cyl_ctx* c) {
  RadialCorr r{nullptr, 0, 0.0, 0};
  if (is_tree(c) && c->tr.rad && c->tr.rad_nb > 0) {
    r.tab = c->tr.rad;
    r.nb = c->tr.rad_nb;
    r.rmax = c->tr.rad_rmax;
    r.sph = is_r3(c) ? 1 : 0;
  }
  return r;
}

// Scale of the fixed-point accumulators of the symmetric kernels, from a bound
// on any particle's pair sum |sum_j m_j v_ij| (positions in units of L): one
// image's softened force is at most 4 / hh^2 <= (L / h_min)^2 (the peak of the
// spline of eq. Force_spline_kernel with hh >= 2 h_min), the other images of
// the window add at most 2 sum_k 1 / (k - 1/2)^2 < 10, and the masses add up
// to M. With a factor 16 to spare, 2^S = 2^61 / (16 B) rounded down to a power
// of two. Below 2^40 (a softening so small that the unit 2^-S would not be far
// below FP32 rounding of typical sums) the row kernels are used instead.
int fix_scale(steps_cyl_ctx* c) {
  std::vector<double> hm(c->n), hh(c->n);
  CK(cudaMemcpyAsync(hm.data(), c->m, sizeof(double) * c->n, cudaMemcpyDeviceToHost, c->st));
  CK(cudaMemcpyAsync(hh.data(), c->h, sizeof(double) * c->n, cudaMemcpyDeviceToHost, c->st));
  CK(cudaStreamSynchronize(c->st));
  double M = 0.0, hmin = INFINITY, hmax = 0.0;
  for (int k = 0; k < c->n; ++k) {
    M += std::fabs(hm[k]);
    hmin = std::min(hmin, hh[k]);
    hmax = std::max(hmax, hh[k]);
  }
  c->h_max = hmax;
  const double q = c->p.L / hmin;
  const double B = M * (q * q + 10.0);
  const int S = (int)std::floor(57.0 - std::log2(B));
  c->fix_ok = std::isfinite(B) && B > 0 && S >= 40 && S <= 1000;
  c->fix_scale = c->fix_ok ? std::ldexp(1.0, S) : 0.0;
  c->fix_ready = true;
  return STEPS_OK;
}

#ifndef STEPS_SYMMETRIC
#define STEPS_SYMMETRIC 1  // evaluate each unordered pair once (build-time switch)
#endif

// The FP32 direct forms of an S1xR2 context take the symmetric kernels, unless
// its rows are shared with other ranks (a rank has no j side for rows it does
// not own).
bool use_sym(const steps_cyl_ctx* c) {
  return STEPS_SYMMETRIC && (!c->shard || c->shard_world == 1) && !is_r3(c) && c->fix_ok;
}

// The pair form of the next force evaluation: FP64, the selected modelled tail
// when it is accepted, else the plain image sum (for the infinite window, which
// has none, the correction table built at init).
enum class Form { FP64, SURROGATE, TABLE, PLAIN };
Form force_form(const steps_cyl_ctx* c) {
  if (c->p.precision == STEPS_FP64) return Form::FP64;
  if (c->p.tail == STEPS_TAIL_SURROGATE && c->surr_ok) return Form::SURROGATE;
  if ((c->p.tail == STEPS_TAIL_TABLE || is_inf(c)) && c->tab_ok) return Form::TABLE;
  return Form::PLAIN;
}

// Pairs the symmetric kernels evaluate over all units: the unordered pairs
// across blocks once, the ordered pairs inside each 128-row block both ways.
double sym_pairs(const steps_cyl_ctx* c) {
  double within = 0.0;
  for (int b = 0; b < c->NB; ++b) {
    const double nb = (double)(std::min(c->n, (b + 1) * kBI) - b * kBI);
    within += nb * (nb - 1.0);
  }
  const double all = (double)c->n * (double)(c->n - 1);
  return 0.5 * (all - within) + within;
}

// The symmetric kernel of the form over the units [Ua, Ua + U) into F.
// The symmetric table kernel in the context's table read (compiled per read, so
// that the filtered CIC path carries none of the other reads' arithmetic).
// The straight-run calls of the learned tail and of the residual tables: a
// finite window, near range n0 = 4, and every softening support within half a
// period (h_i + h_j < L / 2), so that only the centre image of a pair can be
// softened. (The infinite window keeps the tiered calls.)
bool straight_run(const steps_cyl_ctx* c) {
  return !is_inf(c) && c->p.n0 == 4 && 2.0 * c->h_max < 0.5 * c->p.L;
}

template <bool KAHAN, bool INF>
void launch_sym_table(steps_cyl_ctx* c, int C, int n, int nc, int NB, long long Ua, long long U, const FixAcc& F) {
  const TableTail& T = c->tab;
  const bool far4 = straight_run(c);
  switch (T.read) {
    case kReadTsc:
      if (far4)
        pair_sym_table_kernel<KAHAN, INF, kReadTsc, true><<<C, kBI, 0, c->st>>>(c->jA, c->jB, n, nc, NB, Ua, U, C, T,
                                                                               c->tab_const, F);
      else
        pair_sym_table_kernel<KAHAN, INF, kReadTsc><<<C, kBI, 0, c->st>>>(c->jA, c->jB, n, nc, NB, Ua, U, C, T,
                                                                           c->tab_const, F);
      break;
    case kReadCicExact:
      pair_sym_table_kernel<KAHAN, INF, kReadCicExact><<<C, kBI, 0, c->st>>>(c->jA, c->jB, n, nc, NB, Ua, U, C, T,
                                                                              c->tab_const, F);
      break;
    case kReadTscExact:
      pair_sym_table_kernel<KAHAN, INF, kReadTscExact><<<C, kBI, 0, c->st>>>(c->jA, c->jB, n, nc, NB, Ua, U, C, T,
                                                                              c->tab_const, F);
      break;
    default:
      if (far4)
        pair_sym_table_kernel<KAHAN, INF, kReadCic, true><<<C, kBI, 0, c->st>>>(c->jA, c->jB, n, nc, NB, Ua, U, C, T,
                                                                               c->tab_const, F);
      else
        pair_sym_table_kernel<KAHAN, INF, kReadCic><<<C, kBI, 0, c->st>>>(c->jA, c->jB, n, nc, NB, Ua, U, C, T,
                                                                           c->tab_const, F);
  }
}

template <bool FAR4>
void launch_sym_surr(steps_cyl_ctx* c, int C, int n, int nc, int NB, long long Ua, long long U, const FixAcc& F) {
  const bool kahan = c->p.precision == STEPS_FP32_KAHAN;
  const SurrLane* wl = c->surr_lanes;
  if (is_inf(c) && kahan)
    pair_sym_surr_kernel<true, true, FAR4><<<C, kBI, 0, c->st>>>(c->jA, c->jB, n, 0, NB, Ua, U, C, wl, c->surr, F);
  else if (is_inf(c))
    pair_sym_surr_kernel<false, true, FAR4><<<C, kBI, 0, c->st>>>(c->jA, c->jB, n, 0, NB, Ua, U, C, wl, c->surr, F);
  else if (kahan)
    pair_sym_surr_kernel<true, false, FAR4><<<C, kBI, 0, c->st>>>(c->jA, c->jB, n, nc, NB, Ua, U, C, wl, c->surr, F);
  else
    pair_sym_surr_kernel<false, false, FAR4><<<C, kBI, 0, c->st>>>(c->jA, c->jB, n, nc, NB, Ua, U, C, wl, c->surr, F);
}

int launch_sym(steps_cyl_ctx* c, Form form, long long Ua, long long U, const FixAcc& F) {
  const bool kahan = c->p.precision == STEPS_FP32_KAHAN;
  c->last_straight = (form == Form::SURROGATE || (form == Form::TABLE && (c->tab.read == kReadCic ||
                                                                          c->tab.read == kReadTsc))) &&
                     straight_run(c);
  const int nc = c->p.n_cut, n = c->n, NB = c->NB;
  auto ctas = [&](int full) {  // the CTA count of the whole triangle, scaled to a share of it
    return (int)std::max<long long>(1, std::min<long long>(U, (long long)full * U / std::max<long long>(c->Usym, 1)));
  };
  if (form == Form::SURROGATE) {
    const int C = ctas(c->SYSC);
    if (straight_run(c))
      launch_sym_surr<true>(c, C, n, nc, NB, Ua, U, F);
    else
      launch_sym_surr<false>(c, C, n, nc, NB, Ua, U, F);
    CKLAUNCH("pair_sym_surrogate");
  } else if (form == Form::TABLE) {
    const int C = ctas(c->SYTC);
    if (is_inf(c) && kahan)
      launch_sym_table<true, true>(c, C, n, 0, NB, Ua, U, F);
    else if (is_inf(c))
      launch_sym_table<false, true>(c, C, n, 0, NB, Ua, U, F);
    else if (kahan)
      launch_sym_table<true, false>(c, C, n, nc, NB, Ua, U, F);
    else
      launch_sym_table<false, false>(c, C, n, nc, NB, Ua, U, F);
    CKLAUNCH("pair_sym_table");
  } else {
    const int C = ctas(c->SYC);
    if (kahan)
      pair_sym_kernel<true><<<C, kBI, 0, c->st>>>(c->jA, c->jB, n, nc, NB, Ua, U, C, F);
    else
      pair_sym_kernel<false><<<C, kBI, 0, c->st>>>(c->jA, c->jB, n, nc, NB, Ua, U, C, F);
    CKLAUNCH("pair_sym");
  }
  return STEPS_OK;
}

// One force evaluation at the current packed positions. Stores g = a^3 (pair +
// background) in gx/gy/gz (internal order); kicks p by K when kick is set.
int eval_forces(steps_cyl_ctx* c, bool kick, double K) {
  Range range("steps_cyl.forces");
  const double pair_scale = -c->p.G * c->invL * c->invL;
  c->forces_stale = false;
  if (is_tree(c)) {  // the octree: its own build and walk, then the common finalize
    CK(cudaEventRecord(c->e0, c->st));
    int rc = tree_forces(c, c->part);
    if (rc) return rc;
    CK(cudaEventRecord(c->e1, c->st));
    c->timed = true;
    c->last_images = c->tr.interactions;
    c->last_pairs = c->tr.interactions;
    c->last_sym = false;
    finalize_kernel<<<(c->n + 255) / 256, 256, 0, c->st>>>(
        c->part, c->n, 0, c->U, c->C, pair_scale, bg_params(c), c->x, c->y, c->z, c->gx, c->gy, c->gz, K,
        kick ? c->px : nullptr, kick ? c->py : nullptr, kick ? c->pz : nullptr, 1.0, nullptr, nullptr, nullptr,
        c->err, radial_corr(c));
    CKLAUNCH("finalize");
    return STEPS_OK;
  }
  const Form form = force_form(c);
  if (form == Form::PLAIN && is_inf(c)) return fail(STEPS_ENOSURROGATE, "the infinite window has no correction table");
  if (!c->fix_ready) {
    int rc = fix_scale(c);
    if (rc) return rc;
  }
  if (form != Form::FP64 && use_sym(c)) {
    CK(cudaMemsetAsync(c->facc, 0, sizeof(unsigned long long) * 3 * (size_t)c->n, c->st));
    CK(cudaEventRecord(c->e0, c->st));
    int rc = launch_sym(c, form, 0, c->Usym, FixAcc{c->facc, c->n, c->fix_scale, c->err, 0, 0, 0, 0});
    if (rc) return rc;
    CK(cudaEventRecord(c->e1, c->st));
    c->timed = true;
    c->last_images = (double)c->n * (double)(c->n - 1) * images_per_pair(c);
    c->last_pairs = sym_pairs(c);
    c->last_sym = true;
    finalize_fix_kernel<<<(c->n + 255) / 256, 256, 0, c->st>>>(
        c->facc, c->n, 0, c->n, 1.0 / c->fix_scale, pair_scale, bg_params(c), c->x, c->y, c->z, c->gx, c->gy, c->gz,
        K, kick ? c->px : nullptr, kick ? c->py : nullptr, kick ? c->pz : nullptr, c->err);
    CKLAUNCH("finalize_fix");
    return STEPS_OK;
  }
  CK(cudaEventRecord(c->e0, c->st));
  if (form == Form::FP64) {
    int rc = launch_fp64(c, nullptr, c->n, c->part);  // never sharded
    if (rc) return rc;
  } else if (form == Form::SURROGATE) {
    const bool kahan = c->p.precision == STEPS_FP32_KAHAN;
    if (is_inf(c) && kahan)
      pair_fp32_surr_kernel<true, true><<<c->SC, kBI, 0, c->st>>>(c->jA, c->jB, c->n, 0, c->U, c->NT, c->SC,
                                                                  c->surr_lanes, c->surr, c->part, c->b0);
    else if (is_inf(c))
      pair_fp32_surr_kernel<false, true><<<c->SC, kBI, 0, c->st>>>(c->jA, c->jB, c->n, 0, c->U, c->NT, c->SC,
                                                                   c->surr_lanes, c->surr, c->part, c->b0);
    else if (kahan)
      pair_fp32_surr_kernel<true><<<c->SC, kBI, 0, c->st>>>(c->jA, c->jB, c->n, c->p.n_cut, c->U, c->NT, c->SC,
                                                             c->surr_lanes, c->surr, c->part, c->b0);
    else
      pair_fp32_surr_kernel<false><<<c->SC, kBI, 0, c->st>>>(c->jA, c->jB, c->n, c->p.n_cut, c->U, c->NT, c->SC,
                                                              c->surr_lanes, c->surr, c->part, c->b0);
    CKLAUNCH("pair_fp32_surrogate");
  } else if (form == Form::TABLE) {
    const bool kahan = c->p.precision == STEPS_FP32_KAHAN;
    if (is_inf(c) && kahan)
      pair_fp32_table_kernel<true, true><<<c->TC, kBI, 0, c->st>>>(c->jA, c->jB, c->n, 0, c->U, c->NT, c->TC, c->tab,
                                                                   c->tab_const, c->part, c->b0);
    else if (is_inf(c))
      pair_fp32_table_kernel<false, true><<<c->TC, kBI, 0, c->st>>>(c->jA, c->jB, c->n, 0, c->U, c->NT, c->TC, c->tab,
                                                                    c->tab_const, c->part, c->b0);
    else if (kahan)
      pair_fp32_table_kernel<true><<<c->TC, kBI, 0, c->st>>>(c->jA, c->jB, c->n, c->p.n_cut, c->U, c->NT, c->TC,
                                                              c->tab, c->tab_const, c->part, c->b0);
    else
      pair_fp32_table_kernel<false><<<c->TC, kBI, 0, c->st>>>(c->jA, c->jB, c->n, c->p.n_cut, c->U, c->NT, c->TC,
                                                               c->tab, c->tab_const, c->part, c->b0);
    CKLAUNCH("pair_fp32_table");
  } else if (is_r3(c)) {
    if (c->p.precision == STEPS_FP32_KAHAN)
      pair_r3_kernel<true><<<c->C, kBI, 0, c->st>>>(c->jA, c->jB, c->n, c->U, c->NT, c->C, c->part, c->b0);
    else
      pair_r3_kernel<false><<<c->C, kBI, 0, c->st>>>(c->jA, c->jB, c->n, c->U, c->NT, c->C, c->part, c->b0);
    CKLAUNCH("pair_fp32_r3");
  } else if (c->p.precision == STEPS_FP32_KAHAN) {
    pair_fp32_kernel<true><<<c->C, kBI, 0, c->st>>>(c->jA, c->jB, c->n, c->p.n_cut, c->U, c->NT, c->C, c->part,
                                                    c->b0);
    CKLAUNCH("pair_fp32_kahan");
  } else {
    pair_fp32_kernel<false><<<c->C, kBI, 0, c->st>>>(c->jA, c->jB, c->n, c->p.n_cut, c->U, c->NT, c->C, c->part,
                                                     c->b0);
    CKLAUNCH("pair_fp32_plain");
  }
  CK(cudaEventRecord(c->e1, c->st));
  c->timed = true;
  c->last_images = (double)(c->k1 - c->k0) * (double)(c->n - 1) * images_per_pair(c);
  c->last_pairs = (double)(c->k1 - c->k0) * (double)(c->n - 1);
  c->last_sym = false;
  const int NT = form == Form::FP64 ? 0 : c->NT;
  const int ctas = form == Form::SURROGATE ? c->SC : form == Form::TABLE ? c->TC : c->C;
  // rows [k0, k1): every row, or the rows this context owns when they are sharded
  finalize_kernel<<<(c->k1 - c->k0 + 255) / 256, 256, 0, c->st>>>(
      c->part, c->k1, NT, c->U, ctas, pair_scale, bg_params(c), c->x, c->y, c->z, c->gx, c->gy, c->gz, K,
      kick ? c->px : nullptr, kick ? c->py : nullptr, kick ? c->pz : nullptr, 1.0, nullptr, nullptr, nullptr, c->err,
      RadialCorr{nullptr, 0, 0.0, 0}, c->k0);
  CKLAUNCH("finalize");
  return STEPS_OK;
}

// Stage the caller's positions (any memory) into stage[0 .. 3n).
int stage_positions(steps_cyl_ctx* c, const double* x, const double* y, const double* z) {
  const size_t b = sizeof(double) * (size_t)c->n;
  double* s = c->stage;
  CK(cudaMemcpyAsync(s, x, b, cudaMemcpyDefault, c->st));
  CK(cudaMemcpyAsync(s + c->n, y, b, cudaMemcpyDefault, c->st));
  CK(cudaMemcpyAsync(s + 2 * (size_t)c->n, z, b, cudaMemcpyDefault, c->st));
  return STEPS_OK;
}

// Caller-order array (any memory) -> internal array, scaled.
int gather_in(steps_cyl_ctx* c, const double* src, double* dst, double scale) {
  // the last third of stage is free once the positions are gathered
  double* tmp = c->stage + 2 * (size_t)c->n;
  CK(cudaMemcpyAsync(tmp, src, sizeof(double) * c->n, cudaMemcpyDefault, c->st));
  gather_kernel<<<grid_for(c->n, 256), 256, 0, c->st>>>(tmp, c->perm, c->n, scale, dst);
  CKLAUNCH("gather");
  return STEPS_OK;
}

// Staged positions (caller order) and caller velocities -> internal state.
int install_state(steps_cyl_ctx* c, const double* vx, const double* vy, const double* vz) {
  double* s = c->stage;
  gather_kernel<<<grid_for(c->n, 256), 256, 0, c->st>>>(s, c->perm, c->n, 1.0, c->x);
  gather_kernel<<<grid_for(c->n, 256), 256, 0, c->st>>>(s + c->n, c->perm, c->n, 1.0, c->y);
  gather_kernel<<<grid_for(c->n, 256), 256, 0, c->st>>>(s + 2 * (size_t)c->n, c->perm, c->n, 1.0, c->z);
  CKLAUNCH("gather positions");
  int rc;
  const double a2 = c->a * c->a;  // canonical momentum p = a^2 dx/dt
  if ((rc = gather_in(c, vx, c->px, a2))) return rc;
  if ((rc = gather_in(c, vy, c->py, a2))) return rc;
  if ((rc = gather_in(c, vz, c->pz, a2))) return rc;
  return STEPS_OK;
}

int validate_state(steps_cyl_ctx* c) {
  CK(cudaMemsetAsync(c->err, 0, sizeof(int), c->st));
  validate_kernel<<<grid_for(c->n, 256), 256, 0, c->st>>>(c->x, c->y, c->z, c->px, c->py, c->pz, c->m, c->h, c->n,
                                                           is_r3(c) ? 0.0 : c->p.L, c->err);
  CKLAUNCH("validate");
  int bad = 0;
  int rc = read_and_clear_err(c, &bad);
  if (rc) return rc;
  if (bad & 1) return fail(STEPS_EINVAL, "non-finite position or velocity");
  if (bad & 2) return fail(STEPS_EINVAL, "masses must be finite and > 0");
  if (bad & 4) return fail(STEPS_EINVAL, "softenings must be finite and > 0");
  if (bad & 8) return fail(STEPS_EINVAL, "z must lie in [0, L)");
  return STEPS_OK;
}

int pack_positions(steps_cyl_ctx* c) {
  Range range("steps_cyl.pack");
  pack_kernel<<<grid_for(c->n, 256), 256, 0, c->st>>>(c->x, c->y, c->z, c->m, c->h, c->n, c->invL, c->jA, c->jB);
  CKLAUNCH("pack");
  return STEPS_OK;
}

// Re-order the device-resident particles along the Morton curve of their
// current (x, y): all per-particle arrays are permuted in place through a
// temporary, perm is composed, and the packed arrays are rebuilt.
int reorder(steps_cyl_ctx* c) {
  if (c->p.reorder_every < 0) return STEPS_OK;
  std::vector<double> hx(c->n), hy(c->n);
  CK(cudaMemcpyAsync(hx.data(), c->x, sizeof(double) * c->n, cudaMemcpyDeviceToHost, c->st));
  CK(cudaMemcpyAsync(hy.data(), c->y, sizeof(double) * c->n, cudaMemcpyDeviceToHost, c->st));
  CK(cudaStreamSynchronize(c->st));
  std::vector<int> o;
  morton_order(hx, hy, o);
  CK(cudaMemcpyAsync(c->ord, o.data(), sizeof(int) * c->n, cudaMemcpyHostToDevice, c->st));
  double* tmp = c->part;  // part_elems >= 3 n
  double* arrays[11] = {c->x, c->y, c->z, c->px, c->py, c->pz, c->m, c->h, c->gx, c->gy, c->gz};
  for (double* arr : arrays) {
    gather_kernel<<<grid_for(c->n, 256), 256, 0, c->st>>>(arr, c->ord, c->n, 1.0, tmp);
    CK(cudaMemcpyAsync(arr, tmp, sizeof(double) * c->n, cudaMemcpyDeviceToDevice, c->st));
  }
  CKLAUNCH("reorder");
  std::vector<int> np(c->n);
  for (int k = 0; k < c->n; ++k) np[k] = c->perm_h[o[k]];
  c->perm_h.swap(np);
  c->steps_since_order = 0;
  int rc;
  if ((rc = upload_perm(c))) return rc;
  return pack_positions(c);
}

void release(steps_cyl_ctx* c) {
  if (!c) return;
  int prev = 0;
  cudaGetDevice(&prev);
  cudaSetDevice(c->dev);
  if (c->st) cudaStreamSynchronize(c->st);
  cudaFree(c->state);
  cudaFree(c->jA);
  cudaFree(c->jB);
  cudaFree(c->part);
  cudaFree(c->stage);
  cudaFree(c->red);
  cudaFree(c->perm);
  cudaFree(c->iperm);
  cudaFree(c->ord);
  cudaFree(c->idx);
  cudaFree(c->sub);
  cudaFree(c->err);
  cudaFree(c->bgtab);
  cudaFree(c->surr_lanes);
  if (c->tab.tex) cudaDestroyTextureObject(c->tab.tex);
  if (c->tab_arr) cudaFreeArray(c->tab_arr);
  cudaFree(c->chk);
  cudaFree(c->shard_off);
  cudaFree(c->facc);
  {
    auto& T = c->tr;
    void* ptrs[] = {T.key[0], T.key[1], T.val[0], T.val[1], T.hist, T.offs, T.u4, T.u4s, T.zt, T.sA, T.sB,
                    T.link, T.geo, T.hmf, T.pre, T.mom, T.hmx, T.nA, T.nB, T.active[0], T.active[1], T.cnt,
                    T.beg, T.pos, T.totals, T.inter, T.rad};
    for (void* q : ptrs) cudaFree(q);
    if (T.totals_h) cudaFreeHost(T.totals_h);
    if (T.t0) cudaEventDestroy(T.t0);
    if (T.t1) cudaEventDestroy(T.t1);
    if (T.t2) cudaEventDestroy(T.t2);
  }
  if (c->e0) cudaEventDestroy(c->e0);
  if (c->e1) cudaEventDestroy(c->e1);
  cudaSetDevice(prev);
  delete c;
}

// RAII device guard: every entry point runs with the context's device current.
struct DeviceGuard {
  int prev = -1;
  explicit DeviceGuard(int dev) {
    cudaGetDevice(&prev);
    cudaSetDevice(dev);
  }
  ~DeviceGuard() {
    if (prev >= 0) cudaSetDevice(prev);
  }
};

// Internal-order arrays -> caller-order outputs (any memory), scaled. Device
// outputs receive the scatter directly; host outputs go through stage.
// Internal arrays -> caller order, scaled. A sharded context writes its own
// rows and zeros elsewhere, so a sum over the ranks assembles the whole.
int scatter_out(steps_cyl_ctx* c, const double* const src[3], double* const dst[3], double scale) {
  bool host = false;
  for (int q = 0; q < 3; ++q) {
    if (!dst[q]) continue;
    double* d = is_host_ptr(dst[q]) ? c->stage + (size_t)q * c->n : dst[q];
    if (c->shard)
      scatter_rows_kernel<<<grid_for(c->n, 256), 256, 0, c->st>>>(src[q], c->perm, c->n, scale, c->k0, c->k1, d);
    else
      scatter_kernel<<<grid_for(c->n, 256), 256, 0, c->st>>>(src[q], c->perm, c->n, scale, d);
    CKLAUNCH("scatter");
    if (d != dst[q]) {
      CK(cudaMemcpyAsync(dst[q], d, sizeof(double) * c->n, cudaMemcpyDeviceToHost, c->st));
      host = true;
    }
  }
  if (host) CK(cudaStreamSynchronize(c->st));
  return STEPS_OK;
}

// ---------------------------------------------------------------------------
// Learned far-image surrogate: host side (see surrogate_train.cuh and
// surrogate_pair.cuh for the definition and the kernels).
// ---------------------------------------------------------------------------

uint32_t half_bits(float v) {
  __half_raw r = __float2half_rn(v);
  return (uint32_t)r.x;
}
uint32_t pack_half2(float lo, float hi) { return half_bits(lo) | (half_bits(hi) << 16); }

// Per-lane mma fragments of a parameter vector (layout in include/steps_cyl.h).
void build_lanes(const float* P, SurrLane lanes[32]) {
  const float *W1 = P + kOW1, *b1 = P + kOB1, *W2 = P + kOW2, *b2 = P + kOB2, *W3 = P + kOW3;
  for (int L = 0; L < 32; ++L) {
    SurrLane& s = lanes[L];
    std::memset(&s, 0, sizeof s);
    const int g = L >> 2, t = L & 3;
    for (int nb = 0; nb < 4; ++nb) {
      const int o = 8 * nb + g;
      // rows 2t, 2t + 1 of the first layer's [8 x 32] B operand: inputs 0..2,
      // then the constant-1 input whose weight is the bias, then zeros
      const float w0 = t == 0 ? W1[o * 3] : (t == 1 ? W1[o * 3 + 2] : 0.f);
      const float w1 = t == 0 ? W1[o * 3 + 1] : (t == 1 ? b1[o] : 0.f);
      s.w1[nb] = pack_half2(w0, w1);
      // accumulator seeds: columns 2t, 2t + 1 of rows g and g + 8 of n-block nb
      for (int q = 0; q < 4; ++q) s.c2[4 * nb + q] = b2[8 * nb + 2 * t + (q & 1)];
      for (int kb = 0; kb < 2; ++kb) {
        const int k = 16 * kb + 2 * t;
        s.w2[(nb * 2 + kb) * 2] = pack_half2(W2[o * kH + k], W2[o * kH + k + 1]);
        s.w2[(nb * 2 + kb) * 2 + 1] = pack_half2(W2[o * kH + k + 8], W2[o * kH + k + 9]);
      }
    }
    // output column n = g carries output (n & 1); the even m-tile's product
    // fills columns 0..3 and the odd tile's columns 4..7, so that every lane
    // of a quad holds both outputs of its own pair
    uint32_t* w3 = g < 4 ? s.w3e : s.w3o;
    for (int kb = 0; kb < 2; ++kb) {
      const int k = 16 * kb + 2 * t, o = g & 1;
      w3[kb * 2] = pack_half2(W3[o * kH + k], W3[o * kH + k + 1]);
      w3[kb * 2 + 1] = pack_half2(W3[o * kH + k + 8], W3[o * kH + k + 9]);
    }
  }
}

// The output shift the kernels add: mu + sc b3, so that b3 enters the tail as
// E (sc (y + b3) + mu) with the network's last layer run without its bias.
void surr_shift(const float* P, float shift[2]) {
  shift[0] = (float)((double)P[kNW] + (double)P[kNW + 2] * (double)P[kOB3]);
  shift[1] = (float)((double)P[kNW + 1] + (double)P[kNW + 3] * (double)P[kOB3 + 1]);
}

int install_surrogate(steps_cyl_ctx* c, const float* P) {
  SurrLane lanes[32];
  build_lanes(P, lanes);
  if (!c->surr_lanes) CK(cudaMalloc(&c->surr_lanes, sizeof lanes));
  CK(cudaMemcpyAsync(c->surr_lanes, lanes, sizeof lanes, cudaMemcpyHostToDevice, c->st));
  CK(cudaStreamSynchronize(c->st));
  float shift[2];
  surr_shift(P, shift);
  c->surr.mu0 = shift[0];
  c->surr.mu1 = shift[1];
  c->surr.sc0 = P[kNW + 2];
  c->surr.sc1 = P[kNW + 3];
  c->surr.dR_max = P[kNW + 4];
  c->surr.inv_dR_max = 1.0f / P[kNW + 4];
  c->surr.n0 = c->p.n0;
  surr_const_finish(c->surr, c->p.n_cut);
  c->surr_params.assign(P, P + STEPS_SURR_NPARAM);
  return STEPS_OK;
}

int grow(steps_cyl_ctx* c, size_t elems) {
  if (elems <= c->chk_elems) return STEPS_OK;
  cudaFree(c->chk);
  c->chk = nullptr;
  c->chk_elems = 0;
  CK(cudaMalloc(&c->chk, sizeof(double) * elems));
  c->chk_elems = elems;
  return STEPS_OK;
}

// Total accelerations (times a^3) of a particle sample with the plain image sum
// and with a modelled tail (STEPS_TAIL_SURROGATE or STEPS_TAIL_TABLE); relative
// error statistics of the latter.
int run_check(steps_cyl_ctx* c, int model, int ncheck, uint64_t seed, double* med, double* p999,
              double* ms_plain, double* ms_surr) {
  // the reference: the plain image sum, or for the infinite window (which has
  // none) its correction table, exact to well below the FP32 arithmetic
  if (is_inf(c) && (model != STEPS_TAIL_SURROGATE || !c->tab_ok))
    return fail(STEPS_EINVAL, "the infinite window checks only a surrogate, against its correction table");
  // the sample is drawn from the rows this context evaluates (all, or its shard)
  const int nrows = c->k1 - c->k0;
  const int ni = std::max(1, std::min(ncheck, nrows));
  std::vector<int64_t> pick(ni);
  {
    std::vector<int> all(nrows);
    for (int k = 0; k < nrows; ++k) all[k] = c->k0 + k;
    SplitMix rng(seed);
    for (int q = 0; q < ni; ++q) {  // partial Fisher-Yates: distinct internal indices
      const int r = q + (int)(rng.next() % (uint64_t)(nrows - q));
      std::swap(all[q], all[r]);
      pick[q] = all[q];
    }
  }
  if (ni > c->idx_cap) {
    cudaFree(c->idx);
    cudaFree(c->sub);
    c->idx = nullptr;
    c->sub = nullptr;
    c->idx_cap = 0;
    CK(cudaMalloc(&c->idx, sizeof(int64_t) * ni));
    CK(cudaMalloc(&c->sub, sizeof(double) * ni * 3));
    c->idx_cap = ni;
  }
  CK(cudaMemcpyAsync(c->idx, pick.data(), sizeof(int64_t) * ni, cudaMemcpyHostToDevice, c->st));
  int sms = 0;
  CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c->dev));
  const int gx = (ni + kBI - 1) / kBI;
  const int want = std::max(1, std::min(c->NT, (sms * 8 + gx - 1) / gx));
  const int tpc = (c->NT + want - 1) / want;
  const int JC = (c->NT + tpc - 1) / tpc;
  int rc;
  if ((rc = grow(c, (size_t)JC * 3 * ni + 12 * (size_t)ni))) return rc;
  double* part = c->chk;
  double* sums = part + (size_t)JC * 3 * ni;
  double* tot = sums + 3 * (size_t)ni;  // [2][3][ni]
  const double pair_scale = -c->p.G * c->invL * c->invL;
  float ms[2] = {0.f, 0.f};
  for (int form = 0; form < 2; ++form) {
    CK(cudaEventRecord(c->e0, c->st));
    if (form == 0 && is_inf(c))
      pair_fp32_table_subset_kernel<true, true><<<dim3(gx, JC), kBI, 0, c->st>>>(c->jA, c->jB, c->n, 0, c->idx, ni,
                                                                                 tpc, c->tab, c->tab_const, part);
    else if (form == 0)
      pair_fp32_subset_kernel<true, false><<<dim3(gx, JC), kBI, 0, c->st>>>(c->jA, c->jB, c->n, c->p.n_cut, c->idx,
                                                                            ni, tpc, c->surr_lanes, c->surr, part);
    else if (is_inf(c))
      pair_fp32_subset_kernel<true, true, true><<<dim3(gx, JC), kBI, 0, c->st>>>(c->jA, c->jB, c->n, 0, c->idx, ni,
                                                                                 tpc, c->surr_lanes, c->surr, part);
    else if (model == STEPS_TAIL_SURROGATE)
      pair_fp32_subset_kernel<true, true><<<dim3(gx, JC), kBI, 0, c->st>>>(c->jA, c->jB, c->n, c->p.n_cut, c->idx,
                                                                           ni, tpc, c->surr_lanes, c->surr, part);
    else
      pair_fp32_table_subset_kernel<true><<<dim3(gx, JC), kBI, 0, c->st>>>(c->jA, c->jB, c->n, c->p.n_cut, c->idx,
                                                                           ni, tpc, c->tab, c->tab_const, part);
    CKLAUNCH("pair_fp32_subset");
    CK(cudaEventRecord(c->e1, c->st));
    CK(cudaEventSynchronize(c->e1));
    CK(cudaEventElapsedTime(&ms[form], c->e0, c->e1));
    chunk_sum_kernel<<<(ni + 255) / 256, 256, 0, c->st>>>(part, ni, JC, sums);
    double* o = tot + (size_t)form * 3 * ni;
    subset_finalize_kernel<<<(ni + 255) / 256, 256, 0, c->st>>>(sums, ni, c->idx, pair_scale, bg_params(c), c->x,
                                                                c->y, c->z, 1.0, o, o + ni, o + 2 * (size_t)ni,
                                                                c->err);
    CKLAUNCH("check_finalize");
  }
  std::vector<double> h(6 * (size_t)ni);
  CK(cudaMemcpyAsync(h.data(), tot, sizeof(double) * 6 * ni, cudaMemcpyDeviceToHost, c->st));
  CK(cudaStreamSynchronize(c->st));
  std::vector<double> rel(ni);
  for (int q = 0; q < ni; ++q) {
    double d2 = 0.0, r2 = 0.0;
    for (int a = 0; a < 3; ++a) {
      const double p = h[(size_t)a * ni + q], s = h[3 * (size_t)ni + (size_t)a * ni + q];
      d2 += (s - p) * (s - p);
      r2 += p * p;
    }
    rel[q] = r2 > 0 ? std::sqrt(d2 / r2) : std::sqrt(d2);
  }
  std::sort(rel.begin(), rel.end());
  auto quant = [&](double f) {
    const double pos = f * (ni - 1);
    const int lo = (int)std::floor(pos);
    const int hi = std::min(ni - 1, lo + 1);
    return rel[lo] + (pos - lo) * (rel[hi] - rel[lo]);
  };
  *med = quant(0.5);
  *p999 = quant(0.999);
  if (ms_plain) *ms_plain = ms[0];
  if (ms_surr) *ms_surr = ms[1];
  return STEPS_OK;
}

// A frame's arguments: S1xR2 zeta in [0, L), phi finite; R^3 a finite centre
// inside R_sim / 2 of the origin, a unit axis (to 1e-12) and a finite angle.
int check_frame(const steps_cyl_ctx* c, const TreeDraw& f) {
  if (!is_r3(c)) {
    if (!(f.zeta >= 0.0 && f.zeta < c->p.L) || !std::isfinite(f.phi))
      return fail(STEPS_EINVAL, "zeta must lie in [0, L) and phi be finite");
    return STEPS_OK;
  }
  const double r2 = f.cen[0] * f.cen[0] + f.cen[1] * f.cen[1] + f.cen[2] * f.cen[2];
  const double a2 = f.axis[0] * f.axis[0] + f.axis[1] * f.axis[1] + f.axis[2] * f.axis[2];
  if (!(r2 <= 0.25 * c->p.R_sim * c->p.R_sim) || !(std::fabs(a2 - 1.0) <= 1e-12) || !std::isfinite(f.angle))
    return fail(STEPS_EINVAL, "the frame needs a centre within R_sim / 2, a unit axis and a finite angle");
  return STEPS_OK;
}

// Install a radial correction table (nb bin means over [0, rmax]).
int set_radial(steps_cyl_ctx* c, const std::vector<double>& tab, double rmax) {
  auto& T = c->tr;
  cudaFree(T.rad);
  T.rad = nullptr;
  T.rad_nb = 0;
  CK(cudaMalloc(&T.rad, sizeof(double) * tab.size()));
  CK(cudaMemcpyAsync(T.rad, tab.data(), sizeof(double) * tab.size(), cudaMemcpyHostToDevice, c->st));
  CK(cudaStreamSynchronize(c->st));
  T.rad_nb = (int)tab.size();
  T.rad_rmax = rmax;
  T.rad_h = tab;
  return STEPS_OK;
}

// Radial calibration of the octree (Sect. 2.4): the mean radial component of
// (octree - direct) pair force over a particle sample and several frames, in
// bins of the radius (the cylindrical rho in S1xR2, the distance from the
// origin in R^3). The direct reference is the same pair form summed over all j:
// the infinite window's table form, or in R^3 the FP64 pair force.
int tree_calibrate(steps_cyl_ctx* c, int nf, int nb, int ns, const double* frames, const int64_t* sample,
                   std::vector<double>& table, double* rmax_out) {
  const int n = c->n;
  const int ni = std::min(ns, n);
  std::vector<int> inv(n);
  for (int k = 0; k < n; ++k) inv[c->perm_h[k]] = k;
  std::vector<int64_t> pick(ni);
  if (sample) {
    for (int q = 0; q < ni; ++q) {
      if (sample[q] < 0 || sample[q] >= n) return fail(STEPS_EINVAL, "sample index out of range");
      pick[q] = inv[sample[q]];
    }
  } else {
    std::vector<int> all(n);
    for (int k = 0; k < n; ++k) all[k] = k;
    SplitMix rng(0xca1b0000ull ^ c->p.tree_seed);
    for (int q = 0; q < ni; ++q) {
      const int r = q + (int)(rng.next() % (uint64_t)(n - q));
      std::swap(all[q], all[r]);
      pick[q] = all[q];
    }
  }
  const bool sph = is_r3(c);
  std::vector<double> hx(n), hy(n), hz(n, 0.0);
  CK(cudaMemcpyAsync(hx.data(), c->x, sizeof(double) * n, cudaMemcpyDeviceToHost, c->st));
  CK(cudaMemcpyAsync(hy.data(), c->y, sizeof(double) * n, cudaMemcpyDeviceToHost, c->st));
  if (sph) CK(cudaMemcpyAsync(hz.data(), c->z, sizeof(double) * n, cudaMemcpyDeviceToHost, c->st));
  CK(cudaStreamSynchronize(c->st));
  auto radius = [&](int k) { return sph ? std::sqrt(hx[k] * hx[k] + hy[k] * hy[k] + hz[k] * hz[k]) : std::hypot(hx[k], hy[k]); };
  double rmax = 0.0;
  for (int k = 0; k < n; ++k) rmax = std::max(rmax, radius(k));
  if (!(rmax > 0)) return fail(STEPS_EINVAL, "every particle sits at the centre");
  // direct pair sums of the sample
  if (ni > c->idx_cap) {
    cudaFree(c->idx);
    cudaFree(c->sub);
    c->idx = nullptr;
    c->sub = nullptr;
    c->idx_cap = 0;
    CK(cudaMalloc(&c->idx, sizeof(int64_t) * ni));
    CK(cudaMalloc(&c->sub, sizeof(double) * ni * 3));
    c->idx_cap = ni;
  }
  CK(cudaMemcpyAsync(c->idx, pick.data(), sizeof(int64_t) * ni, cudaMemcpyHostToDevice, c->st));
  int sms = 0;
  CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c->dev));
  const int gx = (ni + kBI - 1) / kBI;
  const int want = std::max(1, std::min(c->NT, (sms * 8 + gx - 1) / gx));
  const int tpc = (c->NT + want - 1) / want;
  const int JC = (c->NT + tpc - 1) / tpc;
  int rc;
  if ((rc = grow(c, (size_t)JC * 3 * ni + 3 * (size_t)ni))) return rc;
  double* sums = nullptr;  // [3][ni]
  CK(cudaMalloc(&sums, sizeof(double) * 3 * ni));
  if (sph) {
    rc = launch_fp64(c, c->idx, ni, sums);
  } else {
    double* part = c->chk;
    pair_fp32_table_subset_kernel<true, true><<<dim3(gx, JC), kBI, 0, c->st>>>(c->jA, c->jB, n, 0, c->idx, ni, tpc,
                                                                               c->tab, c->tab_const, part);
    chunk_sum_kernel<<<(ni + 255) / 256, 256, 0, c->st>>>(part, ni, JC, sums);
  }
  if (!rc && cudaGetLastError() != cudaSuccess) rc = fail(STEPS_ECUDA, "calibration direct launch failed");
  if (rc) {
    cudaFree(sums);
    return rc;
  }
  std::vector<double> D(3 * (size_t)ni), Tq(3 * (size_t)ni);
  const cudaError_t ce = cudaMemcpyAsync(D.data(), sums, sizeof(double) * 3 * ni, cudaMemcpyDeviceToHost, c->st);
  const cudaError_t cs = cudaStreamSynchronize(c->st);
  cudaFree(sums);
  if (ce != cudaSuccess || cs != cudaSuccess) return fail(STEPS_ECUDA, "calibration direct read-back failed");
  // octree pair sums of the sample in each frame (all particles walk: groups are fixed by the key order)
  int* dpick = nullptr;
  std::vector<int> pick32(pick.begin(), pick.end());
  CK(cudaMalloc(&dpick, sizeof(int) * ni));
  CK(cudaMemcpyAsync(dpick, pick32.data(), sizeof(int) * ni, cudaMemcpyHostToDevice, c->st));
  const double pair_scale = -c->p.G * c->invL * c->invL;
  std::vector<double> sum(nb, 0.0);
  std::vector<long long> cnt(nb, 0);
  SplitMix fr(0xf4a3e000ull ^ c->p.tree_seed);
  for (int f = 0; f < nf && rc == STEPS_OK; ++f) {
    TreeDraw fd{};
    if (!frames) {
      fd = tree_draw(c, fr);
    } else if (sph) {  // 7 doubles per frame: centre, unit axis, angle
      const double* q = frames + 7 * (size_t)f;
      for (int a = 0; a < 3; ++a) {
        fd.cen[a] = q[a];
        fd.axis[a] = q[3 + a];
      }
      fd.angle = q[6];
    } else {
      fd.zeta = frames[2 * f];
      fd.phi = frames[2 * f + 1];
    }
    if ((rc = check_frame(c, fd))) break;
    if ((rc = tree_build(c, fd)) || (rc = tree_walk(c, c->part))) break;
    for (int a = 0; a < 3; ++a)
      gather_kernel<<<grid_for(ni, 256), 256, 0, c->st>>>(c->part + (size_t)a * n, dpick, ni, 1.0,
                                                         c->sub + (size_t)a * ni);
    if (cudaMemcpyAsync(Tq.data(), c->sub, sizeof(double) * 3 * ni, cudaMemcpyDeviceToHost, c->st) != cudaSuccess ||
        cudaStreamSynchronize(c->st) != cudaSuccess) {
      rc = fail(STEPS_ECUDA, "calibration read-back failed");
      break;
    }
    for (int q = 0; q < ni; ++q) {
      const int i = (int)pick[q];
      const double rho = radius(i);
      if (!(rho > 0)) continue;
      const double ex = pair_scale * (Tq[q] - D[q]), ey = pair_scale * (Tq[(size_t)ni + q] - D[(size_t)ni + q]);
      const double ez = sph ? pair_scale * (Tq[2 * (size_t)ni + q] - D[2 * (size_t)ni + q]) : 0.0;
      const int k = std::min(nb - 1, (int)(rho / rmax * nb));
      sum[k] += (ex * hx[i] + ey * hy[i] + ez * hz[i]) / rho;
      ++cnt[k];
    }
  }
  cudaFree(dpick);
  if (rc) return rc;
  int e = 0;
  if ((rc = read_and_clear_err(c, &e))) return rc;
  if (e) return device_error(e);
  table.assign(nb, 0.0);
  for (int k = 0; k < nb; ++k) table[k] = cnt[k] ? sum[k] / (double)cnt[k] : 0.0;
  *rmax_out = rmax;
  return STEPS_OK;
}

// Install parameters, check them against the plain sum and keep them only
// when both error bounds hold.
int accept_surrogate(steps_cyl_ctx* c, const float* P, double bmed, double bp999, int ncheck, double* med,
                     double* p999, bool* ok) {
  int rc;
  if (is_r3(c)) return fail(STEPS_EINVAL, "the R^3 topology has no image tail to model");
  if (c->p.precision == STEPS_FP64) return fail(STEPS_EINVAL, "the surrogate needs an FP32 precision");
  bool finite = true;
  for (int k = 0; k < STEPS_SURR_NPARAM; ++k) finite = finite && std::isfinite(P[k]);
  if (!finite || !(P[kNW + 4] > 0.f) || !(P[kNW + 2] > 0.f) || !(P[kNW + 3] > 0.f)) {
    *med = *p999 = INFINITY;
    *ok = false;
    c->surr_ok = false;
    return STEPS_OK;
  }
  if ((rc = install_surrogate(c, P))) return rc;
  c->surr_ok = true;
  if ((rc = run_check(c, STEPS_TAIL_SURROGATE, ncheck, 0x5eed0000ull + (uint64_t)c->steps_since_check, med, p999,
                       nullptr, nullptr)))
    return rc;
  *ok = std::isfinite(*med) && std::isfinite(*p999) && *med <= bmed && *p999 <= bp999;
  c->surr_ok = *ok;
  c->surr_bound_med = bmed;
  c->surr_bound_p999 = bp999;
  if (!*ok) c->surr_params.clear();
  return STEPS_OK;
}

// Ewald construction of the infinite-window table: split parameter (1/L), the
// real-space images |k| <= nmax and the Fourier modes m <= mmax.
struct EwaldParams {
  double alpha;
  int nmax, mmax;
};

// Device buffers of one table build, freed on every exit path.
struct TableBuffers {
  cudaStream_t st;
  double2 *node = nullptr, *direct = nullptr;
  float2* f32 = nullptr;
  ~TableBuffers() {
    for (void* p : {(void*)node, (void*)direct, (void*)f32})
      if (p) cudaFreeAsync(p, st);
  }
};

// Correction-table tail: node residuals in FP64 on the GPU, stored as an FP32
// float2 array and read through a texture with bilinear filtering (the
// cloud-in-cell read). dR_max 0 = 2.2 x the largest particle radius. With ew
// (infinite window only) the nodes come from the Ewald summation, and the
// direct construction runs beside it for the report: ew_rep = largest node
// difference, largest node magnitude (both in envelope units), Ewald build ms,
// direct build ms.
int build_table(steps_cyl_ctx* c, int nx, int ny, double dR_max, double* ms, const EwaldParams* ew = nullptr,
                double* ew_rep = nullptr) {
  Range range("steps_cyl.build_table");
  if (is_r3(c)) return fail(STEPS_EINVAL, "the R^3 topology has no image tail to model");
  if (c->p.n0 < 0 || (c->p.n_cut > 0 && c->p.n0 >= c->p.n_cut))
    return fail(STEPS_EINVAL, "the context needs 0 <= n0 < n_cut");
  if (ew && c->p.n_cut != 0) return fail(STEPS_EINVAL, "the Ewald construction is for the infinite window (n_cut = 0)");
  if (dR_max == 0.0) {
    std::vector<double> hx(c->n), hy(c->n);
    CK(cudaMemcpyAsync(hx.data(), c->x, sizeof(double) * c->n, cudaMemcpyDeviceToHost, c->st));
    CK(cudaMemcpyAsync(hy.data(), c->y, sizeof(double) * c->n, cudaMemcpyDeviceToHost, c->st));
    CK(cudaStreamSynchronize(c->st));
    double rm = 0.0;
    for (int i = 0; i < c->n; ++i) rm = std::max(rm, std::hypot(hx[i], hy[i]));
    dR_max = std::max(2.2 * rm * c->invL, 1.0);
  }
  const int count = nx * ny;
  TableBuffers tb{c->st};
  CK(cudaMallocAsync(&tb.node, sizeof(double2) * count, c->st));
  CK(cudaMallocAsync(&tb.f32, sizeof(float2) * count, c->st));
  float t_direct = 0.f, t_ewald = 0.f;
  CK(cudaEventRecord(c->e0, c->st));
  tail_table_kernel<<<grid_for(count, 128), 128, 0, c->st>>>(nx, ny, dR_max, c->p.n_cut, c->p.n0, tb.node);
  CKLAUNCH("tail_table");
  CK(cudaEventRecord(c->e1, c->st));
  CK(cudaStreamSynchronize(c->st));
  CK(cudaEventElapsedTime(&t_direct, c->e0, c->e1));
  if (ew) {
    EwaldRule G;
    std::vector<double> gx, gw;
    gauss_legendre(8, gx, gw);
    std::copy(gx.begin(), gx.end(), G.x);
    std::copy(gw.begin(), gw.end(), G.w);
    tb.direct = tb.node;
    tb.node = nullptr;
    CK(cudaMallocAsync(&tb.node, sizeof(double2) * count, c->st));
    CK(cudaEventRecord(c->e0, c->st));
    tail_table_ewald_kernel<<<grid_for(count, 128), 128, 0, c->st>>>(nx, ny, dR_max, c->p.n0, ew->alpha, ew->nmax,
                                                                     ew->mmax, G, tb.node);
    CKLAUNCH("tail_table_ewald");
    CK(cudaEventRecord(c->e1, c->st));
    std::vector<double2> he(count), hd(count);
    CK(cudaMemcpyAsync(he.data(), tb.node, sizeof(double2) * count, cudaMemcpyDeviceToHost, c->st));
    CK(cudaMemcpyAsync(hd.data(), tb.direct, sizeof(double2) * count, cudaMemcpyDeviceToHost, c->st));
    CK(cudaStreamSynchronize(c->st));
    CK(cudaEventElapsedTime(&t_ewald, c->e0, c->e1));
    double dmax = 0.0, vmax = 0.0;
    for (int q = 0; q < count; ++q) {
      if (!std::isfinite(he[q].x) || !std::isfinite(he[q].y)) return fail(STEPS_ECUDA, "Ewald table node %d is not finite", q);
      dmax = std::max({dmax, std::fabs(he[q].x - hd[q].x), std::fabs(he[q].y - hd[q].y)});
      vmax = std::max({vmax, std::fabs(hd[q].x), std::fabs(hd[q].y)});
    }
    if (ew_rep) {
      ew_rep[0] = dmax;
      ew_rep[1] = vmax;
      ew_rep[2] = t_ewald;
      ew_rep[3] = t_direct;
    }
  }
  table_to_float_kernel<<<grid_for(count, 128), 128, 0, c->st>>>(tb.node, count, tb.f32);
  CKLAUNCH("table_to_float");
  c->tab_ok = false;
  if (c->tab.tex) CK(cudaDestroyTextureObject(c->tab.tex));
  c->tab.tex = 0;
  if (c->tab_arr) CK(cudaFreeArray(c->tab_arr));
  c->tab_arr = nullptr;
  const cudaChannelFormatDesc ch = cudaCreateChannelDesc<float2>();
  cudaError_t e = cudaMallocArray(&c->tab_arr, &ch, nx, ny);
  if (e == cudaSuccess)
    e = cudaMemcpy2DToArrayAsync(c->tab_arr, 0, 0, tb.f32, sizeof(float2) * nx, sizeof(float2) * nx, ny,
                                 cudaMemcpyDeviceToDevice, c->st);
  if (e != cudaSuccess) return fail(STEPS_ECUDA, "table array: %s", cudaGetErrorString(e));
  cudaResourceDesc res;
  std::memset(&res, 0, sizeof res);
  res.resType = cudaResourceTypeArray;
  res.res.array.array = c->tab_arr;
  cudaTextureDesc td;
  std::memset(&td, 0, sizeof td);
  td.addressMode[0] = td.addressMode[1] = cudaAddressModeClamp;
  td.filterMode = cudaFilterModeLinear;
  td.readMode = cudaReadModeElementType;
  td.normalizedCoords = 0;
  CK(cudaCreateTextureObject(&c->tab.tex, &res, &td, nullptr));
  c->tab.hx = 0.5f * (nx - 1);
  c->tab.hy = 0.5f * (ny - 1);
  // the nearest-image table (n0 = 0) is read with exact weights (see tail_table.cuh)
  c->tab.read = (c->tab_read_next == STEPS_TABLE_READ_TSC ? kReadTsc : kReadCic) + (c->p.n0 == 0 ? 2 : 0);
  c->tab_const = SurrConst{0.f, 0.f, 1.f, 1.f, (float)(1.0 / dR_max), (float)dR_max, c->p.n0, 0.f, 0.f, 0.f, 0.f};
  surr_const_finish(c->tab_const, c->p.n_cut);
  c->tab_nx = nx;
  c->tab_ny = ny;
  c->tab_dR_max = dR_max;
  CK(cudaStreamSynchronize(c->st));
  if (ms) *ms = ew ? t_ewald : t_direct;
  return STEPS_OK;
}

// Check the table form against the plain sum and keep it when both bounds hold.
int accept_table(steps_cyl_ctx* c, double bmed, double bp999, int ncheck, double* med, double* p999, bool* ok) {
  int rc;
  c->tab_ok = true;
  if ((rc = run_check(c, STEPS_TAIL_TABLE, ncheck, 0x7ab1e000ull + (uint64_t)c->steps_since_check, med, p999,
                      nullptr, nullptr)))
    return rc;
  *ok = std::isfinite(*med) && std::isfinite(*p999) && *med <= bmed && *p999 <= bp999;
  c->tab_ok = *ok;
  c->tab_bound_med = bmed;
  c->tab_bound_p999 = bp999;
  return STEPS_OK;
}

// Device buffers of one training run (freed on every exit path).
struct TrainBuffers {
  cudaStream_t st = nullptr;
  double *smp = nullptr, *tail = nullptr, *r = nullptr;
  float *u = nullptr, *t = nullptr, *w = nullptr, *m1 = nullptr, *m2 = nullptr, *gpart = nullptr, *lpart = nullptr,
        *loss = nullptr;
  int* order = nullptr;
  ~TrainBuffers() {
    for (void* p : {(void*)smp, (void*)tail, (void*)r, (void*)u, (void*)t, (void*)w, (void*)m1, (void*)m2,
                    (void*)gpart, (void*)lpart, (void*)loss, (void*)order})
      if (p) cudaFreeAsync(p, st);
    if (st) cudaStreamSynchronize(st);
  }
};

// Sum of a block-partial loss vector (device) read back to the host.
int read_loss(cudaStream_t st, const float* lpart, int nblocks, float* dev_out, float* host_out) {
  sum_floats_kernel<<<1, 32, 0, st>>>(lpart, nblocks, 1.0f, dev_out);
  CKLAUNCH("sum_floats");
  CK(cudaMemcpyAsync(host_out, dev_out, sizeof(float), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  return STEPS_OK;
}

int train_surrogate(steps_cyl_ctx* c, const steps_cyl_train_cfg* cfg, double* report) {
  Range range("steps_cyl.train_surrogate");
  const int64_t ns = cfg->n_samples;
  if (ns < 1024 || cfg->epochs < 1 || cfg->batch < 64 || cfg->batch % kTrainThreads != 0 || !(cfg->lr > 0) ||
      cfg->dR_max < 0 || cfg->reserved != 0 || cfg->check_particles < 1)
    return fail(STEPS_EINVAL, "bad training configuration");
  const int n_cut = c->p.n_cut, n0 = c->p.n0;
  if (is_r3(c)) return fail(STEPS_EINVAL, "the R^3 topology has no image tail to model");
  if (n0 < 1 || (n_cut > 0 && n0 >= n_cut)) return fail(STEPS_EINVAL, "the context needs 1 <= n0 < n_cut");
  const double A = n0 + 0.5;
  double dR_max = cfg->dR_max;
  if (dR_max == 0.0) {
    std::vector<double> hx(c->n), hy(c->n);
    CK(cudaMemcpyAsync(hx.data(), c->x, sizeof(double) * c->n, cudaMemcpyDeviceToHost, c->st));
    CK(cudaMemcpyAsync(hy.data(), c->y, sizeof(double) * c->n, cudaMemcpyDeviceToHost, c->st));
    CK(cudaStreamSynchronize(c->st));
    double rm = 0.0;
    for (int i = 0; i < c->n; ++i) rm = std::max(rm, std::hypot(hx[i], hy[i]));
    dR_max = std::max(2.2 * rm * c->invL, 1.0);
  }
  cudaEvent_t t0, t1;
  CK(cudaEventCreate(&t0));
  CK(cudaEventCreate(&t1));
  CK(cudaEventRecord(t0, c->st));
  // samples: dR with density ~ dR (pairs in a plane), |dz| and h uniform
  SplitMix rng(cfg->seed);
  std::vector<double> smp(3 * (size_t)ns);
  for (int64_t s = 0; s < ns; ++s) {
    smp[3 * s] = dR_max * std::sqrt(rng.uniform());
    smp[3 * s + 1] = 0.5 * rng.uniform();
    smp[3 * s + 2] = A * rng.uniform();
  }
  TrainBuffers B;
  B.st = c->st;
  const int maxblocks = cfg->batch / kTrainThreads;
  const int hold_blocks = 256;
  const int nb_alloc = std::max(maxblocks, hold_blocks);
  CK(cudaMallocAsync(&B.smp, sizeof(double) * 3 * ns, c->st));
  CK(cudaMallocAsync(&B.tail, sizeof(double) * 2 * ns, c->st));
  CK(cudaMallocAsync(&B.r, sizeof(double) * 2 * ns, c->st));
  CK(cudaMallocAsync(&B.u, sizeof(float) * 3 * ns, c->st));
  CK(cudaMallocAsync(&B.t, sizeof(float) * 2 * ns, c->st));
  CK(cudaMallocAsync(&B.order, sizeof(int) * ns, c->st));
  CK(cudaMallocAsync(&B.w, sizeof(float) * kNW, c->st));
  CK(cudaMallocAsync(&B.m1, sizeof(float) * kNW, c->st));
  CK(cudaMallocAsync(&B.m2, sizeof(float) * kNW, c->st));
  CK(cudaMallocAsync(&B.gpart, sizeof(float) * kNW * nb_alloc, c->st));
  CK(cudaMallocAsync(&B.lpart, sizeof(float) * nb_alloc, c->st));
  CK(cudaMallocAsync(&B.loss, sizeof(float), c->st));
  CK(cudaMemcpyAsync(B.smp, smp.data(), sizeof(double) * 3 * ns, cudaMemcpyHostToDevice, c->st));
  // exact FP64 targets, residual over the base, in envelope units
  tail_sums_fp64_kernel<<<grid_for((int)std::min<int64_t>(ns, 1 << 30), 128), 128, 0, c->st>>>(B.smp, ns, n_cut, n0,
                                                                                             B.tail);
  surrogate_dataset_kernel<<<grid_for((int)std::min<int64_t>(ns, 1 << 30), 256), 256, 0, c->st>>>(
      B.smp, B.tail, ns, n_cut, n0, dR_max, B.u, B.r);
  CKLAUNCH("dataset");
  const int64_t nhold = ns / 16, ntrain = ns - nhold;
  std::vector<double> r(2 * (size_t)ns);
  CK(cudaMemcpyAsync(r.data(), B.r, sizeof(double) * 2 * ns, cudaMemcpyDeviceToHost, c->st));
  CK(cudaStreamSynchronize(c->st));
  double mu[2] = {0, 0}, sc[2] = {0, 0};
  for (int o = 0; o < 2; ++o) {
    double s = 0.0;
    for (int64_t k = 0; k < ntrain; ++k) s += r[2 * k + o];
    mu[o] = s / ntrain;
    double v = 0.0;
    for (int64_t k = 0; k < ntrain; ++k) v += (r[2 * k + o] - mu[o]) * (r[2 * k + o] - mu[o]);
    sc[o] = std::sqrt(v / ntrain);
    if (!(sc[o] > 0)) sc[o] = 1.0;
  }
  std::vector<float> tn(2 * (size_t)ns);
  for (int64_t k = 0; k < ns; ++k)
    for (int o = 0; o < 2; ++o) tn[2 * k + o] = (float)((r[2 * k + o] - mu[o]) / sc[o]);
  CK(cudaMemcpyAsync(B.t, tn.data(), sizeof(float) * 2 * ns, cudaMemcpyHostToDevice, c->st));
  // initial weights: uniform in +-1/sqrt(fan_in)
  std::vector<float> w(kNW);
  auto fill = [&](int off, int cnt, int fan_in) {
    const double b = 1.0 / std::sqrt((double)fan_in);
    for (int k = 0; k < cnt; ++k) w[off + k] = (float)((2.0 * rng.uniform() - 1.0) * b);
  };
  fill(kOW1, kH * 3, 3);
  fill(kOB1, kH, 3);
  fill(kOW2, kH * kH, kH);
  fill(kOB2, kH, kH);
  fill(kOW3, 2 * kH, kH);
  fill(kOB3, 2, kH);
  CK(cudaMemcpyAsync(B.w, w.data(), sizeof(float) * kNW, cudaMemcpyHostToDevice, c->st));
  CK(cudaMemsetAsync(B.m1, 0, sizeof(float) * kNW, c->st));
  CK(cudaMemsetAsync(B.m2, 0, sizeof(float) * kNW, c->st));
  const float beta1 = 0.9f, beta2 = 0.999f, eps = 1e-8f;
  std::vector<int> order(ntrain);
  int64_t step = 0;
  float last_loss = 0.f;
  int64_t last_count = 1;
  for (int ep = 0; ep < cfg->epochs; ++ep) {
    for (int64_t k = 0; k < ntrain; ++k) order[k] = (int)k;
    for (int64_t k = ntrain - 1; k > 0; --k) std::swap(order[k], order[rng.next() % (uint64_t)(k + 1)]);
    CK(cudaMemcpyAsync(B.order, order.data(), sizeof(int) * ntrain, cudaMemcpyHostToDevice, c->st));
    const float lr = (float)(cfg->lr * 0.5 * (1.0 + std::cos(M_PI * ep / cfg->epochs)));
    for (int64_t first = 0; first < ntrain; first += cfg->batch) {
      const int64_t count = std::min<int64_t>(cfg->batch, ntrain - first);
      const int nblk = (int)((count + kTrainThreads - 1) / kTrainThreads);
      mlp_fwd_bwd_kernel<<<nblk, kTrainThreads, 0, c->st>>>(B.w, B.u, B.t, B.order, first, count, B.gpart, B.lpart);
      ++step;
      const float cb1 = (float)(1.0 - std::pow((double)beta1, (double)step));
      const float cb2 = (float)(1.0 - std::pow((double)beta2, (double)step));
      mlp_reduce_adam_kernel<<<(kNW + 127) / 128, 128, 0, c->st>>>(B.gpart, nblk, 1.0f / (float)count, B.w, B.m1,
                                                                   B.m2, lr, beta1, beta2, eps, cb1, cb2, 1, nullptr);
      last_count = count;
    }
    CKLAUNCH("train epoch");
  }
  {
    int rc = read_loss(c->st, B.lpart, (int)((last_count + kTrainThreads - 1) / kTrainThreads), B.loss, &last_loss);
    if (rc) return rc;
  }
  // held-out loss (forward and backward over the held-out tail, no update)
  double hold_sum = 0.0;
  for (int64_t first = ntrain; first < ns; first += (int64_t)hold_blocks * kTrainThreads) {
    const int64_t count = std::min<int64_t>((int64_t)hold_blocks * kTrainThreads, ns - first);
    const int nblk = (int)((count + kTrainThreads - 1) / kTrainThreads);
    mlp_fwd_bwd_kernel<<<nblk, kTrainThreads, 0, c->st>>>(B.w, B.u, B.t, nullptr, first, count, B.gpart, B.lpart);
    CKLAUNCH("held-out");
    float l = 0.f;
    int rc = read_loss(c->st, B.lpart, nblk, B.loss, &l);
    if (rc) return rc;
    hold_sum += l;
  }
  CK(cudaEventRecord(t1, c->st));
  CK(cudaMemcpyAsync(w.data(), B.w, sizeof(float) * kNW, cudaMemcpyDeviceToHost, c->st));
  CK(cudaStreamSynchronize(c->st));
  float train_ms = 0.f;
  CK(cudaEventElapsedTime(&train_ms, t0, t1));
  cudaEventDestroy(t0);
  cudaEventDestroy(t1);
  std::vector<float> P(STEPS_SURR_NPARAM);
  std::copy(w.begin(), w.end(), P.begin());
  P[kNW] = (float)mu[0];
  P[kNW + 1] = (float)mu[1];
  P[kNW + 2] = (float)sc[0];
  P[kNW + 3] = (float)sc[1];
  P[kNW + 4] = (float)dR_max;
  double med = 0, p999 = 0;
  bool ok = false;
  int rc = accept_surrogate(c, P.data(), cfg->err_median, cfg->err_p999, cfg->check_particles, &med, &p999, &ok);
  if (rc) return rc;
  if (report) {
    report[0] = last_loss / (double)last_count;
    report[1] = std::sqrt(2.0 * hold_sum / (double)std::max<int64_t>(nhold, 1) / 2.0);
    report[2] = med;
    report[3] = p999;
    report[4] = ok ? 1.0 : 0.0;
    report[5] = train_ms;
    report[6] = mu[0];
    report[7] = sc[0];
  }
  if (!ok) return fail(STEPS_ESURROGATE_REJECTED, "surrogate rejected: median %.3g, p99.9 %.3g", med, p999);
  return STEPS_OK;
}

// Device buffers and the work split of a context whose n, device and stream
// are set (init and resume).
// The pair kernels evaluate the i-blocks [b0, b0 + nbo): their stream-K units
// and CTA counts for that range.
void set_rows(steps_cyl_ctx* c, int b0, int nbo) {
  c->b0 = b0;
  c->nbo = nbo;
  c->k0 = b0 * kBI;
  c->k1 = std::min(c->n, (b0 + nbo) * kBI);
  c->U = (long long)nbo * c->NT;
  c->C = (int)std::min<long long>(c->U, c->Ccap);
  c->SC = (int)std::min<long long>(c->U, c->SCcap);
  c->TC = (int)std::min<long long>(c->U, c->TCcap);
}

int allocate_context(steps_cyl_ctx* c) {
#define CKA(call)                                                                            \
  do {                                                                                       \
    cudaError_t e_ = (call);                                                                 \
    if (e_ != cudaSuccess)                                                                   \
      return fail(e_ == cudaErrorMemoryAllocation ? STEPS_ENOMEM : STEPS_ECUDA, "%s: %s", #call, \
                  cudaGetErrorString(e_));                                                   \
  } while (0)
  const size_t nb = (size_t)c->n;
  CKA(cudaEventCreate(&c->e0));
  CKA(cudaEventCreate(&c->e1));
  CKA(cudaMalloc(&c->state, sizeof(double) * nb * 11));
  double* s = c->state;
  c->x = s; c->y = s + nb; c->z = s + 2 * nb; c->px = s + 3 * nb; c->py = s + 4 * nb; c->pz = s + 5 * nb;
  c->m = s + 6 * nb; c->h = s + 7 * nb; c->gx = s + 8 * nb; c->gy = s + 9 * nb; c->gz = s + 10 * nb;
  CKA(cudaMalloc(&c->jA, sizeof(float4) * nb));
  CKA(cudaMalloc(&c->jB, sizeof(float4) * nb));
  CKA(cudaMalloc(&c->stage, sizeof(double) * nb * 3));
  CKA(cudaMalloc(&c->red, sizeof(double) * (kRedBlocks * 6 + 8)));
  CKA(cudaMalloc(&c->perm, sizeof(int) * nb));
  CKA(cudaMalloc(&c->iperm, sizeof(int) * nb));
  CKA(cudaMalloc(&c->ord, sizeof(int) * nb));
  CKA(cudaMalloc(&c->err, sizeof(int)));
  CKA(cudaMemsetAsync(c->err, 0, sizeof(int), c->st));

  // stream-K split of the FP32 pair kernel: C CTAs share U units
  int sms = 0, occ = 0;
  CKA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c->dev));
  CKA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, pair_fp32_kernel<true>, kBI, 0));
  c->NB = (c->n + kBI - 1) / kBI;
  c->NT = (c->n + kBJ - 1) / kBJ;
  c->U = (long long)c->NB * c->NT;
  c->Ccap = sms * std::max(occ, 1) * STEPS_CTA_MULT;
  int socc = 0;
  CKA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&socc, pair_fp32_surr_kernel<true>, kBI, 0));
  c->SCcap = sms * std::max(socc, 1) * STEPS_CTA_MULT;
  int tocc = 0;
  CKA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&tocc, pair_fp32_table_kernel<true>, kBI, 0));
  c->TCcap = sms * std::max(tocc, 1) * STEPS_CTA_MULT;
  set_rows(c, 0, c->NB);
  // the symmetric kernels share the upper triangle of the block grid
  c->Usym = (long long)c->NB * (c->NB + 1) / 2;
  int yocc = 0, ysocc = 0, ytocc = 0;
  CKA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&yocc, pair_sym_kernel<true>, kBI, 0));
  CKA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&ysocc, pair_sym_surr_kernel<true, false>, kBI, 0));
  CKA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&ytocc, pair_sym_table_kernel<true, false, kReadCic>, kBI, 0));
  c->SYC = (int)std::min<long long>(c->Usym, (long long)sms * std::max(yocc, 1) * STEPS_CTA_MULT);
  c->SYSC = (int)std::min<long long>(c->Usym, (long long)sms * std::max(ysocc, 1) * STEPS_CTA_MULT);
  c->SYTC = (int)std::min<long long>(c->Usym, (long long)sms * std::max(ytocc, 1) * STEPS_CTA_MULT);
  CKA(cudaMalloc(&c->facc, sizeof(unsigned long long) * nb * 3));
  c->part_elems = std::max((size_t)(c->NB + std::max({c->C, c->SC, c->TC})) * 3 * kBI, nb * 3);
  CKA(cudaMalloc(&c->part, sizeof(double) * c->part_elems));

#undef CKA
  return STEPS_OK;
}

}  // namespace

// ===========================================================================
// C ABI
// ===========================================================================
extern "C" {

int steps_cyl_params_default(steps_cyl_params* p) {
  if (!p) return fail(STEPS_EINVAL, "params is NULL");
  std::memset(p, 0, sizeof *p);
  p->G = 1.0;
  p->L = 1.0;
  p->R_sim = 0.5 * std::tan(0.45 * M_PI);
  p->rho_bar = 0.0;
  p->n_cut = 16;
  p->n0 = 4;
  p->precision = STEPS_FP32_KAHAN;
  p->tail = STEPS_TAIL_FULL;
  p->background = STEPS_BG_FINITE;
  p->comoving = 0;
  p->H0 = 1.0;
  p->Omega_m = 0.3;
  p->Omega_r = 0.0;
  p->Omega_L = 0.7;
  p->w0 = -1.0;
  p->wa = 0.0;
  p->a_start = 1.0;
  p->t_start = 0.0;
  p->device = 0;
  p->reorder_every = 32;
  p->check_every = 50;
  p->check_particles = 1024;
  p->stream = nullptr;
  p->force = STEPS_FORCE_DIRECT;
  p->leaf_size = 16;
  p->theta = 0.5;
  p->tree_seed = 1;
  return STEPS_OK;
}

int steps_cyl_init(steps_cyl_ctx** out, const steps_cyl_params* p, int64_t n, const double* x, const double* y,
                   const double* z, const double* vx, const double* vy, const double* vz, const double* m,
                   const double* h) {
  g_last_error.clear();
  if (!out) return fail(STEPS_EINVAL, "out is NULL");
  *out = nullptr;
  int rc = check_params(p);
  if (rc) return rc;
  if (n < 2 || n > 0x7fffffffLL - kBI) return fail(STEPS_EINVAL, "n must be in [2, 2^31 - 129)");
  if (!x || !y || !z || !vx || !vy || !vz || !m || !h) return fail(STEPS_EINVAL, "NULL input array");
  if (p->tail == STEPS_TAIL_SURROGATE) return fail(STEPS_ENOSURROGATE, "no surrogate network is loaded");
  if (p->tail == STEPS_TAIL_TABLE && p->n_cut > 0) return fail(STEPS_ENOSURROGATE, "no correction table is built");
  int ndev = 0;
  CK(cudaGetDeviceCount(&ndev));
  if (p->device < 0 || p->device >= ndev) return fail(STEPS_EINVAL, "device %d out of range", p->device);
  DeviceGuard guard(p->device);

  steps_cyl_ctx* c = new steps_cyl_ctx();
  c->p = *p;
  c->n = (int)n;
  c->dev = p->device;
  c->st = (cudaStream_t)p->stream;
  c->cosmo = Cosmology{p->H0, p->Omega_m, p->Omega_r, p->Omega_L, p->w0, p->wa, p->comoving != 0};
  c->a = p->comoving ? p->a_start : 1.0;
  c->t = p->t_start;
  c->invL = 1.0 / p->L;
  auto bail = [&](int code) {
    release(c);
    return code;
  };
#define CKI(call)                                                                            \
  do {                                                                                       \
    cudaError_t e_ = (call);                                                                 \
    if (e_ != cudaSuccess) {                                                                 \
      int code_ = (e_ == cudaErrorMemoryAllocation) ? STEPS_ENOMEM : STEPS_ECUDA;            \
      fail(code_, "%s: %s", #call, cudaGetErrorString(e_));                                  \
      return bail(code_);                                                                    \
    }                                                                                        \
  } while (0)
  const size_t nb = (size_t)n;
  if ((rc = allocate_context(c))) return bail(rc);

  // caller order -> internal (Morton) order
  if ((rc = stage_positions(c, x, y, z))) return bail(rc);
  if ((rc = order_from_stage(c, c->stage, c->stage + nb, false))) return bail(rc);
  if ((rc = install_state(c, vx, vy, vz))) return bail(rc);
  if ((rc = gather_in(c, m, c->m, 1.0))) return bail(rc);
  if ((rc = gather_in(c, h, c->h, 1.0))) return bail(rc);
  if ((rc = validate_state(c))) return bail(rc);

  // comoving mean density of the background term
  if (p->rho_bar > 0) {
    c->rho0 = p->rho_bar;
  } else {
    std::vector<double> hm(nb);
    CKI(cudaMemcpyAsync(hm.data(), c->m, sizeof(double) * nb, cudaMemcpyDeviceToHost, c->st));
    CKI(cudaStreamSynchronize(c->st));
    double tot = 0.0, comp = 0.0;
    for (double v : hm) {  // compensated sum
      const double yv = v - comp, tv = tot + yv;
      comp = (tv - tot) - yv;
      tot = tv;
    }
    c->rho0 = p->topology == STEPS_TOPO_R3 ? tot / (4.0 / 3.0 * M_PI * p->R_sim * p->R_sim * p->R_sim)
                                           : tot / (M_PI * p->R_sim * p->R_sim * p->L);
  }
  if ((rc = build_background(c))) return bail(rc);
  if ((rc = pack_positions(c))) return bail(rc);
  if (p->n_cut == 0) {  // infinite window: the table is the definition of the tail, built here
    if ((rc = build_table(c, 257, 33, 0.0, nullptr))) return bail(rc);
    c->tab_ok = true;
  }
  if ((rc = eval_forces(c, false, 0.0))) return bail(rc);
  int e = 0;
  if ((rc = read_and_clear_err(c, &e))) return bail(rc);
  if (e) return bail(device_error(e));
#undef CKI
  *out = c;
  return STEPS_OK;
}

int steps_cyl_forces(steps_cyl_ctx* c, double* ax, double* ay, double* az) {
  g_last_error.clear();
  if (!c) return fail(STEPS_EINVAL, "ctx is NULL");
  if (!ax || !ay || !az) return fail(STEPS_EINVAL, "NULL output");
  if (c->drifted) return fail(STEPS_EINVAL, "a sharded step is half done: steps_cyl_shard_kick must come first");
  DeviceGuard guard(c->dev);
  int rc;
  if ((rc = eval_forces(c, false, 0.0))) return rc;
  const double* src[3] = {c->gx, c->gy, c->gz};
  double* dst[3] = {ax, ay, az};
  if ((rc = scatter_out(c, src, dst, 1.0 / (c->a * c->a * c->a)))) return rc;
  if (is_host_ptr(ax) || is_host_ptr(ay) || is_host_ptr(az)) {
    int e = 0;
    if ((rc = read_and_clear_err(c, &e))) return rc;
    if (e) return device_error(e);
  }
  return STEPS_OK;
}

int steps_cyl_forces_subset(steps_cyl_ctx* c, int64_t ni, const int64_t* idx, double* ax, double* ay, double* az) {
  g_last_error.clear();
  if (!c) return fail(STEPS_EINVAL, "ctx is NULL");
  if (c->shard) return refuse_sharded(c, "steps_cyl_forces_subset");
  if (ni < 0 || ni > c->n) return fail(STEPS_EINVAL, "ni must be in [0, n]");
  if (ni == 0) return STEPS_OK;
  if (!idx || !ax || !ay || !az) return fail(STEPS_EINVAL, "NULL argument");
  DeviceGuard guard(c->dev);
  if (ni > c->idx_cap) {
    cudaFree(c->idx);
    cudaFree(c->sub);
    c->idx = nullptr;
    c->sub = nullptr;
    c->idx_cap = 0;
    CK(cudaMalloc(&c->idx, sizeof(int64_t) * ni));
    CK(cudaMalloc(&c->sub, sizeof(double) * ni * 3));
    c->idx_cap = (int)ni;
  }
  CK(cudaMemcpyAsync(c->idx, idx, sizeof(int64_t) * ni, cudaMemcpyDefault, c->st));
  CK(cudaMemsetAsync(c->err, 0, sizeof(int), c->st));
  map_idx_kernel<<<((int)ni + 255) / 256, 256, 0, c->st>>>(c->idx, (int)ni, c->n, c->iperm, c->err);
  CKLAUNCH("map_idx");
  int e = 0, rc;
  if ((rc = read_and_clear_err(c, &e))) return rc;
  if (e) return fail(STEPS_EINVAL, "subset index out of range");
  const double inv_a3 = 1.0 / (c->a * c->a * c->a);
  double* o = c->stage;  // 3 ni <= 3 n
  if (c->p.precision == STEPS_FP64) {
    CK(cudaEventRecord(c->e0, c->st));
    if ((rc = launch_fp64(c, c->idx, (int)ni, c->sub))) return rc;
    CK(cudaEventRecord(c->e1, c->st));
    c->timed = true;
    c->last_images = (double)ni * (double)(c->n - 1) * images_per_pair(c);
    subset_finalize_kernel<<<((int)ni + 255) / 256, 256, 0, c->st>>>(c->sub, (int)ni, c->idx, -c->p.G * c->invL * c->invL,
                                                                     bg_params(c), c->x, c->y, c->z, inv_a3, o, o + ni,
                                                                     o + 2 * ni, c->err);
    CKLAUNCH("subset_finalize");
  } else {
    // FP32 forms: full evaluation, then gather the listed particles
    if ((rc = eval_forces(c, false, 0.0))) return rc;
    gather3_kernel<<<((int)ni + 255) / 256, 256, 0, c->st>>>(c->gx, c->gy, c->gz, c->idx, (int)ni, inv_a3, o, o + ni,
                                                             o + 2 * ni);
    CKLAUNCH("gather");
  }
  const size_t b = sizeof(double) * (size_t)ni;
  CK(cudaMemcpyAsync(ax, o, b, cudaMemcpyDefault, c->st));
  CK(cudaMemcpyAsync(ay, o + ni, b, cudaMemcpyDefault, c->st));
  CK(cudaMemcpyAsync(az, o + 2 * ni, b, cudaMemcpyDefault, c->st));
  if ((rc = read_and_clear_err(c, &e))) return rc;
  if (e) return device_error(e);
  return STEPS_OK;
}

int steps_cyl_kdk_step(steps_cyl_ctx* c, double dt, int32_t nsteps) {
  g_last_error.clear();
  if (!c) return fail(STEPS_EINVAL, "ctx is NULL");
  if (c->shard) return refuse_sharded(c, "steps_cyl_kdk_step");
  if (!(dt > 0) || !std::isfinite(dt)) return fail(STEPS_EINVAL, "dt must be finite and > 0");
  if (nsteps < 0) return fail(STEPS_EINVAL, "nsteps must be >= 0");
  DeviceGuard guard(c->dev);
  int rc;
  bool rejected = false;
  char reject_msg[160] = "";
  if (nsteps > 0 && c->forces_stale && (rc = eval_forces(c, false, 0.0))) return rc;
  for (int s = 0; s < nsteps; ++s) {
    Range range("steps_cyl.kdk_step");
    const Factors f = kdk_factors(c->cosmo, c->a, dt);
    if (!std::isfinite(f.K1) || !std::isfinite(f.D) || !std::isfinite(f.a_next) || !(f.a_next > 0))
      return fail(STEPS_EINVAL, "the Friedmann integration left the valid range (a = %g)", f.a_next);
    kick_drift_pack_kernel<<<grid_for(c->n, 256), 256, 0, c->st>>>(c->x, c->y, c->z, c->px, c->py, c->pz, c->gx,
                                                                   c->gy, c->gz, c->m, c->h, c->n, f.K1, f.D, c->p.L,
                                                                   c->invL, c->jA, c->jB, c->err, is_r3(c) ? 0 : 1);
    CKLAUNCH("kick_drift_pack");
    if ((rc = eval_forces(c, true, f.K2))) return rc;
    c->a = f.a_next;
    c->t += dt;
    if (c->p.reorder_every > 0 && ++c->steps_since_order >= c->p.reorder_every) {
      if ((rc = reorder(c))) return rc;
    }
    // modelled tail: periodic comparison with the plain image sum
    const bool surr = c->p.tail == STEPS_TAIL_SURROGATE && c->surr_ok;
    const bool table = c->p.tail == STEPS_TAIL_TABLE && c->tab_ok && !is_inf(c);  // the infinite window's reference
    if ((surr || table) && c->p.check_every > 0 && ++c->steps_since_check >= c->p.check_every) {
      c->steps_since_check = 0;
      double med = 0, p999 = 0;
      const int ncheck = c->p.check_particles > 0 ? c->p.check_particles : 1024;
      if ((rc = run_check(c, c->p.tail, ncheck, 0xc4ec0000ull + (uint64_t)s, &med, &p999, nullptr, nullptr)))
        return rc;
      const double bmed = surr ? c->surr_bound_med : c->tab_bound_med;
      const double bp999 = surr ? c->surr_bound_p999 : c->tab_bound_p999;
      if (!(med <= bmed && p999 <= bp999)) {
        (surr ? c->surr_ok : c->tab_ok) = false;
        c->p.tail = is_inf(c) ? STEPS_TAIL_TABLE : STEPS_TAIL_FULL;
        rejected = true;
        snprintf(reject_msg, sizeof reject_msg, "%s dropped after a check: median %.3g, p99.9 %.3g",
                 surr ? "surrogate" : "correction table", med, p999);
      }
    }
  }
  int e = 0;
  if ((rc = read_and_clear_err(c, &e))) return rc;
  if (e) return device_error(e);
  if (rejected) return fail(STEPS_ESURROGATE_REJECTED, "%s", reject_msg);
  return STEPS_OK;
}

int steps_cyl_get_state(steps_cyl_ctx* c, double* x, double* y, double* z, double* vx, double* vy, double* vz,
                        double* a, double* t) {
  g_last_error.clear();
  if (!c) return fail(STEPS_EINVAL, "ctx is NULL");
  DeviceGuard guard(c->dev);
  int rc;
  {
    const double* src[3] = {c->x, c->y, c->z};
    double* dst[3] = {x, y, z};
    if ((rc = scatter_out(c, src, dst, 1.0))) return rc;
  }
  {
    const double* src[3] = {c->px, c->py, c->pz};
    double* dst[3] = {vx, vy, vz};
    if ((rc = scatter_out(c, src, dst, 1.0 / (c->a * c->a)))) return rc;
  }
  if (a) *a = c->a;
  if (t) *t = c->t;
  return STEPS_OK;
}

int steps_cyl_set_state(steps_cyl_ctx* c, const double* x, const double* y, const double* z, const double* vx,
                        const double* vy, const double* vz) {
  g_last_error.clear();
  if (!c) return fail(STEPS_EINVAL, "ctx is NULL");
  if (c->shard) return refuse_sharded(c, "steps_cyl_set_state");
  if (!x || !y || !z || !vx || !vy || !vz) return fail(STEPS_EINVAL, "NULL input array");
  DeviceGuard guard(c->dev);
  int rc;
  if ((rc = stage_positions(c, x, y, z))) return rc;
  CK(cudaMemsetAsync(c->err, 0, sizeof(int), c->st));
  double* s = c->stage;
  positions_changed_kernel<<<grid_for(c->n, 256), 256, 0, c->st>>>(c->x, c->y, c->z, s, s + c->n,
                                                                   s + 2 * (size_t)c->n, c->perm, c->n, c->err);
  CKLAUNCH("positions_changed");
  int changed = 0;
  if ((rc = read_and_clear_err(c, &changed))) return rc;
  if (changed && (rc = order_from_stage(c, s, s + c->n, true))) return rc;
  if ((rc = install_state(c, vx, vy, vz))) return rc;
  if ((rc = validate_state(c))) return rc;
  // the cached forces stay valid when the positions are bitwise unchanged
  if (changed) {
    if ((rc = pack_positions(c))) return rc;
    if ((rc = eval_forces(c, false, 0.0))) return rc;
  }
  return STEPS_OK;
}

int steps_cyl_set_precision(steps_cyl_ctx* c, int32_t precision) {
  g_last_error.clear();
  if (!c) return fail(STEPS_EINVAL, "ctx is NULL");
  if (precision < STEPS_FP64 || precision > STEPS_FP32_PLAIN) return fail(STEPS_EINVAL, "bad precision");
  if (precision == STEPS_FP64 && is_inf(c)) return fail(STEPS_EINVAL, "the infinite window needs an FP32 precision");
  if (precision == STEPS_FP64 && is_tree(c)) return fail(STEPS_EINVAL, "the octree needs an FP32 precision");
  if (precision == STEPS_FP64 && c->shard) return fail(STEPS_EINVAL, "a sharded context needs an FP32 precision");
  DeviceGuard guard(c->dev);
  c->p.precision = precision;
  if (precision == STEPS_FP64) c->p.tail = STEPS_TAIL_FULL;
  c->forces_stale = true;  // refreshed by the next force evaluation or KDK step
  return STEPS_OK;
}

int steps_cyl_diagnostics(steps_cyl_ctx* c, double out[8]) {
  g_last_error.clear();
  if (!c || !out) return fail(STEPS_EINVAL, "NULL argument");
  DeviceGuard guard(c->dev);
  const int k0 = c->k0;  // sharded: the rows this context owns
  diag_partial_kernel<<<kRedBlocks, kRedThreads, 0, c->st>>>(c->x + k0, c->y + k0, c->px + k0, c->py + k0, c->pz + k0,
                                                             c->m + k0, c->k1 - k0, c->red);
  CKLAUNCH("diag_partial");
  diag_final_kernel<<<1, 32, 0, c->st>>>(c->red, kRedBlocks, c->red + kRedBlocks * 6);
  CKLAUNCH("diag_final");
  double r[6];
  CK(cudaMemcpyAsync(r, c->red + kRedBlocks * 6, sizeof r, cudaMemcpyDeviceToHost, c->st));
  CK(cudaStreamSynchronize(c->st));
  const double a2 = c->a * c->a;
  out[0] = r[0];
  out[1] = r[1];
  out[2] = r[2];
  out[3] = r[3];
  out[4] = r[4] / (a2 * a2);
  out[5] = c->a;
  out[6] = c->t;
  out[7] = r[5];
  return STEPS_OK;
}

int steps_cyl_shard(steps_cyl_ctx* c, int32_t rank, int32_t world, int64_t* rows) {
  g_last_error.clear();
  if (!c || !rows) return fail(STEPS_EINVAL, "NULL argument");
  if (c->shard) return fail(STEPS_EINVAL, "the context is sharded already");
  if (world < 1 || rank < 0 || rank >= world) return fail(STEPS_EINVAL, "need 0 <= rank < world");
  if (world > c->NB) return fail(STEPS_EINVAL, "world = %d exceeds the %d blocks of %d rows", world, c->NB, kBI);
  if (is_tree(c)) return fail(STEPS_EINVAL, "the octree is not row-sharded");
  // the FP64 pair kernel reads the FP64 positions of every j, and only the
  // packed FP32 words of the other ranks' rows are exchanged
  if (c->p.precision == STEPS_FP64) return fail(STEPS_EINVAL, "a sharded context needs an FP32 precision");
  DeviceGuard guard(c->dev);
  // balanced contiguous ranges of i-blocks, the same on every rank
  const int base = c->NB / world, extra = c->NB % world;
  std::vector<int> off(world + 1);
  for (int r = 0; r <= world; ++r) off[r] = std::min(c->n, (r * base + std::min(r, extra)) * kBI);
  int chunk = 0;
  for (int r = 0; r < world; ++r) chunk = std::max(chunk, off[r + 1] - off[r]);
  const int b0 = rank * base + std::min(rank, extra), nbo = base + (rank < extra ? 1 : 0);
  const int k0 = off[rank], k1 = off[rank + 1];
  int rc0 = 0;
  if (!c->fix_ready && (rc0 = fix_scale(c))) return rc0;  // the scale of the symmetric step's sums
  int* d_off = nullptr;
  cudaError_t e = cudaMalloc(&d_off, sizeof(int) * (world + 1));
  if (e == cudaSuccess) e = cudaMemcpyAsync(d_off, off.data(), sizeof(int) * (world + 1), cudaMemcpyHostToDevice, c->st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->st);
  if (e != cudaSuccess) {  // the context stays whole and unsharded
    cudaFree(d_off);
    return fail(e == cudaErrorMemoryAllocation ? STEPS_ENOMEM : STEPS_ECUDA, "steps_cyl_shard: %s",
                cudaGetErrorString(e));
  }
  c->shard_off = d_off;
  set_rows(c, b0, nbo);
  c->shard_sym = world > 1 && STEPS_SYMMETRIC && !is_r3(c) && c->fix_ok;
  c->shard = true;
  c->shard_rank = rank;
  c->shard_world = world;
  c->chunk = chunk;
  c->p.reorder_every = -1;  // the internal order stays the one every rank holds
  rows[0] = k0;
  rows[1] = k1;
  rows[2] = chunk;
  return STEPS_OK;
}

// A caller's exchange buffer: device memory, 16-byte aligned (float4 rows).
static bool exchange_buffer_ok(const void* p) { return p && !is_host_ptr(p) && ((uintptr_t)p & 15u) == 0; }

int steps_cyl_shard_drift(steps_cyl_ctx* c, double dt, float* send) {
  g_last_error.clear();
  if (!c) return fail(STEPS_EINVAL, "ctx is NULL");
  if (!c->shard) return fail(STEPS_EINVAL, "the context is not sharded (steps_cyl_shard)");
  if (c->drifted) return fail(STEPS_EINVAL, "steps_cyl_shard_kick must follow the last steps_cyl_shard_drift");
  if (!(dt > 0) || !std::isfinite(dt)) return fail(STEPS_EINVAL, "dt must be finite and > 0");
  if (!exchange_buffer_ok(send)) return fail(STEPS_EINVAL, "send must be 16-byte aligned device memory");
  DeviceGuard guard(c->dev);
  Range range("steps_cyl.shard_drift");
  int rc;
  if (c->forces_stale && (rc = eval_forces(c, false, 0.0))) return rc;
  const Factors f = kdk_factors(c->cosmo, c->a, dt);
  if (!std::isfinite(f.K1) || !std::isfinite(f.D) || !std::isfinite(f.a_next) || !(f.a_next > 0))
    return fail(STEPS_EINVAL, "the Friedmann integration left the valid range (a = %g)", f.a_next);
  const int k0 = c->k0, rows = c->k1 - c->k0;
  kick_drift_pack_kernel<<<grid_for(rows, 256), 256, 0, c->st>>>(
      c->x + k0, c->y + k0, c->z + k0, c->px + k0, c->py + k0, c->pz + k0, c->gx + k0, c->gy + k0, c->gz + k0,
      c->m + k0, c->h + k0, rows, f.K1, f.D, c->p.L, c->invL, c->jA + k0, c->jB + k0, c->err, is_r3(c) ? 0 : 1);
  CKLAUNCH("kick_drift_pack");
  shard_send_kernel<<<grid_for(c->chunk, 256), 256, 0, c->st>>>(c->jA, c->jB, k0, rows, c->chunk,
                                                                 reinterpret_cast<float4*>(send));
  CKLAUNCH("shard_send");
  c->pend_K2 = f.K2;
  c->pend_a = f.a_next;
  c->pend_dt = dt;
  c->drifted = true;
  return STEPS_OK;
}

int steps_cyl_shard_kick(steps_cyl_ctx* c, const float* recv) {
  g_last_error.clear();
  if (!c) return fail(STEPS_EINVAL, "ctx is NULL");
  if (!c->shard) return fail(STEPS_EINVAL, "the context is not sharded (steps_cyl_shard)");
  if (!c->drifted) return fail(STEPS_EINVAL, "steps_cyl_shard_drift must come first");
  if (c->forced) return fail(STEPS_EINVAL, "steps_cyl_shard_force was called: finish with steps_cyl_shard_finish");
  if (!exchange_buffer_ok(recv)) return fail(STEPS_EINVAL, "recv must be 16-byte aligned device memory");
  DeviceGuard guard(c->dev);
  Range range("steps_cyl.shard_kick");
  shard_recv_kernel<<<dim3(grid_for(c->chunk, 256), c->shard_world), 256, 0, c->st>>>(
      reinterpret_cast<const float4*>(recv), c->shard_off, c->chunk, c->jA, c->jB);
  CKLAUNCH("shard_recv");
  int rc;
  if ((rc = eval_forces(c, true, c->pend_K2))) return rc;
  c->a = c->pend_a;
  c->t += c->pend_dt;
  c->drifted = false;
  int e = 0;
  if ((rc = read_and_clear_err(c, &e))) return rc;
  if (e) return device_error(e);
  return STEPS_OK;
}

int steps_cyl_last_timing(steps_cyl_ctx* c, double* pair_images, double* pair_ms) {
  g_last_error.clear();
  if (!c) return fail(STEPS_EINVAL, "ctx is NULL");
  if (!c->timed) return fail(STEPS_EINVAL, "no force evaluation yet");
  DeviceGuard guard(c->dev);
  CK(cudaEventSynchronize(c->e1));
  float ms = 0.f;
  CK(cudaEventElapsedTime(&ms, c->e0, c->e1));
  if (pair_images) *pair_images = c->last_images;
  if (pair_ms) *pair_ms = ms;
  return STEPS_OK;
}

int steps_cyl_shard_mode(steps_cyl_ctx* c, int32_t* symmetric, int64_t* sums_len) {
  g_last_error.clear();
  if (!c || !symmetric) return fail(STEPS_EINVAL, "NULL argument");
  if (!c->shard) return fail(STEPS_EINVAL, "the context is not sharded (steps_cyl_shard)");
  *symmetric = c->shard_sym ? 1 : 0;
  if (sums_len) *sums_len = c->shard_sym ? (int64_t)c->shard_world * 3 * c->chunk : 0;
  return STEPS_OK;
}

int steps_cyl_shard_force(steps_cyl_ctx* c, const float* recv, int64_t* sums) {
  g_last_error.clear();
  if (!c) return fail(STEPS_EINVAL, "ctx is NULL");
  if (!c->shard || !c->shard_sym) return fail(STEPS_EINVAL, "the context has no symmetric sharded step");
  if (!c->drifted || c->forced) return fail(STEPS_EINVAL, "steps_cyl_shard_force must follow steps_cyl_shard_drift");
  if (!exchange_buffer_ok(recv) || !exchange_buffer_ok(sums))
    return fail(STEPS_EINVAL, "recv and sums must be 16-byte aligned device memory");
  const Form form = force_form(c);
  if (form == Form::FP64 || (form == Form::PLAIN && is_inf(c)))
    return fail(STEPS_EINVAL, "the symmetric sharded step needs an FP32 direct form");
  DeviceGuard guard(c->dev);
  Range range("steps_cyl.shard_force");
  shard_recv_kernel<<<dim3(grid_for(c->chunk, 256), c->shard_world), 256, 0, c->st>>>(
      reinterpret_cast<const float4*>(recv), c->shard_off, c->chunk, c->jA, c->jB);
  CKLAUNCH("shard_recv");
  const size_t len = (size_t)c->shard_world * 3 * c->chunk;
  CK(cudaMemsetAsync(sums, 0, sizeof(int64_t) * len, c->st));
  // this rank's equal share of the upper-triangle units, both sides of each pair
  const int W = c->shard_world, r = c->shard_rank;
  const long long Ua = (long long)r * c->Usym / W, Ub = (long long)(r + 1) * c->Usym / W;
  const FixAcc F{reinterpret_cast<unsigned long long*>(sums), c->n, c->fix_scale, c->err, W, c->NB / W, c->NB % W,
                 c->chunk};
  CK(cudaEventRecord(c->e0, c->st));
  int rc = launch_sym(c, form, Ua, Ub - Ua, F);
  if (rc) return rc;
  CK(cudaEventRecord(c->e1, c->st));
  c->timed = true;
  c->last_images = (double)(c->k1 - c->k0) * (double)(c->n - 1) * images_per_pair(c);
  c->last_pairs = sym_pairs(c) * (double)(Ub - Ua) / (double)c->Usym;
  c->last_sym = true;
  c->forced = true;
  return STEPS_OK;
}

int steps_cyl_shard_finish(steps_cyl_ctx* c, const int64_t* own) {
  g_last_error.clear();
  if (!c) return fail(STEPS_EINVAL, "ctx is NULL");
  if (!c->forced) return fail(STEPS_EINVAL, "steps_cyl_shard_force must come first");
  if (!exchange_buffer_ok(own)) return fail(STEPS_EINVAL, "own must be 16-byte aligned device memory");
  DeviceGuard guard(c->dev);
  Range range("steps_cyl.shard_finish");
  const int rows = c->k1 - c->k0;
  finalize_fix_kernel<<<(rows + 255) / 256, 256, 0, c->st>>>(
      reinterpret_cast<const unsigned long long*>(own), c->k1, c->k0, c->chunk, 1.0 / c->fix_scale,
      -c->p.G * c->invL * c->invL, bg_params(c), c->x, c->y, c->z, c->gx, c->gy, c->gz, c->pend_K2, c->px, c->py,
      c->pz, c->err);
  CKLAUNCH("finalize_fix");
  c->forces_stale = false;
  c->a = c->pend_a;
  c->t += c->pend_dt;
  c->drifted = false;
  c->forced = false;
  int e = 0, rc;
  if ((rc = read_and_clear_err(c, &e))) return rc;
  if (e) return device_error(e);
  return STEPS_OK;
}

int steps_cyl_last_eval(steps_cyl_ctx* c, double out[4]) {
  g_last_error.clear();
  if (!c || !out) return fail(STEPS_EINVAL, "NULL argument");
  if (!c->timed) return fail(STEPS_EINVAL, "no force evaluation yet");
  DeviceGuard guard(c->dev);
  CK(cudaEventSynchronize(c->e1));
  float ms = 0.f;
  CK(cudaEventElapsedTime(&ms, c->e0, c->e1));
  out[0] = c->last_images;
  out[1] = c->last_pairs;
  out[2] = ms;
  out[3] = c->last_sym ? (c->last_straight ? 2.0 : 1.0) : 0.0;
  return STEPS_OK;
}

int steps_cyl_free(steps_cyl_ctx* c) {
  g_last_error.clear();
  release(c);
  return STEPS_OK;
}

const char* steps_cyl_strerror(int code) {
  switch (code) {
    case STEPS_OK: return "ok";
    case STEPS_EINVAL: return "invalid argument";
    case STEPS_ECUDA: return "CUDA runtime error";
    case STEPS_ENOMEM: return "device out of memory";
    case STEPS_EDEVICE: return "device error word set";
    case STEPS_ESURROGATE_REJECTED: return "surrogate rejected; plain image sum used";
    case STEPS_ENOSURROGATE: return "no surrogate network loaded";
    default: return "unknown status";
  }
}

const char* steps_cyl_last_error(void) { return g_last_error.c_str(); }

// ---------------------------------------------------------------------------
// Checkpoint file: a fixed header, the background table and the per-particle
// arrays in the context's internal order with the permutation, so that a
// resumed context continues bit-identically.
// ---------------------------------------------------------------------------
struct CkptHeader {
  char magic[8];
  uint32_t version, header_bytes;
  steps_cyl_params p;
  int64_t n;
  double a, t, rho0, bg_dr, bound_med, bound_p999;
  int32_t steps_since_order, steps_since_check, surr_ok, bgK;
  float surr[STEPS_SURR_NPARAM];
  int32_t tab_ok, tab_nx, tab_ny, tab_read;  // correction table: rebuilt on resume from its grid and read
  double tab_dR_max, tab_bound_med, tab_bound_p999;
  uint64_t tree_evals;                  // octree: frame counter, fixed frame, radial table (after the header)
  int32_t tree_fixed, rad_nb;
  double tree_frame[9], rad_rmax;       // zeta, phi, centre, axis, angle
};
constexpr uint32_t kCkptVersion = 4;

int steps_cyl_checkpoint(steps_cyl_ctx* c, const char* path) {
  g_last_error.clear();
  if (!c || !path) return fail(STEPS_EINVAL, "NULL argument");
  if (c->shard) return refuse_sharded(c, "steps_cyl_checkpoint");
  DeviceGuard guard(c->dev);
  CkptHeader hd;
  std::memset(&hd, 0, sizeof hd);
  std::memcpy(hd.magic, "STEPSCYL", 8);
  hd.version = kCkptVersion;
  hd.header_bytes = sizeof hd;
  hd.p = c->p;
  hd.p.stream = nullptr;
  hd.n = c->n;
  hd.a = c->a;
  hd.t = c->t;
  hd.rho0 = c->rho0;
  hd.bg_dr = c->bg_dr;
  hd.bound_med = c->surr_bound_med;
  hd.bound_p999 = c->surr_bound_p999;
  hd.steps_since_order = c->steps_since_order;
  hd.steps_since_check = c->steps_since_check;
  hd.surr_ok = c->surr_ok ? 1 : 0;
  hd.bgK = c->bgtab ? c->bgK : 0;
  if (c->surr_ok) std::memcpy(hd.surr, c->surr_params.data(), sizeof hd.surr);
  hd.tab_ok = c->tab_ok ? 1 : 0;
  hd.tab_read = (c->tab.read == kReadTsc || c->tab.read == kReadTscExact) ? STEPS_TABLE_READ_TSC : STEPS_TABLE_READ_CIC;
  hd.tab_nx = c->tab_nx;
  hd.tab_ny = c->tab_ny;
  hd.tab_dR_max = c->tab_dR_max;
  hd.tab_bound_med = c->tab_bound_med;
  hd.tab_bound_p999 = c->tab_bound_p999;
  hd.tree_evals = c->tr.evals;
  hd.tree_fixed = c->tr.fixed ? 1 : 0;
  {
    const TreeDraw& f = c->tr.fd;
    const double v[9] = {f.zeta, f.phi, f.cen[0], f.cen[1], f.cen[2], f.axis[0], f.axis[1], f.axis[2], f.angle};
    std::memcpy(hd.tree_frame, v, sizeof v);
  }
  hd.rad_nb = c->tr.rad ? c->tr.rad_nb : 0;
  hd.rad_rmax = c->tr.rad_rmax;
  if (c->forces_stale) {
    int rc = eval_forces(c, false, 0.0);
    if (rc) return rc;
  }
  std::vector<double> arr((size_t)c->n * 11);
  std::vector<double> tab(hd.bgK ? hd.bgK + 4 : 0);
  CK(cudaMemcpyAsync(arr.data(), c->state, sizeof(double) * arr.size(), cudaMemcpyDeviceToHost, c->st));
  if (hd.bgK) CK(cudaMemcpyAsync(tab.data(), c->bgtab, sizeof(double) * tab.size(), cudaMemcpyDeviceToHost, c->st));
  CK(cudaStreamSynchronize(c->st));
  FILE* f = std::fopen(path, "wb");
  if (!f) return fail(STEPS_EINVAL, "cannot open %s for writing", path);
  bool ok = std::fwrite(&hd, sizeof hd, 1, f) == 1;
  if (ok && hd.bgK) ok = std::fwrite(tab.data(), sizeof(double), tab.size(), f) == tab.size();
  if (ok && hd.rad_nb) ok = std::fwrite(c->tr.rad_h.data(), sizeof(double), hd.rad_nb, f) == (size_t)hd.rad_nb;
  if (ok) ok = std::fwrite(arr.data(), sizeof(double), arr.size(), f) == arr.size();
  if (ok) ok = std::fwrite(c->perm_h.data(), sizeof(int), c->n, f) == (size_t)c->n;
  ok = (std::fclose(f) == 0) && ok;
  if (!ok) return fail(STEPS_EINVAL, "write to %s failed", path);
  return STEPS_OK;
}

int steps_cyl_resume(steps_cyl_ctx** out, const char* path, int32_t device, void* stream) {
  g_last_error.clear();
  if (!out || !path) return fail(STEPS_EINVAL, "NULL argument");
  *out = nullptr;
  FILE* f = std::fopen(path, "rb");
  if (!f) return fail(STEPS_EINVAL, "cannot open %s", path);
  CkptHeader hd;
  if (std::fread(&hd, sizeof hd, 1, f) != 1 || std::memcmp(hd.magic, "STEPSCYL", 8) != 0 ||
      hd.version != kCkptVersion || hd.header_bytes != sizeof hd || hd.n < 2 || hd.n > 0x7fffffffLL - kBI ||
      hd.bgK < 0 || hd.bgK > (1 << 20) || hd.rad_nb < 0 || hd.rad_nb > 4096) {
    std::fclose(f);
    return fail(STEPS_EINVAL, "%s is not a checkpoint of this library version", path);
  }
  // The header fixes the file's exact size; checking it first keeps a corrupt
  // particle count from sizing the buffers below.
  const long long need = (long long)sizeof hd + (hd.bgK ? (hd.bgK + 4LL) * 8 : 0) + hd.rad_nb * 8LL +
                         hd.n * (11LL * 8 + 4);
  if (std::fseek(f, 0, SEEK_END) != 0 || std::ftell(f) != need || std::fseek(f, (long)sizeof hd, SEEK_SET) != 0) {
    std::fclose(f);
    return fail(STEPS_EINVAL, "%s is truncated or has trailing bytes", path);
  }
  std::vector<double> tab(hd.bgK ? hd.bgK + 4 : 0), arr((size_t)hd.n * 11), rad(hd.rad_nb);
  std::vector<int> perm(hd.n);
  bool ok = !hd.bgK || std::fread(tab.data(), sizeof(double), tab.size(), f) == tab.size();
  ok = ok && (!hd.rad_nb || std::fread(rad.data(), sizeof(double), rad.size(), f) == rad.size());
  ok = ok && std::fread(arr.data(), sizeof(double), arr.size(), f) == arr.size();
  ok = ok && std::fread(perm.data(), sizeof(int), perm.size(), f) == perm.size();
  std::fclose(f);
  if (!ok) return fail(STEPS_EINVAL, "%s is truncated", path);
  hd.p.stream = stream;
  hd.p.device = device;
  int rc = check_params(&hd.p);
  if (rc) return rc;
  // Everything read from the file that indexes device memory or sizes a table
  // is checked before the first CUDA call: the permutation must be one of
  // [0, n), and a finite-cylinder background needs its table.
  {
    std::vector<char> seen(hd.n, 0);
    for (int64_t k = 0; k < hd.n; ++k) {
      const int v = perm[k];
      if (v < 0 || v >= hd.n || seen[v]) return fail(STEPS_EINVAL, "corrupt checkpoint (permutation)");
      seen[v] = 1;
    }
  }
  if (hd.p.background == STEPS_BG_FINITE && (hd.bgK < 1 || !(hd.bg_dr > 0.0) || !std::isfinite(hd.bg_dr)))
    return fail(STEPS_EINVAL, "corrupt checkpoint (background table)");
  if (!(hd.a > 0.0) || !std::isfinite(hd.a) || !std::isfinite(hd.t) || !(hd.rho0 >= 0.0) ||
      !std::isfinite(hd.rho0))
    return fail(STEPS_EINVAL, "corrupt checkpoint (a, t or rho0)");
  int ndev = 0;
  CK(cudaGetDeviceCount(&ndev));
  if (device < 0 || device >= ndev) return fail(STEPS_EINVAL, "device %d out of range", device);
  DeviceGuard guard(device);
  steps_cyl_ctx* c = new steps_cyl_ctx();
  c->p = hd.p;
  c->n = (int)hd.n;
  c->dev = device;
  c->st = (cudaStream_t)stream;
  c->cosmo = Cosmology{hd.p.H0, hd.p.Omega_m, hd.p.Omega_r, hd.p.Omega_L, hd.p.w0, hd.p.wa, hd.p.comoving != 0};
  c->a = hd.a;
  c->t = hd.t;
  c->rho0 = hd.rho0;
  c->invL = 1.0 / hd.p.L;
  c->steps_since_order = hd.steps_since_order;
  c->steps_since_check = hd.steps_since_check;
  c->tr.evals = hd.tree_evals;
  c->tr.fixed = hd.tree_fixed != 0;
  {
    TreeDraw& f = c->tr.fd;
    const double* v = hd.tree_frame;
    f.zeta = v[0];
    f.phi = v[1];
    for (int a = 0; a < 3; ++a) {
      f.cen[a] = v[2 + a];
      f.axis[a] = v[5 + a];
    }
    f.angle = v[8];
  }
  c->surr_bound_med = hd.bound_med;
  c->surr_bound_p999 = hd.bound_p999;
  c->perm_h = perm;
  auto bail = [&](int code) {
    release(c);
    return code;
  };
  if (c->tr.fixed && (rc = check_frame(c, c->tr.fd))) return bail(rc);
  if ((rc = allocate_context(c))) return bail(rc);
  if (cudaMemcpyAsync(c->state, arr.data(), sizeof(double) * arr.size(), cudaMemcpyHostToDevice, c->st) !=
      cudaSuccess)
    return bail(fail(STEPS_ECUDA, "upload failed"));
  if (hd.bgK) {
    c->bgK = hd.bgK;
    c->bg_dr = hd.bg_dr;
    if (cudaMalloc(&c->bgtab, sizeof(double) * tab.size()) != cudaSuccess ||
        cudaMemcpyAsync(c->bgtab, tab.data(), sizeof(double) * tab.size(), cudaMemcpyHostToDevice, c->st) !=
            cudaSuccess)
      return bail(fail(STEPS_ECUDA, "background table upload failed"));
  }
  if ((rc = upload_perm(c))) return bail(rc);
  if ((rc = validate_state(c))) return bail(rc);
  if ((rc = pack_positions(c))) return bail(rc);
  if (hd.surr_ok) {
    if ((rc = install_surrogate(c, hd.surr))) return bail(rc);
    c->surr_ok = true;
  }
  if (hd.tab_ok) {  // the table is a deterministic function of its grid: rebuilt, not stored
    if (hd.tab_nx < 2 || hd.tab_nx > 4096 || hd.tab_ny < 2 || hd.tab_ny > 1024 || !(hd.tab_dR_max > 0) ||
        (hd.tab_read != STEPS_TABLE_READ_CIC && hd.tab_read != STEPS_TABLE_READ_TSC))
      return bail(fail(STEPS_EINVAL, "corrupt checkpoint (table grid)"));
    c->tab_read_next = hd.tab_read;
    if ((rc = build_table(c, hd.tab_nx, hd.tab_ny, hd.tab_dR_max, nullptr))) return bail(rc);
    c->tab_ok = true;
    c->tab_bound_med = hd.tab_bound_med;
    c->tab_bound_p999 = hd.tab_bound_p999;
  }
  if (hd.rad_nb) {
    bool good = hd.rad_rmax > 0 && std::isfinite(hd.rad_rmax);
    for (double v : rad) good = good && std::isfinite(v);
    if (!good) return bail(fail(STEPS_EINVAL, "corrupt checkpoint (radial table)"));
    if ((rc = set_radial(c, rad, hd.rad_rmax))) return bail(rc);
  }
  if (cudaStreamSynchronize(c->st) != cudaSuccess) return bail(fail(STEPS_ECUDA, "synchronise failed"));
  *out = c;
  return STEPS_OK;
}

int steps_cyl_train_cfg_default(steps_cyl_train_cfg* cfg) {
  if (!cfg) return fail(STEPS_EINVAL, "cfg is NULL");
  std::memset(cfg, 0, sizeof *cfg);
  cfg->n_samples = 1 << 20;
  cfg->epochs = 60;
  cfg->batch = 8192;
  cfg->lr = 3e-3;
  cfg->dR_max = 0.0;
  cfg->seed = 1;
  cfg->err_median = 1e-5;
  cfg->err_p999 = 1e-3;
  cfg->check_particles = 1024;
  return STEPS_OK;
}

int steps_cyl_tail_sums(int64_t ns, const double* samples, int32_t n_cut, int32_t n0, double* out, void* stream) {
  g_last_error.clear();
  if (ns < 0 || !samples || !out) return fail(STEPS_EINVAL, "bad arguments");
  if (n_cut < 0 || n_cut > 4096 || n0 < 0 || (n_cut > 0 && n0 >= n_cut) || (n_cut == 0 && n0 >= kKInf))
    return fail(STEPS_EINVAL, "need 0 <= n0 < n_cut <= 4096, or n_cut = 0 and 0 <= n0 < %d", kKInf);
  if (ns == 0) return STEPS_OK;
  cudaStream_t st = (cudaStream_t)stream;
  double *ds = nullptr, *dout = nullptr;
  CK(cudaMallocAsync(&ds, sizeof(double) * 3 * ns, st));
  CK(cudaMallocAsync(&dout, sizeof(double) * 2 * ns, st));
  CK(cudaMemcpyAsync(ds, samples, sizeof(double) * 3 * ns, cudaMemcpyDefault, st));
  tail_sums_fp64_kernel<<<grid_for((int)std::min<int64_t>(ns, 1 << 30), 128), 128, 0, st>>>(ds, ns, n_cut, n0, dout);
  CKLAUNCH("tail_sums");
  CK(cudaMemcpyAsync(out, dout, sizeof(double) * 2 * ns, cudaMemcpyDefault, st));
  CK(cudaFreeAsync(ds, st));
  CK(cudaFreeAsync(dout, st));
  CK(cudaStreamSynchronize(st));
  return STEPS_OK;
}

int steps_cyl_mlp_loss_grad(int64_t ns, const float* w, const float* u, const float* t, float* loss, float* grad,
                            void* stream) {
  g_last_error.clear();
  if (ns < 1 || ns > (1 << 26) || !w || !u || !t || !loss || !grad) return fail(STEPS_EINVAL, "bad arguments");
  cudaStream_t st = (cudaStream_t)stream;
  const int nblk = (int)((ns + kTrainThreads - 1) / kTrainThreads);
  float *dw, *du, *dt, *gp, *lp, *dg, *dl;
  CK(cudaMallocAsync(&dw, sizeof(float) * kNW, st));
  CK(cudaMallocAsync(&du, sizeof(float) * 3 * ns, st));
  CK(cudaMallocAsync(&dt, sizeof(float) * 2 * ns, st));
  CK(cudaMallocAsync(&gp, sizeof(float) * kNW * (size_t)nblk, st));
  CK(cudaMallocAsync(&lp, sizeof(float) * nblk, st));
  CK(cudaMallocAsync(&dg, sizeof(float) * kNW, st));
  CK(cudaMallocAsync(&dl, sizeof(float), st));
  CK(cudaMemcpyAsync(dw, w, sizeof(float) * kNW, cudaMemcpyDefault, st));
  CK(cudaMemcpyAsync(du, u, sizeof(float) * 3 * ns, cudaMemcpyDefault, st));
  CK(cudaMemcpyAsync(dt, t, sizeof(float) * 2 * ns, cudaMemcpyDefault, st));
  mlp_fwd_bwd_kernel<<<nblk, kTrainThreads, 0, st>>>(dw, du, dt, nullptr, 0, ns, gp, lp);
  mlp_reduce_adam_kernel<<<(kNW + 127) / 128, 128, 0, st>>>(gp, nblk, 1.0f / (float)ns, nullptr, nullptr, nullptr,
                                                            0.f, 0.f, 0.f, 0.f, 1.f, 1.f, 0, dg);
  sum_floats_kernel<<<1, 32, 0, st>>>(lp, nblk, 1.0f / (float)ns, dl);
  CKLAUNCH("mlp_loss_grad");
  CK(cudaMemcpyAsync(grad, dg, sizeof(float) * kNW, cudaMemcpyDefault, st));
  CK(cudaMemcpyAsync(loss, dl, sizeof(float), cudaMemcpyDefault, st));
  for (float* p : {dw, du, dt, gp, lp, dg, dl}) CK(cudaFreeAsync(p, st));
  CK(cudaStreamSynchronize(st));
  return STEPS_OK;
}

int steps_cyl_train_surrogate(steps_cyl_ctx* c, const steps_cyl_train_cfg* cfg, double* report) {
  g_last_error.clear();
  if (!c || !cfg) return fail(STEPS_EINVAL, "NULL argument");
  if (c->shard) return refuse_sharded(c, "steps_cyl_train_surrogate (train before sharding)");
  DeviceGuard guard(c->dev);
  if (c->p.precision == STEPS_FP64) return fail(STEPS_EINVAL, "the surrogate needs an FP32 precision");
  const int32_t tail = c->p.tail;
  c->p.tail = STEPS_TAIL_FULL;  // the check compares against the plain sum explicitly
  int rc = train_surrogate(c, cfg, report);
  c->p.tail = (rc == STEPS_OK) ? tail : STEPS_TAIL_FULL;
  return rc;
}

int steps_cyl_set_surrogate(steps_cyl_ctx* c, const float* params, double err_median, double err_p999,
                            double* report) {
  g_last_error.clear();
  if (!c || !params) return fail(STEPS_EINVAL, "NULL argument");
  if (c->shard) return refuse_sharded(c, "steps_cyl_set_surrogate (install before sharding)");
  if (!(err_median > 0) || !(err_p999 > 0)) return fail(STEPS_EINVAL, "bounds must be > 0");
  if (is_r3(c) || c->p.n0 < 1 || (c->p.n_cut > 0 && c->p.n0 >= c->p.n_cut))
    return fail(STEPS_EINVAL, "the learned tail needs 1 <= n0 < n_cut (S1xR2)");
  DeviceGuard guard(c->dev);
  std::vector<float> P(STEPS_SURR_NPARAM);
  CK(cudaMemcpyAsync(P.data(), params, sizeof(float) * STEPS_SURR_NPARAM, cudaMemcpyDefault, c->st));
  CK(cudaStreamSynchronize(c->st));
  double med = 0, p999 = 0;
  bool ok = false;
  const int ncheck = c->p.check_particles > 0 ? c->p.check_particles : 1024;
  int rc = accept_surrogate(c, P.data(), err_median, err_p999, ncheck, &med, &p999, &ok);
  if (rc) return rc;
  if (report) {
    report[0] = med;
    report[1] = p999;
    report[2] = ok ? 1.0 : 0.0;
    report[3] = 0.0;
  }
  if (!ok) {
    c->p.tail = STEPS_TAIL_FULL;
    return fail(STEPS_ESURROGATE_REJECTED, "surrogate rejected: median %.3g, p99.9 %.3g", med, p999);
  }
  return STEPS_OK;
}

int steps_cyl_surrogate_lanes(const float* params, uint32_t* lanes, float* shift) {
  g_last_error.clear();
  if (!params || !lanes || !shift) return fail(STEPS_EINVAL, "NULL argument");
  static_assert(sizeof(SurrLane) == 4 * STEPS_SURR_LANE_WORDS, "lane record size");
  SurrLane rec[32];
  build_lanes(params, rec);
  std::memcpy(lanes, rec, sizeof rec);
  surr_shift(params, shift);
  return STEPS_OK;
}

int steps_cyl_get_surrogate(steps_cyl_ctx* c, float* params) {
  g_last_error.clear();
  if (!c || !params) return fail(STEPS_EINVAL, "NULL argument");
  if (!c->surr_ok || c->surr_params.size() != STEPS_SURR_NPARAM)
    return fail(STEPS_ENOSURROGATE, "no accepted surrogate is loaded");
  std::memcpy(params, c->surr_params.data(), sizeof(float) * STEPS_SURR_NPARAM);
  return STEPS_OK;
}

int steps_cyl_set_tail(steps_cyl_ctx* c, int32_t tail) {
  g_last_error.clear();
  if (!c) return fail(STEPS_EINVAL, "ctx is NULL");
  if (tail != STEPS_TAIL_FULL && tail != STEPS_TAIL_SURROGATE && tail != STEPS_TAIL_TABLE)
    return fail(STEPS_EINVAL, "bad tail mode");
  if (is_inf(c) && tail == STEPS_TAIL_FULL) return fail(STEPS_EINVAL, "the infinite window has no plain image sum");
  if (is_tree(c) && tail != (is_r3(c) ? STEPS_TAIL_FULL : STEPS_TAIL_TABLE))
    return fail(STEPS_EINVAL, "the octree evaluates one pair form (S1xR2: the correction table; R^3: the plain force)");
  if (tail == STEPS_TAIL_SURROGATE && !c->surr_ok) return fail(STEPS_ENOSURROGATE, "no accepted surrogate is loaded");
  if (tail == STEPS_TAIL_TABLE && !c->tab_ok) return fail(STEPS_ENOSURROGATE, "no accepted correction table is built");
  if (tail != STEPS_TAIL_FULL && c->p.precision == STEPS_FP64)
    return fail(STEPS_EINVAL, "a modelled tail needs an FP32 precision");
  c->p.tail = tail;
  c->steps_since_check = 0;
  c->forces_stale = true;  // refreshed by the next force evaluation or KDK step
  return STEPS_OK;
}

int steps_cyl_check_surrogate(steps_cyl_ctx* c, int32_t check_particles, double* report) {
  g_last_error.clear();
  if (!c || !report || check_particles < 1) return fail(STEPS_EINVAL, "bad arguments");
  if (!c->surr_ok) return fail(STEPS_ENOSURROGATE, "no accepted surrogate is loaded");
  DeviceGuard guard(c->dev);
  return run_check(c, STEPS_TAIL_SURROGATE, check_particles, 0xc4ec0000ull + (uint64_t)c->steps_since_check,
                   &report[0], &report[1], &report[2], &report[3]);
}

int steps_cyl_build_tail_table(steps_cyl_ctx* c, int32_t nx, int32_t ny, double dR_max, double err_median,
                               double err_p999, int32_t check_particles, double* report) {
  g_last_error.clear();
  if (!c) return fail(STEPS_EINVAL, "ctx is NULL");
  if (c->shard) return refuse_sharded(c, "steps_cyl_build_tail_table (build before sharding)");
  if (nx < 2 || nx > 4096 || ny < 2 || ny > 1024) return fail(STEPS_EINVAL, "nx must be in [2, 4096], ny in [2, 1024]");
  if (!(dR_max >= 0) || !std::isfinite(dR_max)) return fail(STEPS_EINVAL, "dR_max must be finite and >= 0");
  if (!(err_median > 0) || !(err_p999 > 0) || check_particles < 1) return fail(STEPS_EINVAL, "bad check bounds");
  if (c->p.precision == STEPS_FP64) return fail(STEPS_EINVAL, "the correction table needs an FP32 precision");
  DeviceGuard guard(c->dev);
  double ms = 0.0;
  int rc = build_table(c, nx, ny, dR_max, &ms);
  if (rc) return rc;
  double med = NAN, p999 = NAN;
  bool ok = true;
  if (is_inf(c))
    c->tab_ok = true;  // the infinite window has no plain sum to check against: the table is its definition
  else if ((rc = accept_table(c, err_median, err_p999, check_particles, &med, &p999, &ok)))
    return rc;
  if (report) {
    report[0] = med;
    report[1] = p999;
    report[2] = ok ? 1.0 : 0.0;
    report[3] = ms;
  }
  if (!ok) return fail(STEPS_ESURROGATE_REJECTED, "correction table rejected: median %.3g, p99.9 %.3g", med, p999);
  return STEPS_OK;
}

int steps_cyl_build_tail_table_ewald(steps_cyl_ctx* c, int32_t nx, int32_t ny, double dR_max, double alpha,
                                     int32_t nmax, int32_t mmax, double* report) {
  g_last_error.clear();
  if (!c) return fail(STEPS_EINVAL, "ctx is NULL");
  if (c->shard) return refuse_sharded(c, "steps_cyl_build_tail_table_ewald (build before sharding)");
  if (!is_inf(c)) return fail(STEPS_EINVAL, "the Ewald construction is for the infinite window (n_cut = 0)");
  if (nx < 2 || nx > 4096 || ny < 2 || ny > 1024) return fail(STEPS_EINVAL, "nx must be in [2, 4096], ny in [2, 1024]");
  if (!(dR_max >= 0) || !std::isfinite(dR_max)) return fail(STEPS_EINVAL, "dR_max must be finite and >= 0");
  if (!(alpha >= 0.25 && alpha <= 8.0)) return fail(STEPS_EINVAL, "alpha must be in [0.25, 8] (units 1/L)");
  if (nmax < c->p.n0 || nmax > 64 || mmax < 0 || mmax > 64)
    return fail(STEPS_EINVAL, "need n0 <= nmax <= 64 and 0 <= mmax <= 64");
  if (c->p.precision == STEPS_FP64) return fail(STEPS_EINVAL, "the correction table needs an FP32 precision");
  DeviceGuard guard(c->dev);
  const EwaldParams ew{alpha, nmax, mmax};
  double rep[4] = {0, 0, 0, 0};
  int rc = build_table(c, nx, ny, dR_max, nullptr, &ew, rep);
  if (rc) return rc;
  c->tab_ok = true;
  if (report) std::copy(rep, rep + 4, report);
  return STEPS_OK;
}

int steps_cyl_set_table_read(steps_cyl_ctx* c, int32_t read) {
  g_last_error.clear();
  if (!c) return fail(STEPS_EINVAL, "ctx is NULL");
  if (read != STEPS_TABLE_READ_CIC && read != STEPS_TABLE_READ_TSC)
    return fail(STEPS_EINVAL, "read must be STEPS_TABLE_READ_CIC or STEPS_TABLE_READ_TSC");
  c->tab_read_next = read;
  return STEPS_OK;
}

int steps_cyl_get_tail_table(steps_cyl_ctx* c, float* out, int32_t* nx, int32_t* ny, double* dR_max) {
  g_last_error.clear();
  if (!c) return fail(STEPS_EINVAL, "ctx is NULL");
  if (!c->tab_arr) return fail(STEPS_ENOSURROGATE, "no correction table is built");
  if (nx) *nx = c->tab_nx;
  if (ny) *ny = c->tab_ny;
  if (dR_max) *dR_max = c->tab_dR_max;
  if (out) {
    DeviceGuard guard(c->dev);
    CK(cudaMemcpy2DFromArrayAsync(out, sizeof(float2) * c->tab_nx, c->tab_arr, 0, 0, sizeof(float2) * c->tab_nx,
                                  c->tab_ny, cudaMemcpyDeviceToHost, c->st));
    CK(cudaStreamSynchronize(c->st));
  }
  return STEPS_OK;
}

int steps_cyl_check_tail(steps_cyl_ctx* c, int32_t tail, int32_t check_particles, double* report) {
  g_last_error.clear();
  if (!c || !report || check_particles < 1) return fail(STEPS_EINVAL, "bad arguments");
  if (tail == STEPS_TAIL_SURROGATE) return steps_cyl_check_surrogate(c, check_particles, report);
  if (tail != STEPS_TAIL_TABLE) return fail(STEPS_EINVAL, "bad tail mode");
  if (!c->tab_ok) return fail(STEPS_ENOSURROGATE, "no accepted correction table is built");
  if (is_inf(c)) return fail(STEPS_EINVAL, "the infinite window has no plain image sum to check against");
  DeviceGuard guard(c->dev);
  return run_check(c, STEPS_TAIL_TABLE, check_particles, 0xc4ec0000ull + (uint64_t)c->steps_since_check,
                   &report[0], &report[1], &report[2], &report[3]);
}


int steps_cyl_tree_frame(steps_cyl_ctx* c, double zeta, double phi) {
  g_last_error.clear();
  if (!c) return fail(STEPS_EINVAL, "ctx is NULL");
  if (!is_tree(c)) return fail(STEPS_EINVAL, "the context does not use the octree");
  if (is_r3(c)) return fail(STEPS_EINVAL, "the R^3 octree takes steps_cyl_tree_frame_r3");
  if (zeta < 0.0) {
    c->tr.fixed = false;
  } else {
    TreeDraw f{};
    f.zeta = zeta;
    f.phi = phi;
    int rc = check_frame(c, f);
    if (rc) return rc;
    c->tr.fixed = true;
    c->tr.fd = f;
  }
  c->forces_stale = true;
  return STEPS_OK;
}

int steps_cyl_tree_frame_r3(steps_cyl_ctx* c, const double* frame) {
  g_last_error.clear();
  if (!c) return fail(STEPS_EINVAL, "ctx is NULL");
  if (!is_tree(c) || !is_r3(c)) return fail(STEPS_EINVAL, "the context does not use the R^3 octree");
  if (!frame) {
    c->tr.fixed = false;
  } else {
    TreeDraw f{};
    for (int a = 0; a < 3; ++a) {
      f.cen[a] = frame[a];
      f.axis[a] = frame[3 + a];
    }
    f.angle = frame[6];
    int rc = check_frame(c, f);
    if (rc) return rc;
    c->tr.fixed = true;
    c->tr.fd = f;
  }
  c->forces_stale = true;
  return STEPS_OK;
}

int steps_cyl_tree_stats(steps_cyl_ctx* c, double* out) {
  g_last_error.clear();
  if (!c || !out) return fail(STEPS_EINVAL, "NULL argument");
  if (!is_tree(c)) return fail(STEPS_EINVAL, "the context does not use the octree");
  out[0] = c->tr.nodes;
  out[1] = c->tr.depth;
  out[2] = c->tr.interactions;
  out[3] = c->tr.build_ms;
  out[4] = c->tr.walk_ms;
  out[5] = (double)c->tr.evals;
  return STEPS_OK;
}

int steps_cyl_tree_set_radial(steps_cyl_ctx* c, const double* table, int32_t n_bins, double rmax) {
  g_last_error.clear();
  if (!c || !table) return fail(STEPS_EINVAL, "NULL argument");
  if (!is_tree(c)) return fail(STEPS_EINVAL, "the context does not use the octree");
  if (n_bins < 1 || n_bins > 4096 || !(rmax > 0) || !std::isfinite(rmax)) return fail(STEPS_EINVAL, "bad table shape");
  std::vector<double> tab(table, table + n_bins);
  for (double v : tab)
    if (!std::isfinite(v)) return fail(STEPS_EINVAL, "non-finite table entry");
  DeviceGuard guard(c->dev);
  c->forces_stale = true;
  return set_radial(c, tab, rmax);
}

int steps_cyl_tree_calibrate(steps_cyl_ctx* c, int32_t n_frames, int32_t n_bins, int32_t n_sample,
                             const double* frames, const int64_t* sample, double* table, double* rmax) {
  g_last_error.clear();
  if (!c) return fail(STEPS_EINVAL, "ctx is NULL");
  if (!is_tree(c)) return fail(STEPS_EINVAL, "the context does not use the octree");
  if (n_frames < 0 || n_frames > 4096) return fail(STEPS_EINVAL, "n_frames must be in [0, 4096]");
  DeviceGuard guard(c->dev);
  c->forces_stale = true;
  if (n_frames == 0) {
    cudaFree(c->tr.rad);
    c->tr.rad = nullptr;
    c->tr.rad_nb = 0;
    c->tr.rad_h.clear();
    return STEPS_OK;
  }
  if (n_bins < 1 || n_bins > 4096 || n_sample < 1) return fail(STEPS_EINVAL, "bad bins or sample size");
  std::vector<double> tab;
  double rm = 0.0;
  int rc = tree_calibrate(c, n_frames, n_bins, n_sample, frames, sample, tab, &rm);
  if (rc) return rc;
  if ((rc = set_radial(c, tab, rm))) return rc;
  if (table) std::memcpy(table, tab.data(), sizeof(double) * n_bins);
  if (rmax) *rmax = rm;
  return STEPS_OK;
}


}  // extern "C"
