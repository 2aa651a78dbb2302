// C ABI of the S1xR2 StePS hot path (arXiv 2602.20787) on GB300 / sm_103a.
// Declarations and the contract of every entry point are in include/steps_cyl.h.
//
// Host side of the library: context, argument checks, the FP64 Friedmann/RK4
// schedule of the kick and drift factors (Sect. 2.3), the tabulated finite-height
// part of the background term (eq. F_horiz), and the launch sequence of a force
// evaluation and of a KDK step. All particle work runs in the kernels of
// pair_fp32.cuh and nbody_kernels.cuh.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "steps_cyl.h"
#include "nbody_kernels.cuh"

using namespace steps;

namespace {

thread_local std::string g_last_error;

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
struct steps_cyl_ctx {
  steps_cyl_params p{};
  int n = 0;
  int dev = 0;
  cudaStream_t st = nullptr;
  Cosmology cosmo{};
  double a = 1.0, t = 0.0, rho0 = 0.0, invL = 1.0;
  // device state (FP64 SoA)
  double* state = nullptr;  // one allocation for the 11 arrays below
  double *x, *y, *z, *px, *py, *pz, *m, *h, *gx, *gy, *gz;
  float4* jA = nullptr;
  float4* jB = nullptr;
  double* part = nullptr;   // stream-K partials or direct FP64 sums
  size_t part_elems = 0;
  double* stage = nullptr;  // 3 n doubles for outputs
  double* red = nullptr;    // reduction scratch
  int64_t* idx = nullptr;   // subset indices (grown on demand)
  int idx_cap = 0;
  double* sub = nullptr;    // subset sums (3 * idx_cap)
  int* err = nullptr;
  double* bgtab = nullptr;
  int bgK = 0;
  double bg_dr = 0.0;
  int C = 0, NT = 0, NB = 0;
  long long U = 0;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  double last_images = 0.0;
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

int check_params(const steps_cyl_params* p) {
  if (!p) return fail(STEPS_EINVAL, "params is NULL");
  if (!(p->G > 0) || !std::isfinite(p->G)) return fail(STEPS_EINVAL, "G must be finite and > 0");
  if (!(p->L > 0) || !std::isfinite(p->L)) return fail(STEPS_EINVAL, "L must be finite and > 0");
  if (!(p->R_sim > 0) || !std::isfinite(p->R_sim)) return fail(STEPS_EINVAL, "R_sim must be finite and > 0");
  if (!(p->rho_bar >= 0) || !std::isfinite(p->rho_bar)) return fail(STEPS_EINVAL, "rho_bar must be >= 0");
  if (p->n_cut < 1 || p->n_cut > 4096) return fail(STEPS_EINVAL, "n_cut must be in [1, 4096]");
  if (p->precision < STEPS_FP64 || p->precision > STEPS_FP32_PLAIN) return fail(STEPS_EINVAL, "bad precision");
  if (p->tail != STEPS_TAIL_FULL && p->tail != STEPS_TAIL_SURROGATE) return fail(STEPS_EINVAL, "bad tail mode");
  if (p->tail == STEPS_TAIL_SURROGATE && (p->n0 < 1 || p->n0 >= p->n_cut))
    return fail(STEPS_EINVAL, "n0 must be in [1, n_cut)");
  if (p->background < STEPS_BG_OFF || p->background > STEPS_BG_INFINITE) return fail(STEPS_EINVAL, "bad background");
  if (p->comoving) {
    if (!(p->H0 > 0) || !(p->a_start > 0)) return fail(STEPS_EINVAL, "comoving runs need H0 > 0 and a_start > 0");
  }
  if (p->reserved != 0) return fail(STEPS_EINVAL, "reserved must be 0");
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
    if (!(z[i] >= 0.0 && z[i] < L)) b |= 8;
    if (b) atomicOr(bad, b);
  }
}

// Sets *changed when any uploaded position differs bitwise from the current one.
__global__ void positions_changed_kernel(const double* __restrict__ x, const double* __restrict__ y,
                                         const double* __restrict__ z, const double* __restrict__ nx,
                                         const double* __restrict__ ny, const double* __restrict__ nz, int n,
                                         int* __restrict__ changed) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    if (__double_as_longlong(x[i]) != __double_as_longlong(nx[i]) ||
        __double_as_longlong(y[i]) != __double_as_longlong(ny[i]) ||
        __double_as_longlong(z[i]) != __double_as_longlong(nz[i])) {
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

__global__ void gather3_kernel(const double* __restrict__ ax, const double* __restrict__ ay,
                               const double* __restrict__ az, const int64_t* __restrict__ idx, int ni,
                               double* __restrict__ ox, double* __restrict__ oy, double* __restrict__ oz) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q < ni) {
    const int64_t i = idx[q];
    ox[q] = ax[i]; oy[q] = ay[i]; oz[q] = az[i];
  }
}

__global__ void check_idx_kernel(const int64_t* __restrict__ idx, int ni, int n, int* __restrict__ bad) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q < ni && (idx[q] < 0 || idx[q] >= n)) atomicOr(bad, 16);
}

int read_and_clear_err(steps_cyl_ctx* c, int* out) {
  int h = 0;
  CK(cudaMemcpyAsync(&h, c->err, sizeof(int), cudaMemcpyDeviceToHost, c->st));
  CK(cudaStreamSynchronize(c->st));
  CK(cudaMemsetAsync(c->err, 0, sizeof(int), c->st));
  *out = h;
  return STEPS_OK;
}

int device_error(int e) {
  return fail(STEPS_EDEVICE, "device error word 0x%x (%s%s%s)", e, (e & kErrNonFinite) ? "non-finite value " : "",
              (e & kErrBgRange) ? "particle beyond background table " : "", (e & kErrZRange) ? "z range" : "");
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

// One force evaluation at the current packed positions. Stores g = a^3 (pair +
// background) in gx/gy/gz; kicks p by K when kick is set; writes g inv_a3 to
// (ox, oy, oz) when given (device pointers).
int eval_forces(steps_cyl_ctx* c, bool kick, double K, double* ox, double* oy, double* oz, double inv_a3) {
  const double pair_scale = -c->p.G * c->invL * c->invL;
  CK(cudaEventRecord(c->e0, c->st));
  if (c->p.precision == STEPS_FP64) {
    pair_fp64_kernel<<<(c->n + 127) / 128, 128, 0, c->st>>>(c->x, c->y, c->z, c->m, c->h, c->n, nullptr, c->n,
                                                            c->invL, c->p.n_cut, c->part);
    CKLAUNCH("pair_fp64");
  } else if (c->p.precision == STEPS_FP32_KAHAN) {
    pair_fp32_kernel<true><<<c->C, kBI, 0, c->st>>>(c->jA, c->jB, c->n, c->p.n_cut, c->U, c->NT, c->C, c->part);
    CKLAUNCH("pair_fp32_kahan");
  } else {
    pair_fp32_kernel<false><<<c->C, kBI, 0, c->st>>>(c->jA, c->jB, c->n, c->p.n_cut, c->U, c->NT, c->C, c->part);
    CKLAUNCH("pair_fp32_plain");
  }
  CK(cudaEventRecord(c->e1, c->st));
  c->timed = true;
  c->last_images = (double)c->n * (double)(c->n - 1) * 2.0 * c->p.n_cut;
  const int NT = c->p.precision == STEPS_FP64 ? 0 : c->NT;
  finalize_kernel<<<(c->n + 255) / 256, 256, 0, c->st>>>(
      c->part, c->n, NT, c->U, c->C, pair_scale, bg_params(c), c->x, c->y, c->gx, c->gy, c->gz, K,
      kick ? c->px : nullptr, kick ? c->py : nullptr, kick ? c->pz : nullptr, inv_a3, ox, oy, oz, c->err);
  CKLAUNCH("finalize");
  return STEPS_OK;
}

int upload_state(steps_cyl_ctx* c, const double* x, const double* y, const double* z, const double* vx,
                 const double* vy, const double* vz) {
  const size_t b = sizeof(double) * (size_t)c->n;
  CK(cudaMemcpyAsync(c->x, x, b, cudaMemcpyDefault, c->st));
  CK(cudaMemcpyAsync(c->y, y, b, cudaMemcpyDefault, c->st));
  CK(cudaMemcpyAsync(c->z, z, b, cudaMemcpyDefault, c->st));
  CK(cudaMemcpyAsync(c->px, vx, b, cudaMemcpyDefault, c->st));
  CK(cudaMemcpyAsync(c->py, vy, b, cudaMemcpyDefault, c->st));
  CK(cudaMemcpyAsync(c->pz, vz, b, cudaMemcpyDefault, c->st));
  // canonical momentum p = a^2 dx/dt
  if (c->a != 1.0) {
    axpy_scale3_kernel<<<grid_for(c->n, 256), 256, 0, c->st>>>(c->px, c->py, c->pz, c->n, c->a * c->a);
    CKLAUNCH("to_momentum");
  }
  return STEPS_OK;
}

int validate_state(steps_cyl_ctx* c) {
  CK(cudaMemsetAsync(c->err, 0, sizeof(int), c->st));
  validate_kernel<<<grid_for(c->n, 256), 256, 0, c->st>>>(c->x, c->y, c->z, c->px, c->py, c->pz, c->m, c->h, c->n,
                                                           c->p.L, c->err);
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
  pack_kernel<<<grid_for(c->n, 256), 256, 0, c->st>>>(c->x, c->y, c->z, c->m, c->h, c->n, c->invL, c->jA, c->jB);
  CKLAUNCH("pack");
  return STEPS_OK;
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
  cudaFree(c->idx);
  cudaFree(c->sub);
  cudaFree(c->err);
  cudaFree(c->bgtab);
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

int copy_out3(steps_cyl_ctx* c, const double* sx, const double* sy, const double* sz, double* ox, double* oy,
              double* oz, size_t cnt) {
  const size_t b = sizeof(double) * cnt;
  bool host = false;
  if (ox) { CK(cudaMemcpyAsync(ox, sx, b, cudaMemcpyDefault, c->st)); host |= is_host_ptr(ox); }
  if (oy) { CK(cudaMemcpyAsync(oy, sy, b, cudaMemcpyDefault, c->st)); host |= is_host_ptr(oy); }
  if (oz) { CK(cudaMemcpyAsync(oz, sz, b, cudaMemcpyDefault, c->st)); host |= is_host_ptr(oz); }
  if (host) CK(cudaStreamSynchronize(c->st));
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
  p->reserved = 0;
  p->stream = nullptr;
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
  CKI(cudaEventCreate(&c->e0));
  CKI(cudaEventCreate(&c->e1));
  CKI(cudaMalloc(&c->state, sizeof(double) * nb * 11));
  double* s = c->state;
  c->x = s; c->y = s + nb; c->z = s + 2 * nb; c->px = s + 3 * nb; c->py = s + 4 * nb; c->pz = s + 5 * nb;
  c->m = s + 6 * nb; c->h = s + 7 * nb; c->gx = s + 8 * nb; c->gy = s + 9 * nb; c->gz = s + 10 * nb;
  CKI(cudaMalloc(&c->jA, sizeof(float4) * nb));
  CKI(cudaMalloc(&c->jB, sizeof(float4) * nb));
  CKI(cudaMalloc(&c->stage, sizeof(double) * nb * 3));
  CKI(cudaMalloc(&c->red, sizeof(double) * (kRedBlocks * 6 + 8)));
  CKI(cudaMalloc(&c->err, sizeof(int)));
  CKI(cudaMemsetAsync(c->err, 0, sizeof(int), c->st));

  // stream-K split of the FP32 pair kernel: C co-resident CTAs share U units
  int sms = 0, occ = 0;
  CKI(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c->dev));
  CKI(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, pair_fp32_kernel<true>, kBI, 0));
  c->NB = (c->n + kBI - 1) / kBI;
  c->NT = (c->n + kBJ - 1) / kBJ;
  c->U = (long long)c->NB * c->NT;
  c->C = (int)std::min<long long>(c->U, (long long)sms * std::max(occ, 1));
  c->part_elems = std::max((size_t)(c->NB + c->C) * 3 * kBI, nb * 3);
  CKI(cudaMalloc(&c->part, sizeof(double) * c->part_elems));

  CKI(cudaMemcpyAsync(c->m, m, sizeof(double) * nb, cudaMemcpyDefault, c->st));
  CKI(cudaMemcpyAsync(c->h, h, sizeof(double) * nb, cudaMemcpyDefault, c->st));
  if ((rc = upload_state(c, x, y, z, vx, vy, vz))) return bail(rc);
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
    c->rho0 = tot / (M_PI * p->R_sim * p->R_sim * p->L);
  }
  if ((rc = build_background(c))) return bail(rc);
  if ((rc = pack_positions(c))) return bail(rc);
  if ((rc = eval_forces(c, false, 0.0, nullptr, nullptr, nullptr, 1.0))) return bail(rc);
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
  DeviceGuard guard(c->dev);
  const double inv_a3 = 1.0 / (c->a * c->a * c->a);
  const bool host = is_host_ptr(ax) || is_host_ptr(ay) || is_host_ptr(az);
  int rc;
  if (host) {
    double* s = c->stage;
    if ((rc = eval_forces(c, false, 0.0, s, s + c->n, s + 2 * (size_t)c->n, inv_a3))) return rc;
    if ((rc = copy_out3(c, s, s + c->n, s + 2 * (size_t)c->n, ax, ay, az, c->n))) return rc;
    int e = 0;
    if ((rc = read_and_clear_err(c, &e))) return rc;
    if (e) return device_error(e);
  } else {
    if ((rc = eval_forces(c, false, 0.0, ax, ay, az, inv_a3))) return rc;
  }
  return STEPS_OK;
}

int steps_cyl_forces_subset(steps_cyl_ctx* c, int64_t ni, const int64_t* idx, double* ax, double* ay, double* az) {
  g_last_error.clear();
  if (!c) return fail(STEPS_EINVAL, "ctx is NULL");
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
  check_idx_kernel<<<((int)ni + 255) / 256, 256, 0, c->st>>>(c->idx, (int)ni, c->n, c->err);
  CKLAUNCH("check_idx");
  int e = 0, rc;
  if ((rc = read_and_clear_err(c, &e))) return rc;
  if (e) return fail(STEPS_EINVAL, "subset index out of range");
  const double inv_a3 = 1.0 / (c->a * c->a * c->a);
  double* o = c->stage;  // 3 ni <= 3 n
  if (c->p.precision == STEPS_FP64) {
    CK(cudaEventRecord(c->e0, c->st));
    pair_fp64_kernel<<<((int)ni + 127) / 128, 128, 0, c->st>>>(c->x, c->y, c->z, c->m, c->h, c->n, c->idx, (int)ni,
                                                               c->invL, c->p.n_cut, c->sub);
    CKLAUNCH("pair_fp64_subset");
    CK(cudaEventRecord(c->e1, c->st));
    c->timed = true;
    c->last_images = (double)ni * (double)(c->n - 1) * 2.0 * c->p.n_cut;
    subset_finalize_kernel<<<((int)ni + 255) / 256, 256, 0, c->st>>>(c->sub, (int)ni, c->idx, -c->p.G * c->invL * c->invL,
                                                                     bg_params(c), c->x, c->y, inv_a3, o, o + ni,
                                                                     o + 2 * ni, c->err);
    CKLAUNCH("subset_finalize");
  } else {
    // FP32 forms: full evaluation, then gather the listed particles
    if ((rc = eval_forces(c, false, 0.0, nullptr, nullptr, nullptr, inv_a3))) return rc;
    gather3_kernel<<<((int)ni + 255) / 256, 256, 0, c->st>>>(c->gx, c->gy, c->gz, c->idx, (int)ni, o, o + ni,
                                                             o + 2 * ni);
    CKLAUNCH("gather");
    axpy_scale3_kernel<<<grid_for((int)ni, 256), 256, 0, c->st>>>(o, o + ni, o + 2 * ni, (int)ni, inv_a3);
    CKLAUNCH("scale");
  }
  if ((rc = copy_out3(c, o, o + ni, o + 2 * ni, ax, ay, az, (size_t)ni))) return rc;
  if ((rc = read_and_clear_err(c, &e))) return rc;
  if (e) return device_error(e);
  return STEPS_OK;
}

int steps_cyl_kdk_step(steps_cyl_ctx* c, double dt, int32_t nsteps) {
  g_last_error.clear();
  if (!c) return fail(STEPS_EINVAL, "ctx is NULL");
  if (!(dt > 0) || !std::isfinite(dt)) return fail(STEPS_EINVAL, "dt must be finite and > 0");
  if (nsteps < 0) return fail(STEPS_EINVAL, "nsteps must be >= 0");
  DeviceGuard guard(c->dev);
  int rc;
  for (int s = 0; s < nsteps; ++s) {
    const Factors f = kdk_factors(c->cosmo, c->a, dt);
    if (!std::isfinite(f.K1) || !std::isfinite(f.D) || !std::isfinite(f.a_next) || !(f.a_next > 0))
      return fail(STEPS_EINVAL, "the Friedmann integration left the valid range (a = %g)", f.a_next);
    kick_drift_pack_kernel<<<grid_for(c->n, 256), 256, 0, c->st>>>(c->x, c->y, c->z, c->px, c->py, c->pz, c->gx,
                                                                   c->gy, c->gz, c->m, c->h, c->n, f.K1, f.D, c->p.L,
                                                                   c->invL, c->jA, c->jB, c->err);
    CKLAUNCH("kick_drift_pack");
    if ((rc = eval_forces(c, true, f.K2, nullptr, nullptr, nullptr, 1.0))) return rc;
    c->a = f.a_next;
    c->t += dt;
  }
  int e = 0;
  if ((rc = read_and_clear_err(c, &e))) return rc;
  if (e) return device_error(e);
  return STEPS_OK;
}

int steps_cyl_get_state(steps_cyl_ctx* c, double* x, double* y, double* z, double* vx, double* vy, double* vz,
                        double* a, double* t) {
  g_last_error.clear();
  if (!c) return fail(STEPS_EINVAL, "ctx is NULL");
  DeviceGuard guard(c->dev);
  int rc;
  if ((rc = copy_out3(c, c->x, c->y, c->z, x, y, z, c->n))) return rc;
  if (vx || vy || vz) {
    double* s = c->stage;
    const double inv_a2 = 1.0 / (c->a * c->a);
    scale3_kernel<<<grid_for(c->n, 256), 256, 0, c->st>>>(c->px, c->py, c->pz, c->n, inv_a2, s, s + c->n,
                                                          s + 2 * (size_t)c->n);
    CKLAUNCH("velocity");
    if ((rc = copy_out3(c, s, s + c->n, s + 2 * (size_t)c->n, vx, vy, vz, c->n))) return rc;
  }
  if (a) *a = c->a;
  if (t) *t = c->t;
  return STEPS_OK;
}

int steps_cyl_set_state(steps_cyl_ctx* c, const double* x, const double* y, const double* z, const double* vx,
                        const double* vy, const double* vz) {
  g_last_error.clear();
  if (!c) return fail(STEPS_EINVAL, "ctx is NULL");
  if (!x || !y || !z || !vx || !vy || !vz) return fail(STEPS_EINVAL, "NULL input array");
  DeviceGuard guard(c->dev);
  int rc;
  // stage the new positions, compare them with the current ones, then install
  const size_t b = sizeof(double) * (size_t)c->n;
  double* s = c->stage;
  CK(cudaMemcpyAsync(s, x, b, cudaMemcpyDefault, c->st));
  CK(cudaMemcpyAsync(s + c->n, y, b, cudaMemcpyDefault, c->st));
  CK(cudaMemcpyAsync(s + 2 * (size_t)c->n, z, b, cudaMemcpyDefault, c->st));
  CK(cudaMemsetAsync(c->err, 0, sizeof(int), c->st));
  positions_changed_kernel<<<grid_for(c->n, 256), 256, 0, c->st>>>(c->x, c->y, c->z, s, s + c->n,
                                                                   s + 2 * (size_t)c->n, c->n, c->err);
  CKLAUNCH("positions_changed");
  int changed = 0;
  if ((rc = read_and_clear_err(c, &changed))) return rc;
  if ((rc = upload_state(c, s, s + c->n, s + 2 * (size_t)c->n, vx, vy, vz))) return rc;
  if ((rc = validate_state(c))) return rc;
  // the cached forces stay valid when the positions are bitwise unchanged
  if (changed) {
    if ((rc = pack_positions(c))) return rc;
    if ((rc = eval_forces(c, false, 0.0, nullptr, nullptr, nullptr, 1.0))) return rc;
  }
  return STEPS_OK;
}

int steps_cyl_set_precision(steps_cyl_ctx* c, int32_t precision) {
  g_last_error.clear();
  if (!c) return fail(STEPS_EINVAL, "ctx is NULL");
  if (precision < STEPS_FP64 || precision > STEPS_FP32_PLAIN) return fail(STEPS_EINVAL, "bad precision");
  DeviceGuard guard(c->dev);
  c->p.precision = precision;
  return eval_forces(c, false, 0.0, nullptr, nullptr, nullptr, 1.0);
}

int steps_cyl_diagnostics(steps_cyl_ctx* c, double out[8]) {
  g_last_error.clear();
  if (!c || !out) return fail(STEPS_EINVAL, "NULL argument");
  DeviceGuard guard(c->dev);
  diag_partial_kernel<<<kRedBlocks, kRedThreads, 0, c->st>>>(c->x, c->y, c->px, c->py, c->pz, c->m, c->n, c->red);
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

}  // extern "C"
