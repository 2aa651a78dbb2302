// O(N) kernels of the S1xR2 step and the FP64 pair kernel (arXiv 2602.20787,
// eq. ComovingEquationsOfMotionCylindrical and the KDK leapfrog of Sect. 2.1).
#pragma once
#include <cstdint>

#include "pair_fp32.cuh"

namespace steps {
// The kernels below have internal linkage (static): every translation unit
// that includes this header gets its own copy.

constexpr int kErrNonFinite = 1;     // a force, position or momentum is not finite
constexpr int kErrBgRange = 2;       // a particle lies beyond the background table
constexpr int kErrZRange = 4;        // z left [0, L) by more than rounding
constexpr int kErrTreeRange = 8;     // a particle lies outside the octree's root cube
constexpr int kErrTreeStack = 16;    // an octree walk outgrew its stack

// FP64 positions -> FP32 hi/lo words in units of L (see pair_fp32.cuh).
__device__ __forceinline__ void pack_one(double x, double y, double z, double m, double h, int i, double invL,
                                         float4* __restrict__ jA, float4* __restrict__ jB) {
  const double xu = x * invL, yu = y * invL, zu = z * invL;
  const float xh = (float)xu, yh = (float)yu, zh = (float)zu;
  const float xl = (float)(xu - (double)xh), yl = (float)(yu - (double)yh), zl = (float)(zu - (double)zh);
  jA[i] = make_float4(xh, yh, zh, (float)m);
  jB[i] = make_float4(xl, yl, zl, (float)(h * invL));
}

static __global__ void pack_kernel(const double* __restrict__ x, const double* __restrict__ y,
                            const double* __restrict__ z, const double* __restrict__ m,
                            const double* __restrict__ h, int n, double invL, float4* __restrict__ jA,
                            float4* __restrict__ jB) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    pack_one(x[i], y[i], z[i], m[i], h[i], i, invL, jA, jB);
}

// Background of eq. ComovingEquationsOfMotionCylindrical: returns F_h(rho) (< 0
// inside a homogeneous cylinder; the acceleration is -F_h along rho_hat).
// F_h = F_inf + dF, with F_inf the infinite cylinder (-2 pi G rho0 rho inside,
// -2 pi G rho0 R^2 / rho outside) and dF the smooth finite-height remainder,
// tabulated on a uniform grid (nodes -1 .. K+2) and read with 4-point Lagrange.
struct BgParams {
  int mode;            // STEPS_BG_* (3: the R^3 radial term +(4 pi G / 3) rho0 x)
  double two_pi_G_rho0;
  double R;
  const double* tab;   // dF at rho_k = k * dr, k = -1 .. K+2 (tab[0] is k = -1)
  int K;
  double inv_dr;
};

__device__ __forceinline__ double background_F(const BgParams& bg, double rho, int* err) {
  if (bg.mode == 0) return 0.0;
  double F = rho <= bg.R ? -bg.two_pi_G_rho0 * rho : -bg.two_pi_G_rho0 * bg.R * bg.R / rho;
  if (bg.mode == 1) {
    const double s = rho * bg.inv_dr;
    int k = (int)floor(s);
    if (k >= bg.K || !(s >= 0.0)) {
      atomicOr(err, kErrBgRange);
      k = bg.K - 1;
    }
    const double t = s - (double)k;  // in [0, 1)
    // Lagrange weights on nodes k-1, k, k+1, k+2 at offset t from node k
    const double wm = -t * (t - 1.0) * (t - 2.0) / 6.0;
    const double w0 = (t + 1.0) * (t - 1.0) * (t - 2.0) / 2.0;
    const double w1 = -(t + 1.0) * t * (t - 2.0) / 2.0;
    const double w2 = (t + 1.0) * t * (t - 1.0) / 6.0;
    const double* q = bg.tab + k;  // q[0] is node k-1
    F += wm * q[0] + w0 * q[1] + w1 * q[2] + w2 * q[3];
  }
  return F;
}

// The background term of particle (x, y, z) added to g (comoving field, a^3
// times the acceleration): the cylinder's F_h(rho) along -rho_hat (S1xR2), or
// the R^3 radial term +(4 pi G / 3) rho0 x = (2/3) (2 pi G rho0) x.
__device__ __forceinline__ void add_background(const BgParams& bg, double xi, double yi, double zi, double& g0,
                                               double& g1, double& g2, int* err) {
  if (bg.mode == 3) {
    const double c = bg.two_pi_G_rho0 * (2.0 / 3.0);
    g0 += c * xi;
    g1 += c * yi;
    g2 += c * zi;
    return;
  }
  const double rho = sqrt(xi * xi + yi * yi);
  if (rho > 0.0 && bg.mode != 0) {
    const double F = background_F(bg, rho, err);
    g0 -= F * xi / rho;
    g1 -= F * yi / rho;
  }
}

// Sum the stream-K partials of each i in CTA order (or read direct sums when
// NT == 0), scale to the comoving field
// g = a^3 (pair + background), store it, optionally kick p += g K and optionally
// write a = g / a^3 to an output.
// Radial correction of Sect. 2.4: g -= D(rho) rho_hat, D interpolated
// linearly between bin centres (k + 1/2) rmax / nb and held outside them.
// Radial correction of Sect. 2.4: g -= D(r) r_hat, D interpolated linearly
// between bin centres (k + 1/2) rmax / nb and held outside them; r is the
// cylindrical radius (S1xR2) or the distance from the origin (sph, R^3).
struct RadialCorr {
  const double* tab;  // nb bin means; null: no correction
  int nb;
  double rmax;
  int sph;
};

__device__ __forceinline__ void radial_correct(const RadialCorr& R, double x, double y, double z, double& g0,
                                               double& g1, double& g2) {
  if (!R.tab) return;
  const double rho = R.sph ? sqrt(x * x + y * y + z * z) : sqrt(x * x + y * y);
  if (!(rho > 0.0)) return;
  const double s = rho / R.rmax * R.nb - 0.5;
  double D;
  if (s <= 0.0) D = R.tab[0];
  else if (s >= R.nb - 1) D = R.tab[R.nb - 1];
  else {
    const int k = (int)s;
    const double t = s - k;
    D = (1.0 - t) * R.tab[k] + t * R.tab[k + 1];
  }
  g0 -= D * x / rho;
  g1 -= D * y / rho;
  if (R.sph) g2 -= D * z / rho;
}

// The common end of a finalize: the pair sums (sx, sy, sz) scaled to the
// comoving field g = a^3 (pair + background), the radial correction, the
// background; g stored, optionally p += g K, optionally a = g / a^3 written.
__device__ __forceinline__ void finish_particle(int i, double sx, double sy, double sz, double pair_scale,
                                                const BgParams& bg, const double* __restrict__ x,
                                                const double* __restrict__ y, const double* __restrict__ z,
                                                double* __restrict__ gx, double* __restrict__ gy,
                                                double* __restrict__ gz, double K, double* __restrict__ px,
                                                double* __restrict__ py, double* __restrict__ pz, double inv_a3,
                                                double* __restrict__ ox, double* __restrict__ oy,
                                                double* __restrict__ oz, int* __restrict__ err, const RadialCorr& rc) {
  double g0 = pair_scale * sx, g1 = pair_scale * sy, g2 = pair_scale * sz;
  radial_correct(rc, x[i], y[i], z[i], g0, g1, g2);
  add_background(bg, x[i], y[i], z[i], g0, g1, g2, err);
  if (err && (!isfinite(g0) || !isfinite(g1) || !isfinite(g2))) atomicOr(err, kErrNonFinite);
  gx[i] = g0; gy[i] = g1; gz[i] = g2;
  if (px) {
    px[i] += g0 * K;
    py[i] += g1 * K;
    pz[i] += g2 * K;
  }
  if (ox) {
    ox[i] = g0 * inv_a3;
    oy[i] = g1 * inv_a3;
    oz[i] = g2 * inv_a3;
  }
}

static __global__ void finalize_kernel(const double* __restrict__ part, int n, int NT, long long U, int C,
                                double pair_scale, BgParams bg, const double* __restrict__ x,
                                const double* __restrict__ y, const double* __restrict__ z, double* __restrict__ gx,
                                double* __restrict__ gy, double* __restrict__ gz, double K,
                                double* __restrict__ px, double* __restrict__ py, double* __restrict__ pz,
                                double inv_a3, double* __restrict__ ox, double* __restrict__ oy,
                                double* __restrict__ oz, int* __restrict__ err,
                                RadialCorr rc = RadialCorr{nullptr, 0, 0.0, 0}, int i0 = 0) {
  // rows [i0, n), i0 a multiple of kBI (all rows unless they are sharded); the
  // partials and direct sums are indexed from i0
  const int i = i0 + blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double sx = 0.0, sy = 0.0, sz = 0.0;
  if (NT == 0) {
    // direct sums (FP64 pair kernel): part = [3][n - i0]
    const long long q = i - i0, m = n - i0;
    sx = part[q];
    sy = part[m + q];
    sz = part[2 * m + q];
  } else {
    const int b = (i - i0) / kBI, l = (i - i0) % kBI;
    const long long p_lo = (long long)b * NT, p_hi = p_lo + NT - 1;
    const int c_lo = cta_of_unit(p_lo, U, C), c_hi = cta_of_unit(p_hi, U, C);
    for (int c = c_lo; c <= c_hi; ++c) {
      const double* q = part + ((long long)b + c) * 3 * kBI;
      sx += q[l];
      sy += q[kBI + l];
      sz += q[2 * kBI + l];
    }
  }
  finish_particle(i, sx, sy, sz, pair_scale, bg, x, y, z, gx, gy, gz, K, px, py, pz, inv_a3, ox, oy, oz, err, rc);
}

// Finalize from the fixed-point accumulators of the symmetric pair kernels
// (pair_sym.cuh), in units of 1 / scale, for the rows [i0, n): acc[3][stride]
// indexed from i0 (stride = n, i0 = 0 for every row; a rank's own rows of a
// sharded step have i0 = its first row and stride = its exchange chunk).
static __global__ void finalize_fix_kernel(const unsigned long long* __restrict__ acc, int n, int i0, int stride,
                                           double inv_scale, double pair_scale, BgParams bg,
                                           const double* __restrict__ x, const double* __restrict__ y,
                                           const double* __restrict__ z, double* __restrict__ gx,
                                           double* __restrict__ gy, double* __restrict__ gz, double K,
                                           double* __restrict__ px, double* __restrict__ py,
                                           double* __restrict__ pz, int* __restrict__ err) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  const int i = i0 + q;
  if (i >= n) return;
  const double sx = (double)(long long)acc[q] * inv_scale;
  const double sy = (double)(long long)acc[(long long)stride + q] * inv_scale;
  const double sz = (double)(long long)acc[2 * (long long)stride + q] * inv_scale;
  finish_particle(i, sx, sy, sz, pair_scale, bg, x, y, z, gx, gy, gz, K, px, py, pz, 1.0, nullptr, nullptr, nullptr,
                  err, RadialCorr{nullptr, 0, 0.0, 0});
}

// First half of a KDK step: p += g K1; x += p D; z wrapped into [0, L); repack.
static __global__ void kick_drift_pack_kernel(double* __restrict__ x, double* __restrict__ y,
                                       double* __restrict__ z, double* __restrict__ px,
                                       double* __restrict__ py, double* __restrict__ pz,
                                       const double* __restrict__ gx, const double* __restrict__ gy,
                                       const double* __restrict__ gz, const double* __restrict__ m,
                                       const double* __restrict__ h, int n, double K1, double D, double L,
                                       double invL, float4* __restrict__ jA, float4* __restrict__ jB,
                                       int* __restrict__ err, int wrap) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const double qx = px[i] + gx[i] * K1, qy = py[i] + gy[i] * K1, qz = pz[i] + gz[i] * K1;
    px[i] = qx; py[i] = qy; pz[i] = qz;
    const double nx = x[i] + qx * D, ny = y[i] + qy * D;
    double nz = z[i] + qz * D;
    if (wrap) {  // S1xR2: z into [0, L)
      nz -= L * floor(nz * invL);
      if (nz >= L) nz -= L;
      if (nz < 0.0) nz = 0.0;
    }
    if (!isfinite(nx) || !isfinite(ny) || !isfinite(nz)) atomicOr(err, kErrNonFinite);
    x[i] = nx; y[i] = ny; z[i] = nz;
    pack_one(nx, ny, nz, m[i], h[i], i, invL, jA, jB);
  }
}

// y = s x for three arrays (acceleration output = g / a^3).
static __global__ void scale3_kernel(const double* __restrict__ ax, const double* __restrict__ ay,
                              const double* __restrict__ az, int n, double s, double* __restrict__ ox,
                              double* __restrict__ oy, double* __restrict__ oz) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    ox[i] = ax[i] * s; oy[i] = ay[i] * s; oz[i] = az[i] * s;
  }
}

// p = a^2 v (and back) on three arrays.
static __global__ void axpy_scale3_kernel(double* __restrict__ a0, double* __restrict__ a1, double* __restrict__ a2,
                                   int n, double s) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    a0[i] *= s; a1[i] *= s; a2[i] *= s;
  }
}

// Deterministic reductions for the diagnostics: each block writes its partial
// sums of (m px, m py, m pz, m (x py - y px), m |p|^2 / 2, m) into part[block][6].
constexpr int kRedThreads = 256;
constexpr int kRedBlocks = 256;

static __global__ void diag_partial_kernel(const double* __restrict__ x, const double* __restrict__ y,
                                    const double* __restrict__ px, const double* __restrict__ py,
                                    const double* __restrict__ pz, const double* __restrict__ m, int n,
                                    double* __restrict__ part) {
  double v[6] = {0, 0, 0, 0, 0, 0};
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const double mi = m[i];
    v[0] += mi * px[i];
    v[1] += mi * py[i];
    v[2] += mi * pz[i];
    v[3] += mi * (x[i] * py[i] - y[i] * px[i]);
    v[4] += 0.5 * mi * (px[i] * px[i] + py[i] * py[i] + pz[i] * pz[i]);
    v[5] += mi;
  }
  __shared__ double sh[kRedThreads / 32][6];
#pragma unroll
  for (int q = 0; q < 6; ++q) {
    double s = v[q];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5][q] = s;
  }
  __syncthreads();
  if (threadIdx.x < 6) {
    double s = 0.0;
    for (int w = 0; w < kRedThreads / 32; ++w) s += sh[w][threadIdx.x];
    part[blockIdx.x * 6 + threadIdx.x] = s;
  }
}

static __global__ void diag_final_kernel(const double* __restrict__ part, int nblocks, double* __restrict__ out) {
  if (threadIdx.x < 6) {
    double s = 0.0;
    for (int b = 0; b < nblocks; ++b) s += part[b * 6 + threadIdx.x];
    out[threadIdx.x] = s;
  }
}

// ---------------------------------------------------------------------------
// FP64 pair kernel (precision study and reference form): same window and
// softening as the FP32 kernel but evaluated directly (branch on r < h) in
// FP64. idx == nullptr means i = q. Sums are sum_j m_j (dx, dy, dz-part) in
// units of G / L^2 (scaled by the caller), the same quantity as the FP32 sums.
// ---------------------------------------------------------------------------
__device__ __forceinline__ double spline_over_r_fp64(double r, double hh) {
  const double ih = 1.0 / hh, u = r * ih, ih3 = ih * ih * ih;
  if (u < 0.5) return (32.0 / 3.0 + u * u * (32.0 * u - 38.4)) * ih3;
  const double u3 = u * u * u;
  return (64.0 / 3.0 - 48.0 * u + 38.4 * u * u - (32.0 / 3.0) * u3 - 1.0 / (15.0 * u3)) * ih3;
}

__device__ __forceinline__ void image_fp64(double dR2, double o, double hh, double hh2, double w, double& sr,
                                           double& sz) {
  const double r2 = fma(o, o, dR2);
  double f;
  if (r2 < hh2) {
    f = spline_over_r_fp64(sqrt(r2), hh);
  } else {
    const double ri = rsqrt(r2);
    f = ri * ri * ri;
  }
  f *= w;
  sr += f;
  sz = fma(o, f, sz);
}

// CTA (bx, by) takes listed i-particles [bx * 128, +128) against j-tiles
// [by * tpc, (by + 1) * tpc) of 128 j staged in shared memory, so that a short
// list still fills the GPU; part[by][3][ni] receives the partial sums, which
// chunk_sum_kernel adds in chunk order.
static __global__ void __launch_bounds__(128)
pair_fp64_kernel(const double* __restrict__ x, const double* __restrict__ y, const double* __restrict__ z,
                 const double* __restrict__ m, const double* __restrict__ h, int n,
                 const int64_t* __restrict__ idx, int ni, double invL, int n_cut, int tpc, double* __restrict__ part,
                 int r3) {
  __shared__ double sx[128], sy[128], sz[128], sm[128], sh[128];
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  const int qq = min(q, ni - 1);
  const int i = idx ? (int)idx[qq] : qq;
  const double xi = x[i] * invL, yi = y[i] * invL, zi = z[i] * invL, hi = h[i] * invL;
  const int NT = (n + 127) / 128;
  const int t0 = blockIdx.y * tpc, t1 = min(NT, t0 + tpc);
  double ax = 0.0, ay = 0.0, az = 0.0;
  for (int t = t0; t < t1; ++t) {
    __syncthreads();
    const int jl = t * 128 + threadIdx.x;
    if (jl < n) {
      sx[threadIdx.x] = x[jl] * invL;
      sy[threadIdx.x] = y[jl] * invL;
      sz[threadIdx.x] = z[jl] * invL;
      sm[threadIdx.x] = m[jl];
      sh[threadIdx.x] = h[jl] * invL;
    }
    __syncthreads();
    const int jn = min(128, n - t * 128);
    for (int k = 0; k < jn; ++k) {
      if (t * 128 + k == i) continue;
      const double dx = xi - sx[k], dy = yi - sy[k];
      double dz = zi - sz[k];
      if (!r3) dz -= rint(dz);  // R^3: no period, the centre image alone (n_cut = 1, no edge)
      const double dR2 = dx * dx + dy * dy;
      const double hh = hi + sh[k], hh2 = hh * hh;
      double sr = 0.0, szz = 0.0;
      image_fp64(dR2, dz, hh, hh2, 1.0, sr, szz);
      if (!r3) image_fp64(dR2, dz - copysign((double)n_cut, dz), hh, hh2, dz != 0.0 ? 1.0 : 0.0, sr, szz);
      for (int kk = 1; kk < n_cut; ++kk) {
        image_fp64(dR2, dz + (double)kk, hh, hh2, 1.0, sr, szz);
        image_fp64(dR2, dz - (double)kk, hh, hh2, 1.0, sr, szz);
      }
      const double mj = sm[k];
      ax += mj * dx * sr;
      ay += mj * dy * sr;
      az += mj * szz;
    }
  }
  if (q < ni) {
    double* dst = part + (long long)blockIdx.y * 3 * ni;
    dst[q] = ax;
    dst[ni + q] = ay;
    dst[2 * (long long)ni + q] = az;
  }
}

// out[3][ni] = sum over chunks c (in order) of part[c][3][ni]
static __global__ void chunk_sum_kernel(const double* __restrict__ part, int ni, int chunks, double* __restrict__ out) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= ni) return;
  double s0 = 0.0, s1 = 0.0, s2 = 0.0;
  for (int c = 0; c < chunks; ++c) {
    const double* p = part + (long long)c * 3 * ni;
    s0 += p[q];
    s1 += p[ni + q];
    s2 += p[2 * (long long)ni + q];
  }
  out[q] = s0;
  out[ni + q] = s1;
  out[2 * (long long)ni + q] = s2;
}

// out3 (SoA, ni each) = pair_scale * pair + background at the listed i, / a^3
static __global__ void subset_finalize_kernel(const double* __restrict__ pairsum, int ni, const int64_t* __restrict__ idx,
                                       double pair_scale, BgParams bg, const double* __restrict__ x,
                                       const double* __restrict__ y, const double* __restrict__ z, double inv_a3,
                                       double* __restrict__ ox, double* __restrict__ oy, double* __restrict__ oz,
                                       int* __restrict__ err) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= ni) return;
  const int i = idx ? (int)idx[q] : q;
  double g0 = pair_scale * pairsum[q], g1 = pair_scale * pairsum[ni + q], g2 = pair_scale * pairsum[2 * ni + q];
  add_background(bg, x[i], y[i], z[i], g0, g1, g2, err);
  if (!isfinite(g0) || !isfinite(g1) || !isfinite(g2)) atomicOr(err, kErrNonFinite);
  ox[q] = g0 * inv_a3;
  oy[q] = g1 * inv_a3;
  oz[q] = g2 * inv_a3;
}

// ---------------------------------------------------------------------------
// Row sharding (Sect. 2.4's distributed direct engine, one rank per GPU). Each
// rank owns a contiguous range of internal rows; the only exchange of a step is
// the packed positions of every rank's rows, gathered between the drift and the
// force evaluation.
// The owned packed rows [k0, k0 + rows) -> send[chunk][2] = (jA, jB) per row,
// zero rows past the share, so every rank sends chunk rows.
static __global__ void shard_send_kernel(const float4* __restrict__ jA, const float4* __restrict__ jB, int k0,
                                         int rows, int chunk, float4* __restrict__ send) {
  for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < chunk; q += gridDim.x * blockDim.x) {
    const bool own = q < rows;
    send[2 * q] = own ? jA[k0 + q] : make_float4(0.f, 0.f, 0.f, 0.f);
    send[2 * q + 1] = own ? jB[k0 + q] : make_float4(0.f, 0.f, 0.f, 0.f);
  }
}

// The gathered recv[world][chunk][2] -> the packed arrays: rank r's rows are
// [off[r], off[r + 1]) (blockIdx.y = r).
static __global__ void shard_recv_kernel(const float4* __restrict__ recv, const int* __restrict__ off, int chunk,
                                         float4* __restrict__ jA, float4* __restrict__ jB) {
  const int r = blockIdx.y;
  const int o = off[r], rows = off[r + 1] - o;
  for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < rows; q += gridDim.x * blockDim.x) {
    const long long src = 2 * ((long long)r * chunk + q);
    jA[o + q] = recv[src];
    jB[o + q] = recv[src + 1];
  }
}

}  // namespace steps
