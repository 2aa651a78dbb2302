// Correction-table tail (arXiv 2602.20787, Sect. 2.3, eq.
// S1R2EwaldCorrectionTable). The paper tabulates the force of the periodic
// images beyond the nearest on an equally spaced (rho, z) grid and adds it,
// read with cloud-in-cell interpolation, to the nearest-image force. Here the
// same table is stated for the windowed sum of eq. ForceCylindrical: the images
// beyond the near range |k| <= n0, for point masses, as the residual of that
// tail over the continuum base in envelope units,
//   r = ((SR - BR) / ER, (SZ - BZ) / EZ)   at dz = +|dz| (SZ is odd in dz),
// at nodes dR_i = i dR_max / (nx - 1), |dz|_j = j / (2 (ny - 1)). The residual
// is smooth (every tail image is at least n0 + 1/2 away), so a coarse table
// read bilinearly is far more accurate than FP32 force arithmetic.
//
// With n_cut = 0 the window is infinite (Ncut -> infinity, Sect. 2.2): the
// table holds the whole image line beyond n0 against the infinite base.
//
// The pair kernel is the surrogate kernel with the network replaced by one
// texture fetch: the texture unit's bilinear filter is the cloud-in-cell
// read. The near images, the base, the envelope and the exact spline
// correction of softened tail images are those of surrogate_pair.cuh.
#pragma once
#include <cstdint>

#include "surrogate_pair.cuh"
#include "surrogate_train.cuh"

namespace steps {

// Node residuals in FP64 (exact point-mass tail, dz = +|dz|), stored as float2
// [ny][nx]. n_cut = 0 is the infinite window: images to |k| <= kKInf exactly
// and the line ends beyond, against the infinite base.

// A node in the table's frame: for n0 >= 1 the residual of the tail sums over
// the continuum base (BR, BZ) in envelope units (ER, EZ); for n0 = 0 (the table
// over the nearest image alone, whose base would reach the pair itself at
// |dz| = 1/2) the tail sums themselves.
__device__ __forceinline__ double2 table_node(int n0, double sr, double sz, double BR, double BZ, double ER,
                                              double EZ) {
  if (n0 == 0) return make_double2(sr, sz);
  return make_double2((sr - BR) / ER, (sz - BZ) / EZ);
}

static __global__ void tail_table_kernel(int nx, int ny, double dR_max, int n_cut, int n0, double2* __restrict__ out) {
  for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < nx * ny; q += gridDim.x * blockDim.x) {
    const int i = q % nx, j = q / nx;
    const double dR = dR_max * i / (nx - 1), adz = 0.5 * j / (ny - 1), R2 = dR * dR;
    double sr = 0.0, sz = 0.0;
    if (n_cut == 0) {
      for (int k = n0 + 1; k <= kKInf; ++k) {
        const double op = adz + (double)k, om = adz - (double)k;
        const double rp = 1.0 / sqrt(R2 + op * op), rm = 1.0 / sqrt(R2 + om * om);
        const double fp = rp * rp * rp, fm = rm * rm * rm;
        sr += fp + fm;
        sz += op * fp + om * fm;
      }
      line_ends_fp64(R2, adz, sr, sz);
      double BR, BZ, ER, EZ;
      tail_base_inf_fp64(dR, adz, n0, BR, BZ, ER, EZ);
      out[q] = table_node(n0, sr, sz, BR, BZ, ER, EZ);
      continue;
    }
    for (int k = n0 + 1; k <= n_cut + 1; ++k) {
      const double op = adz + (double)k, om = adz - (double)k;
      if (fabs(op) < (double)n_cut) {
        const double ri = 1.0 / sqrt(R2 + op * op), f = ri * ri * ri;
        sr += f;
        sz += op * f;
      }
      if (fabs(om) < (double)n_cut) {
        const double ri = 1.0 / sqrt(R2 + om * om), f = ri * ri * ri;
        sr += f;
        sz += om * f;
      }
    }
    double BR, BZ, ER, EZ;
    tail_base_fp64(dR, adz, n_cut, n0, BR, BZ, ER, EZ);
    out[q] = table_node(n0, sr, sz, BR, BZ, ER, EZ);
  }
}

// ---------------------------------------------------------------------------
// The same residuals of the infinite window from the Ewald summation of the
// line (Sect. 2.3, eqs. cylindricalEwaldSplit, EwaldRealSum, EwaldRecSum and
// the m = 0 term) instead of the direct sum, in FP64, period 1, split
// parameter alpha (1/L):
//   - real space: images |k| <= nmax, each 1/r^3 - alpha^3 E(alpha r) with
//     E(x) = [erf(x) - (2x/sqrt(pi)) exp(-x^2)] / x^3; the near images
//     |k| <= n0 are not part of the tail and keep only -alpha^3 E (finite at
//     r = 0; E from its series below x = 0.25);
//   - Fourier space: mode k = 2 pi m adds 4 cos(kz) J and 2 k sin(kz) B to the
//     sums, with J, B = Int_0^{alpha^2} exp(-rho^2 t - k^2/(4t)) (1, 1/t) dt
//     (the kernel of a line: B -> 2 K0(k rho) as alpha grows; the printed
//     eq. Bkernel is a slab's), taken in s = ln t with composite Gauss-Legendre;
//   - m = 0: 2 (1 - exp(-alpha^2 rho^2)) / rho^2.
struct EwaldRule {
  double x[8], w[8];  // Gauss-Legendre nodes and weights on [-1, 1]
};

__device__ __forceinline__ double ewald_E(double x) {
  const double c = 1.1283791670955126;  // 2 / sqrt(pi)
  if (x < 0.25) {
    // c * sum_{n>=1} (-1)^(n+1) 2n x^(2n-2) / (n! (2n+1))
    const double x2 = x * x;
    double term = 1.0, fact = 1.0, acc = 0.0;
    for (int n = 1; n <= 12; ++n) {
      fact *= (double)n;
      acc += ((n & 1) ? 2.0 : -2.0) * n * term / (fact * (2.0 * n + 1.0));
      term *= x2;
    }
    return c * acc;
  }
  return (erf(x) - c * x * exp(-x * x)) / (x * x * x);
}

// Int over s = ln t in [ln(k^2/300), ln(alpha^2)] of exp(-rho^2 e^s - k^2/(4 e^s)) (e^s for J, 1 for B)
__device__ __forceinline__ void ewald_mode(double k, double rho, double alpha, const EwaldRule& G, double& J,
                                           double& B) {
  J = 0.0;
  B = 0.0;
  const double s_hi = 2.0 * log(alpha), s_lo = log(k * k / 300.0);
  if (s_lo >= s_hi) return;
  constexpr int kPanels = 128;
  const double h = (s_hi - s_lo) / kPanels, half = 0.5 * h;
  for (int p = 0; p < kPanels; ++p) {
    const double mid = s_lo + (p + 0.5) * h;
    double pj = 0.0, pb = 0.0;
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const double t = exp(mid + half * G.x[q]);
      const double g = exp(-rho * rho * t - 0.25 * k * k / t);
      pj = fma(G.w[q], g * t, pj);
      pb = fma(G.w[q], g, pb);
    }
    J = fma(pj, half, J);
    B = fma(pb, half, B);
  }
}

static __global__ void tail_table_ewald_kernel(int nx, int ny, double dR_max, int n0, double alpha, int nmax,
                                               int mmax, EwaldRule G, double2* __restrict__ out) {
  for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < nx * ny; q += gridDim.x * blockDim.x) {
    const int i = q % nx, j = q / nx;
    const double dR = dR_max * i / (nx - 1), adz = 0.5 * j / (ny - 1), R2 = dR * dR;
    const double a3 = alpha * alpha * alpha;
    double sr = 0.0, sz = 0.0;
    for (int k = -nmax; k <= nmax; ++k) {
      const double o = adz + (double)k, r = sqrt(R2 + o * o);
      double f = -a3 * ewald_E(alpha * r);
      if (k < -n0 || k > n0) f += 1.0 / (r * r * r);
      sr += f;
      sz = fma(o, f, sz);
    }
    for (int m = 1; m <= mmax; ++m) {
      const double kk = 6.283185307179586 * m;
      double J, B;
      ewald_mode(kk, dR, alpha, G, J, B);
      sr = fma(4.0 * cos(kk * adz), J, sr);
      sz = fma(2.0 * kk * sin(kk * adz), B, sz);
    }
    const double y = alpha * alpha * R2;
    sr += y > 0.0 ? -2.0 * alpha * alpha * expm1(-y) / y : 2.0 * alpha * alpha;
    double BR, BZ, ER, EZ;
    tail_base_inf_fp64(dR, adz, n0, BR, BZ, ER, EZ);
    out[q] = table_node(n0, sr, sz, BR, BZ, ER, EZ);
  }
}

static __global__ void table_to_float_kernel(const double2* __restrict__ in, int count, float2* __restrict__ out) {
  for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < count; q += gridDim.x * blockDim.x)
    out[q] = make_float2((float)in[q].x, (float)in[q].y);
}

// Texture of the residual table and the map from the network-input scaling
// u = 2 min(dR, dR_max)/dR_max - 1, 4|dz| - 1 to texel coordinates (texel
// centres at index + 1/2): x = (u0 + 1) (nx - 1)/2 + 1/2.
// Table reads: cloud-in-cell (bilinear) or triangular-shaped cloud, each either
// through the texture unit's filter (8-bit fractional weights) or with exact
// FP32 weights on texel-centre fetches. The residual tables (n0 >= 1) take the
// filtered reads; the nearest-image table (n0 = 0), whose nodes vary far more
// between neighbours, takes the exact ones.
constexpr int kReadCic = 0, kReadTsc = 1, kReadCicExact = 2, kReadTscExact = 3;

struct TableTail {
  cudaTextureObject_t tex;
  float hx, hy;  // (nx - 1) / 2, (ny - 1) / 2
  int read;      // kReadCic .. kReadTscExact
};

// TSC along one axis, in node units x: the nearest node i and d = x - i weigh
// nodes i - 1, i, i + 1 by (1/2 - d)^2 / 2, 3/4 - d^2, (1/2 + d)^2 / 2.
__device__ __forceinline__ void tsc_weights(float x, float& i, float& wm, float& w0, float& wp) {
  i = rintf(x);
  const float d = x - i;
  wm = 0.5f * (0.5f - d) * (0.5f - d);
  w0 = 0.75f - d * d;
  wp = 0.5f * (0.5f + d) * (0.5f + d);
}

// The node (i, j) itself: a fetch at its texel centre (the edge clamp gives
// nodes beyond the table the edge value).
__device__ __forceinline__ float2 table_node_at(const TableTail& T, float i, float j) {
  return tex2D<float2>(T.tex, i + 0.5f, j + 0.5f);
}

__device__ __forceinline__ void axpy2(float w, const float2& f, float2& acc) {
  acc.x = fmaf(w, f.x, acc.x);
  acc.y = fmaf(w, f.y, acc.y);
}

// The table at inputs (u0, u1) in [-1, 1]: node coordinates (u + 1) (n - 1) / 2.
// READ: the read fixed at compile time, or -1 for T's.
template <int READ = -1>
__device__ __forceinline__ float2 table_read(const TableTail& T, float u0, float u1) {
  const int read = READ < 0 ? T.read : READ;
  if (read == kReadCic) return tex2D<float2>(T.tex, fmaf(u0, T.hx, T.hx + 0.5f), fmaf(u1, T.hy, T.hy + 0.5f));
  const float x = fminf(fmaf(u0, T.hx, T.hx), 2.0f * T.hx), y = fminf(fmaf(u1, T.hy, T.hy), 2.0f * T.hy);
  float2 acc = make_float2(0.0f, 0.0f);
  if (read == kReadCicExact) {
    const float i = fminf(floorf(x), 2.0f * T.hx - 1.0f), j = fminf(floorf(y), 2.0f * T.hy - 1.0f);
    const float a = x - i, b = y - j;
    axpy2((1.0f - a) * (1.0f - b), table_node_at(T, i, j), acc);
    axpy2(a * (1.0f - b), table_node_at(T, i + 1.0f, j), acc);
    axpy2((1.0f - a) * b, table_node_at(T, i, j + 1.0f), acc);
    axpy2(a * b, table_node_at(T, i + 1.0f, j + 1.0f), acc);
    return acc;
  }
  float ix, wx[3], iy, wy[3];
  tsc_weights(x, ix, wx[0], wx[1], wx[2]);
  tsc_weights(y, iy, wy[0], wy[1], wy[2]);
  if (read == kReadTscExact) {
#pragma unroll
    for (int q = 0; q < 3; ++q)
#pragma unroll
      for (int p = 0; p < 3; ++p) axpy2(wx[p] * wy[q], table_node_at(T, ix + (p - 1), iy + (q - 1)), acc);
    return acc;
  }
  // filtered TSC: per axis the first two weights are one linear fetch between
  // nodes i - 1 and i (weight s at i - 1 + w0 / s), the third a fetch at node i + 1
  const float sx = wx[0] + wx[1], sy = wy[0] + wy[1];
  const float ax = ix - 0.5f + __fdividef(wx[1], sx), bx = ix + 1.5f;
  const float ay = iy - 0.5f + __fdividef(wy[1], sy), by = iy + 1.5f;
  axpy2(sx * sy, tex2D<float2>(T.tex, ax, ay), acc);
  axpy2(sx * wy[2], tex2D<float2>(T.tex, ax, by), acc);
  axpy2(wx[2] * sy, tex2D<float2>(T.tex, bx, ay), acc);
  axpy2(wx[2] * wy[2], tex2D<float2>(T.tex, bx, by), acc);
  return acc;
}

// All pairs of i with the kBJ j of a (padded) tile with the table tail. S holds
// mu = 0, sc = 1 (the table stores raw residuals) and the table's dR_max. INF:
// the infinite window (n_cut = 0).
template <bool KAHAN, bool INF = false>
__device__ __forceinline__ void pair_tile_table(const IParticle& I, const float4* sA, const float4* sB, int self,
                                                int n_cut, const SurrConst& S, const TableTail& T, float& sx,
                                                float& sy, float& sz, float& cx, float& cy, float& cz) {
#pragma unroll 1
  for (int k0 = 0; k0 < kBJ; k0 += STEPS_KAHAN_GROUP) {
    float gx = 0.f, gy = 0.f, gz = 0.f;
#pragma unroll 2
    for (int k = k0; k < k0 + STEPS_KAHAN_GROUP; ++k) {
      const float4 A = sA[k];
      const float4 B = sB[k];
      float dx, dy, dz, dR2, hh;
      int kw;
      pair_geometry(I, A, B, dx, dy, dz, dR2, hh, kw);
      SurrPair P;
      surr_stage_a<INF, -1>(dR2, dz, hh, n_cut, kw, S, P);
      const float2 r = table_read(T, P.u[0], P.u[1]);
      float sr, szz;
      surr_stage_c<INF>(I, A, B, n_cut, kw, S, P, r.x, r.y, sr, szz);
      const float mj = k == self ? 0.0f : A.w;
      const float msr = mj * sr;
      gx = fmaf(dx, msr, gx);
      gy = fmaf(dy, msr, gy);
      gz = fmaf(mj, szz, gz);
    }
    acc<KAHAN>(sx, cx, gx);
    acc<KAHAN>(sy, cy, gy);
    acc<KAHAN>(sz, cz, gz);
  }
}

#ifndef STEPS_TABLE_MIN_BLOCKS
#define STEPS_TABLE_MIN_BLOCKS 6  // co-resident CTAs per SM asked of the register allocator
#endif

// Stream-K kernel with the table tail (work split and partial layout of
// pair_fp32_kernel).
template <bool KAHAN, bool INF = false>
__global__ void __launch_bounds__(kBI, STEPS_TABLE_MIN_BLOCKS)
pair_fp32_table_kernel(const float4* __restrict__ jA, const float4* __restrict__ jB, int n, int n_cut, long long U,
                       int NT, int C, TableTail T, SurrConst S, double* __restrict__ part, int b0 = 0) {
  __shared__ float4 sA[kBJ];
  __shared__ float4 sB[kBJ];
  const int c = blockIdx.x;
  const long long u0 = (long long)c * U / C;
  const long long u1 = (long long)(c + 1) * U / C;
  long long u = u0;
  while (u < u1) {
    const int lb = (int)(u / NT);
    const int b = b0 + lb;
    const int t0 = (int)(u % NT);
    const int t1 = (int)min((long long)NT, (long long)t0 + (u1 - u));
    const int i = b * kBI + threadIdx.x;
    const IParticle I = load_i(jA, jB, min(i, n - 1));
    float sx = 0.f, sy = 0.f, sz = 0.f, cx = 0.f, cy = 0.f, cz = 0.f;
    for (int t = t0; t < t1; ++t) {
      __syncthreads();
      load_tile(jA, jB, n, t, sA, sB);
      __syncthreads();
      pair_tile_table<KAHAN, INF>(I, sA, sB, i - t * kBJ, n_cut, S, T, sx, sy, sz, cx, cy, cz);
    }
    double* dst = part + ((long long)lb + c) * 3 * kBI;
    dst[threadIdx.x] = (double)sx - (KAHAN ? (double)cx : 0.0);
    dst[kBI + threadIdx.x] = (double)sy - (KAHAN ? (double)cy : 0.0);
    dst[2 * kBI + threadIdx.x] = (double)sz - (KAHAN ? (double)cz : 0.0);
    u += t1 - t0;
  }
}

// Subset kernel of the table form (acceptance checks; the layout of
// pair_fp32_subset_kernel).
template <bool KAHAN, bool INF = false>
__global__ void __launch_bounds__(kBI, STEPS_TABLE_MIN_BLOCKS)
pair_fp32_table_subset_kernel(const float4* __restrict__ jA, const float4* __restrict__ jB, int n, int n_cut,
                              const int64_t* __restrict__ idx, int ni, int tpc, TableTail T, SurrConst S,
                              double* __restrict__ part) {
  __shared__ float4 sA[kBJ];
  __shared__ float4 sB[kBJ];
  const int q = blockIdx.x * kBI + threadIdx.x;
  const int i = (int)idx[min(q, ni - 1)];
  const IParticle I = load_i(jA, jB, i);
  const int NT = (n + kBJ - 1) / kBJ;
  const int t0 = blockIdx.y * tpc, t1 = min(NT, t0 + tpc);
  float sx = 0.f, sy = 0.f, sz = 0.f, cx = 0.f, cy = 0.f, cz = 0.f;
  for (int t = t0; t < t1; ++t) {
    __syncthreads();
    load_tile(jA, jB, n, t, sA, sB);
    __syncthreads();
    pair_tile_table<KAHAN, INF>(I, sA, sB, i - t * kBJ, n_cut, S, T, sx, sy, sz, cx, cy, cz);
  }
  if (q < ni) {
    double* dst = part + (long long)blockIdx.y * 3 * ni;
    dst[q] = (double)sx - (KAHAN ? (double)cx : 0.0);
    dst[ni + q] = (double)sy - (KAHAN ? (double)cy : 0.0);
    dst[2 * ni + q] = (double)sz - (KAHAN ? (double)cz : 0.0);
  }
}

}  // namespace steps
