// Training side of the learned far-image surrogate (this project's method; the
// paper sums the image tail directly, eq. ForceCylindrical).
//
// The tail of a pair is the part of the image window of eq. ForceCylindrical
// beyond the near images |k| <= n0 (wrapped frame, lengths in units of L). The
// surrogate writes it as
//   tail = B1 + E * (MLP(u) * sc + mu)            (z component times sign(dz))
// with B1 the continuum integral of the image cells plus the first
// Euler-Maclaurin end correction, E an envelope (e^3 for SR, e^(5/2) for SZ,
// e = 1 / (dR^2 + (n0 + 1/2 + |dz|)^2)), and a 3 -> 32 -> 32 -> 2 ReLU MLP of
// u = (2 min(dR, dR_max)/dR_max - 1, 4|dz| - 1, 2 min(h, n0+1/2)/(n0+1/2) - 1).
//
// Kernels here: exact FP64 tail sums (training targets), the FP64 base and
// envelope, and FP32 forward/backward/Adam. Gradients are accumulated per block
// and reduced in block order, so training is deterministic.
#pragma once
#include <cstdint>

namespace steps {

constexpr int kH = 32;                                   // hidden width
constexpr int kNW = kH * 3 + kH + kH * kH + kH + 2 * kH + 2;  // 1250 weights
// offsets in the flat weight vector: W1[32][3], b1[32], W2[32][32], b2[32], W3[2][32], b3[2]
constexpr int kOW1 = 0, kOB1 = kOW1 + kH * 3, kOW2 = kOB1 + kH, kOB2 = kOW2 + kH * kH, kOW3 = kOB2 + kH,
              kOB3 = kOW3 + 2 * kH;

// Spline F(r,h)/r of eq. Force_spline_kernel in FP64 (support radius h).
__device__ __forceinline__ double spline_over_r_d(double r, double h) {
  if (r >= h) return 1.0 / (r * r * r);
  const double u = r / h, ih3 = 1.0 / (h * h * h);
  if (u < 0.5) return (32.0 / 3.0 + u * u * (32.0 * u - 38.4)) * ih3;
  const double u3 = u * u * u;
  return (64.0 / 3.0 - 48.0 * u + 38.4 * u * u - (32.0 / 3.0) * u3 - 1.0 / (15.0 * u3)) * ih3;
}

// The infinite window (Ncut -> infinity): images |k| <= kKInf are summed one by
// one, those beyond on each side by the continuum cells from kKInf + 1/2 with
// the near end's Euler-Maclaurin term (Newtonian there, as h << kKInf), which
// leaves an error of O(kKInf^-6).
constexpr int kKInf = 512;

// Both line ends beyond |k| = kKInf, added to (sr, sz), offsets o = dz + k.
__host__ __device__ __forceinline__ void line_ends_fp64(double R2, double dz, double& sr, double& sz) {
  const double top = kKInf + 0.5 + dz, bot = kKInf + 0.5 - dz;
  const double rt = sqrt(R2 + top * top), rb = sqrt(R2 + bot * bot), it = 1.0 / rt, ib = 1.0 / rb;
  const double it5 = it * it * it * it * it, ib5 = ib * ib * ib * ib * ib;
  sr += 1.0 / (rt * (rt + top)) - 3.0 * top * it5 / 24.0 + 1.0 / (rb * (rb + bot)) - 3.0 * bot * ib5 / 24.0;
  sz += it + (it * it * it - 3.0 * top * top * it5) / 24.0 - (ib + (ib * ib * ib - 3.0 * bot * bot * ib5) / 24.0);
}

// Exact tail sums of the window (|dz + k| < Ncut, |k| > n0) in FP64, units of L;
// n_cut = 0 is the infinite window.
// samples: ns x 3 (dR, dz, h); out: ns x 2 (SR, SZ).
static __global__ void tail_sums_fp64_kernel(const double* __restrict__ smp, int64_t ns, int n_cut, int n0,
                                             double* __restrict__ out) {
  for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < ns; s += (int64_t)gridDim.x * blockDim.x) {
    const double dR = smp[3 * s], dz = smp[3 * s + 1], h = smp[3 * s + 2];
    const double R2 = dR * dR;
    double sr = 0.0, sz = 0.0;
    if (n_cut == 0) {
      for (int k = n0 + 1; k <= kKInf; ++k) {
        const double op = dz + (double)k, om = dz - (double)k;
        const double fp = spline_over_r_d(sqrt(R2 + op * op), h), fm = spline_over_r_d(sqrt(R2 + om * om), h);
        sr += fp + fm;
        sz += op * fp + om * fm;
      }
      line_ends_fp64(R2, dz, sr, sz);
      out[2 * s] = sr;
      out[2 * s + 1] = sz;
      continue;
    }
    // walk outward from the near region on both sides
    for (int k = n0 + 1; k <= n_cut + 1; ++k) {
      const double op = dz + (double)k, om = dz - (double)k;
      if (fabs(op) < (double)n_cut) {
        const double f = spline_over_r_d(sqrt(R2 + op * op), h);
        sr += f;
        sz += op * f;
      }
      if (fabs(om) < (double)n_cut) {
        const double f = spline_over_r_d(sqrt(R2 + om * om), h);
        sr += f;
        sz += om * f;
      }
    }
    out[2 * s] = sr;
    out[2 * s + 1] = sz;
  }
}

// Continuum base B1 of one side: cells [lo, hi] of the unit-spaced images,
// f = (R^2 + z^2)^(-3/2) for SR and z f for SZ.
__host__ __device__ __forceinline__ void side_base_fp64(double R2, double lo, double hi, double& sr, double& sz) {
  const double rl = sqrt(R2 + lo * lo), rh = sqrt(R2 + hi * hi);
  const double il = 1.0 / rl, ih = 1.0 / rh;
  // Int f = (hi^2 - lo^2) / (rl rh (hi rl + lo rh)) (no cancellation at small R)
  const double IR = (hi - lo) * (hi + lo) / (rl * rh * (hi * rl + lo * rh));
  const double IZ = il - ih;
  const double il2 = il * il, ih2 = ih * ih, il5 = il2 * il2 * il, ih5 = ih2 * ih2 * ih;
  const double dRl = -3.0 * lo * il5, dRh = -3.0 * hi * ih5;
  const double dZl = il2 * il - 3.0 * lo * lo * il5, dZh = ih2 * ih - 3.0 * hi * hi * ih5;
  sr = IR - (dRh - dRl) / 24.0;
  sz = IZ - (dZh - dZl) / 24.0;
}

// B1 and the envelope for |dz| = adz (z component for positive dz).
__host__ __device__ __forceinline__ void tail_base_fp64(double dR, double adz, int n_cut, int n0, double& BR,
                                                        double& BZ, double& ER, double& EZ) {
  const double R2 = dR * dR, A = n0 + 0.5;
  const int kpos = n_cut - 1, kneg = adz > 0.0 ? n_cut : n_cut - 1;
  double r1, z1, r2, z2;
  side_base_fp64(R2, A + adz, kpos + 0.5 + adz, r1, z1);
  side_base_fp64(R2, A - adz, kneg + 0.5 - adz, r2, z2);
  BR = r1 + r2;
  BZ = z1 - z2;
  const double e = 1.0 / (R2 + (A + adz) * (A + adz));
  ER = e * e * e;
  EZ = e * e * sqrt(e);
}

// The same base with both far ends at infinity (the Ncut -> infinity window):
// per side the integral over [A +- |dz|, inf) plus the near end's
// Euler-Maclaurin term, Int = 1/(r (r + lo)) and 1/r.
__host__ __device__ __forceinline__ void tail_base_inf_fp64(double dR, double adz, int n0, double& BR, double& BZ,
                                                            double& ER, double& EZ) {
  const double R2 = dR * dR, A = n0 + 0.5;
  double br[2], bz[2];
  const double lo[2] = {A + adz, A - adz};
  for (int q = 0; q < 2; ++q) {
    const double l = lo[q], r = sqrt(R2 + l * l), il = 1.0 / r, il2 = il * il, il5 = il2 * il2 * il;
    br[q] = 1.0 / (r * (r + l)) - 3.0 * l * il5 / 24.0;
    bz[q] = il + (il2 * il - 3.0 * l * l * il5) / 24.0;
  }
  BR = br[0] + br[1];
  BZ = bz[0] - bz[1];
  const double e = 1.0 / (R2 + (A + adz) * (A + adz));
  ER = e * e * e;
  EZ = e * e * sqrt(e);
}

// Training pairs: inputs u (FP32, ns x 3) and raw targets r = (tail - B1) / E
// (FP64, ns x 2, before the mean/scale normalisation) from exact tail sums
// (n_cut = 0: the infinite window over its base).
static __global__ void surrogate_dataset_kernel(const double* __restrict__ smp, const double* __restrict__ tail,
                                                int64_t ns, int n_cut, int n0, double dR_max,
                                                float* __restrict__ u, double* __restrict__ r) {
  for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < ns; s += (int64_t)gridDim.x * blockDim.x) {
    const double dR = smp[3 * s], adz = fabs(smp[3 * s + 1]), h = smp[3 * s + 2];
    double BR, BZ, ER, EZ;
    if (n_cut == 0)
      tail_base_inf_fp64(dR, adz, n0, BR, BZ, ER, EZ);
    else
      tail_base_fp64(dR, adz, n_cut, n0, BR, BZ, ER, EZ);
    const double A = n0 + 0.5;
    u[3 * s] = (float)(2.0 * fmin(dR, dR_max) / dR_max - 1.0);
    u[3 * s + 1] = (float)(4.0 * adz - 1.0);
    u[3 * s + 2] = (float)(2.0 * fmin(h, A) / A - 1.0);
    const double sg = smp[3 * s + 1] < 0.0 ? -1.0 : 1.0;
    r[2 * s] = (tail[2 * s] - BR) / ER;
    r[2 * s + 1] = (sg * tail[2 * s + 1] - BZ) / EZ;
  }
}

// ---------------------------------------------------------------------------
// FP32 MLP training. One block of kTrainThreads threads takes kTrainThreads
// samples of the minibatch; each thread runs its sample forward and backward,
// the block forms its partial gradient from the per-sample activations and
// deltas staged in shared memory, and writes it to gpart[block][kNW].
// ---------------------------------------------------------------------------
constexpr int kTrainThreads = 64;

static __global__ void __launch_bounds__(kTrainThreads)
mlp_fwd_bwd_kernel(const float* __restrict__ w, const float* __restrict__ u, const float* __restrict__ t,
                   const int* __restrict__ order, int64_t first, int64_t count, float* __restrict__ gpart,
                   float* __restrict__ lpart) {
  __shared__ float s_in[kTrainThreads][4];
  __shared__ float s_a1[kTrainThreads][kH + 1];
  __shared__ float s_d1[kTrainThreads][kH + 1];
  __shared__ float s_a2[kTrainThreads][kH + 1];
  __shared__ float s_d2[kTrainThreads][kH + 1];
  __shared__ float s_e[kTrainThreads][2];
  __shared__ float s_loss[kTrainThreads];
  const int tid = threadIdx.x;
  const int64_t q = (int64_t)blockIdx.x * kTrainThreads + tid;
  const bool valid = q < count;
  const float* W1 = w + kOW1;
  const float* b1 = w + kOB1;
  const float* W2 = w + kOW2;
  const float* b2 = w + kOB2;
  const float* W3 = w + kOW3;
  const float* b3 = w + kOB3;
  float in[3] = {0.f, 0.f, 0.f}, tg[2] = {0.f, 0.f};
  if (valid) {
    const int64_t s = order ? (int64_t)order[first + q] : first + q;
    for (int k = 0; k < 3; ++k) in[k] = u[3 * s + k];
    tg[0] = t[2 * s];
    tg[1] = t[2 * s + 1];
  }
  // forward; ReLU'(z) is read from a = relu(z) > 0 (the same mask)
  float a1[kH], a2[kH];
#pragma unroll
  for (int o = 0; o < kH; ++o) {
    float v = b1[o];
#pragma unroll
    for (int k = 0; k < 3; ++k) v = fmaf(W1[o * 3 + k], in[k], v);
    a1[o] = fmaxf(v, 0.f);
    s_a1[tid][o] = a1[o];
  }
#pragma unroll
  for (int o = 0; o < kH; ++o) {
    float v = b2[o];
#pragma unroll
    for (int k = 0; k < kH; ++k) v = fmaf(W2[o * kH + k], a1[k], v);
    a2[o] = fmaxf(v, 0.f);
  }
  float y[2], e[2];
#pragma unroll
  for (int o = 0; o < 2; ++o) {
    float v = b3[o];
#pragma unroll
    for (int k = 0; k < kH; ++k) v = fmaf(W3[o * kH + k], a2[k], v);
    y[o] = v;
    e[o] = valid ? (y[o] - tg[o]) : 0.f;
  }
  // backward: d2 = (W3^T e) * relu'(z2), d1 = (W2^T d2) * relu'(z1)
  float d2[kH];
#pragma unroll
  for (int k = 0; k < kH; ++k) {
    const float g = W3[k] * e[0] + W3[kH + k] * e[1];
    d2[k] = a2[k] > 0.f ? g : 0.f;
    s_a2[tid][k] = a2[k];
    s_d2[tid][k] = d2[k];
  }
  for (int k = 0; k < kH; ++k) {
    float g = 0.f;
#pragma unroll
    for (int o = 0; o < kH; ++o) g = fmaf(W2[o * kH + k], d2[o], g);
    s_d1[tid][k] = s_a1[tid][k] > 0.f ? g : 0.f;
  }
  for (int k = 0; k < 3; ++k) s_in[tid][k] = in[k];
  s_e[tid][0] = e[0];
  s_e[tid][1] = e[1];
  s_loss[tid] = 0.5f * (e[0] * e[0] + e[1] * e[1]);
  __syncthreads();
  // block partial gradient, one weight per thread per pass, samples in order
  float* gp = gpart + (int64_t)blockIdx.x * kNW;
  for (int p = tid; p < kNW; p += kTrainThreads) {
    float g = 0.f;
    if (p < kOB1) {
      const int o = p / 3, k = p % 3;
      for (int s = 0; s < kTrainThreads; ++s) g = fmaf(s_d1[s][o], s_in[s][k], g);
    } else if (p < kOW2) {
      const int o = p - kOB1;
      for (int s = 0; s < kTrainThreads; ++s) g += s_d1[s][o];
    } else if (p < kOB2) {
      const int o = (p - kOW2) / kH, k = (p - kOW2) % kH;
      for (int s = 0; s < kTrainThreads; ++s) g = fmaf(s_d2[s][o], s_a1[s][k], g);
    } else if (p < kOW3) {
      const int o = p - kOB2;
      for (int s = 0; s < kTrainThreads; ++s) g += s_d2[s][o];
    } else if (p < kOB3) {
      const int o = (p - kOW3) / kH, k = (p - kOW3) % kH;
      for (int s = 0; s < kTrainThreads; ++s) g = fmaf(s_e[s][o], s_a2[s][k], g);
    } else {
      const int o = p - kOB3;
      for (int s = 0; s < kTrainThreads; ++s) g += s_e[s][o];
    }
    gp[p] = g;
  }
  if (tid == 0) {
    float l = 0.f;
    for (int s = 0; s < kTrainThreads; ++s) l += s_loss[s];
    lpart[blockIdx.x] = l;
  }
}

// Sum the block partials of each weight in block order, divide by the batch,
// and (when adam) take an Adam step. grad_out (optional) receives the gradient.
static __global__ void mlp_reduce_adam_kernel(const float* __restrict__ gpart, int nblocks, float inv_batch,
                                              float* __restrict__ w, float* __restrict__ m1, float* __restrict__ m2,
                                              float lr, float beta1, float beta2, float eps, float c1, float c2,
                                              int adam, float* __restrict__ grad_out) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= kNW) return;
  float g = 0.f;
  for (int b = 0; b < nblocks; ++b) g += gpart[(int64_t)b * kNW + p];
  g *= inv_batch;
  if (grad_out) grad_out[p] = g;
  if (adam) {
    const float a = beta1 * m1[p] + (1.f - beta1) * g;
    const float v = beta2 * m2[p] + (1.f - beta2) * g * g;
    m1[p] = a;
    m2[p] = v;
    w[p] -= lr * (a / c1) / (sqrtf(v / c2) + eps);
  }
}

static __global__ void sum_floats_kernel(const float* __restrict__ x, int n, float scale, float* __restrict__ out) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    float s = 0.f;
    for (int i = 0; i < n; ++i) s += x[i];
    *out = s * scale;
  }
}

}  // namespace steps
