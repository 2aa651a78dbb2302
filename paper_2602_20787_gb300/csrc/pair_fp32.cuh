// FP32 pair kernel of the S1xR2 direct force (arXiv 2602.20787, eqs.
// Force_spline_kernel and ForceCylindrical; pair term of eq.
// ComovingEquationsOfMotionCylindrical).
//
// Layout. Positions are pre-divided by L and split into FP32 hi/lo words, so a
// pair separation keeps ~48 bits: d = (hi_i - hi_j) + (lo_i - lo_j). The period
// is then exactly 1. Per particle: jA = (x_hi, y_hi, z_hi, m), jB = (x_lo, y_lo,
// z_lo, h/L), 32 bytes.
//
// Image window. With dz wrapped into [-1/2, 1/2] (up to the lo word), the window of eq.
// ForceCylindrical (|r_z - n L| < Ncut L) is the set of offsets dz + k with
// |dz + k| < Ncut: k in [-(Ncut-1), Ncut-1] plus one edge image at
// dz - sign(dz) Ncut when dz != 0, i.e. 2 Ncut images (2 Ncut - 1 at dz = 0).
//
// Inner loop. Images are walked outward in symmetric pairs (dz + k, dz - k) held
// in one 64-bit register and processed with packed FP32x2 instructions
// (add/fma/mul .f32x2), so each image costs ~3 issue slots plus one MUFU
// rsqrt: the loop is bound by the MUFU pipe (16 rsqrt/SM/clk on sm_103).
// Walking outward keeps the offsets' relative rounding at the ulp level.
//
// Softening. With the softening law of these workloads most pairs have
// dR < h_i + h_j, so the spline of eq. Force_spline_kernel is on the main path.
// Per j the warp takes the largest number kw of image pairs that any of its
// lanes may have inside the support (|k| <= h + 1/2); those images, the centre
// and the edge image use a branch-free packed spline evaluation (one rsqrt per
// image), the remaining images a lean packed Newtonian loop. The loop bounds are
// warp-uniform, so no lane diverges.
//
// Work split (stream-K). The (i-block, j-tile) units are laid out i-block-major
// and every CTA takes an equal contiguous range of them, so all SMs get the same
// work for any N. A CTA writes one partial per i-block it touches into slot
// (i-block + CTA) of a scratch array; the finalize kernel adds the partials of
// each i in CTA order, so results are deterministic and bit-reproducible.
#pragma once
#include <cstdint>

namespace steps {

constexpr int kBI = 128;  // i per CTA (one per thread)
constexpr int kBJ = 128;  // j per shared-memory tile

// Tuning knobs (build-time; the defaults are the measured best on GB300).
#ifndef STEPS_KAHAN_GROUP
#define STEPS_KAHAN_GROUP 4   // pair forces summed plainly in groups of this many j before the Kahan update
#endif
#ifndef STEPS_SPLINE_UNROLL
#define STEPS_SPLINE_UNROLL 2 // unroll of the spline-capable image loop
#endif
constexpr int kSplineUnroll = STEPS_SPLINE_UNROLL;

typedef unsigned long long u64;

__device__ __forceinline__ u64 pk(float a, float b) {
  u64 r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
  return r;
}
__device__ __forceinline__ void upk(u64 r, float& a, float& b) {
  asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(r));
}
__device__ __forceinline__ u64 add2(u64 a, u64 b) {
  u64 r;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
  return r;
}
__device__ __forceinline__ u64 mul2(u64 a, u64 b) {
  u64 r;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
  return r;
}
__device__ __forceinline__ u64 fma2(u64 a, u64 b, u64 c) {
  u64 r;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(a), "l"(b), "l"(c));
  return r;
}
__device__ __forceinline__ float rsq(float x) {
  float y;
  asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ float rcp_approx(float x) {
  float y;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// Which CTA's range contains flattened unit p (ranges [c U / C, (c+1) U / C)).
__host__ __device__ __forceinline__ int cta_of_unit(long long p, long long U, int C) {
  return (int)(((p + 1) * (long long)C - 1) / U);
}

struct IParticle {
  float xh, yh, zh, xl, yl, zl, h;
};

// F(r,h)/r of eq. Force_spline_kernel for two images at once (packed), valid
// for every r: the inner (u < 1/2), outer (1/2 <= u < 1) and Newtonian (u >= 1)
// forms are all evaluated and the right one is selected per lane, so there is
// no branch. u = r/h with r = r^2 rsqrt(r^2); the outer branch's -1/(15 u^3)/h^3
// is -(1/15) rsqrt(r^2)^3, so one MUFU rsqrt per image is the only special
// function. r^2 is floored at 1e-30 so that a coincident pair gives a finite
// (selected inner) value.
__device__ __forceinline__ u64 spline_over_r2(u64 O, u64 DR2, u64 IH, u64 IH3) {
  const u64 R2 = fma2(O, O, DR2);
  float a, b;
  upk(R2, a, b);
  const u64 RI = pk(rsq(fmaxf(a, 1e-30f)), rsq(fmaxf(b, 1e-30f)));
  const u64 N3 = mul2(mul2(RI, RI), RI);
  const u64 U = mul2(mul2(R2, RI), IH);
  const u64 inner = mul2(fma2(mul2(U, U), fma2(U, pk(32.0f, 32.0f), pk(-38.4f, -38.4f)),
                               pk(10.6666666667f, 10.6666666667f)), IH3);
  const u64 poly = fma2(U, fma2(U, fma2(U, pk(-10.6666666667f, -10.6666666667f), pk(38.4f, 38.4f)),
                                pk(-48.0f, -48.0f)), pk(21.3333333333f, 21.3333333333f));
  const u64 outer = fma2(N3, pk(-0.0666666667f, -0.0666666667f), mul2(poly, IH3));
  float ua, ub, ia, ib, oa, ob, na, nb;
  upk(U, ua, ub);
  upk(inner, ia, ib);
  upk(outer, oa, ob);
  upk(N3, na, nb);
  return pk(ua < 0.5f ? ia : (ua < 1.0f ? oa : na), ub < 0.5f ? ib : (ub < 1.0f ? ob : nb));
}

// Image sums of one pair in units of L: sr = sum F(r)/r, sz = sum o F(r)/r over
// the 2 Ncut images of the window (2 Ncut - 1 when dz == 0).
//   kw: warp-uniform number of image pairs (dz +- k, k = 1..kw) that may lie
//       inside the softening support of some lane's pair; they, the centre
//       image and the edge image use spline_over_r2, the rest the Newtonian
//       loop (1/r^3), which is exact there because |dz +- k| >= k - 1/2 > h.
__device__ __forceinline__ void pair_images_fp32(float dR2, float dz, float hh, int n_cut, float fnc, int kw,
                                                 float& sr, float& sz) {
  const u64 DR2 = pk(dR2, dR2);
  const u64 STEP = pk(1.0f, -1.0f);
  // centre image (k = 0) and edge image (dz - sign(dz) Ncut, absent at dz == 0)
  u64 O = pk(dz, dz - copysignf(fnc, dz));
  const u64 W = pk(1.0f, dz != 0.0f ? 1.0f : 0.0f);
  u64 SR, SZ;
  int k = 1;
  if (kw >= 0) {
    // some lane of the warp has its pair inside the softening support
    const float ih = rcp_approx(hh);
    const u64 IH = pk(ih, ih);
    const float ih3 = ih * ih * ih;
    const u64 IH3 = pk(ih3, ih3);
    u64 F = mul2(spline_over_r2(O, DR2, IH, IH3), W);
    SR = F;
    SZ = mul2(O, F);
    const int kg = min(kw, n_cut - 1);
    O = pk(dz, dz);
#pragma unroll(kSplineUnroll)
    for (; k <= kg; ++k) {
      O = add2(O, STEP);
      F = spline_over_r2(O, DR2, IH, IH3);
      SR = add2(SR, F);
      SZ = fma2(O, F, SZ);
    }
  } else {
    const u64 R2 = fma2(O, O, DR2);
    float ra, rb;
    upk(R2, ra, rb);
    const u64 RI = pk(rsq(ra), rsq(rb));
    const u64 R3 = mul2(mul2(mul2(RI, RI), RI), W);
    SR = R3;
    SZ = mul2(O, R3);
    O = pk(dz, dz);
  }
  // Newtonian images
#pragma unroll 4
  for (; k < n_cut; ++k) {
    O = add2(O, STEP);
    const u64 R2 = fma2(O, O, DR2);
    float ra, rb;
    upk(R2, ra, rb);
    const u64 RI = pk(rsq(ra), rsq(rb));
    const u64 R3 = mul2(mul2(RI, RI), RI);
    SR = add2(SR, R3);
    SZ = fma2(O, R3, SZ);
  }
  float s0, s1, z0, z1;
  upk(SR, s0, s1);
  upk(SZ, z0, z1);
  sr = s0 + s1;
  sz = z0 + z1;
}

template <bool KAHAN>
__device__ __forceinline__ void acc(float& s, float& c, float v) {
  if (KAHAN) {
    const float y = __fsub_rn(v, c);
    const float t = __fadd_rn(s, y);
    c = __fsub_rn(__fsub_rn(t, s), y);
    s = t;
  } else {
    s += v;
  }
}

// part layout: [slot][3][kBI] doubles, slot = i-block + CTA.
template <bool KAHAN>
__global__ void __launch_bounds__(kBI, 8)
pair_fp32_kernel(const float4* __restrict__ jA, const float4* __restrict__ jB, int n, int n_cut,
                 long long U, int NT, int C, double* __restrict__ part) {
  __shared__ float4 sA[kBJ];
  __shared__ float4 sB[kBJ];
  const int c = blockIdx.x;
  const long long u0 = (long long)c * U / C;
  const long long u1 = (long long)(c + 1) * U / C;
  const float fnc = (float)n_cut;
  long long u = u0;
  while (u < u1) {
    const int b = (int)(u / NT);
    const int t0 = (int)(u % NT);
    const long long rem = u1 - u;
    const int t1 = (int)min((long long)NT, (long long)t0 + rem);
    const int i = b * kBI + threadIdx.x;
    IParticle I;
    {
      const float4 a = jA[min(i, n - 1)];
      const float4 q = jB[min(i, n - 1)];
      I.xh = a.x; I.yh = a.y; I.zh = a.z; I.xl = q.x; I.yl = q.y; I.zl = q.z; I.h = q.w;
    }
    float sx = 0.f, sy = 0.f, sz = 0.f, cx = 0.f, cy = 0.f, cz = 0.f;
    for (int t = t0; t < t1; ++t) {
      __syncthreads();
      const int jl = t * kBJ + threadIdx.x;
      if (jl < n) {
        sA[threadIdx.x] = jA[jl];
        sB[threadIdx.x] = jB[jl];
      }
      __syncthreads();
      const int jn = min(kBJ, n - t * kBJ);
      const int self = i - t * kBJ;  // local index of the self pair in this tile, if any
      // pair forces are summed plainly over groups of STEPS_KAHAN_GROUP j, and
      // each group sum enters the compensated per-i sum
      for (int k0 = 0; k0 < jn; k0 += STEPS_KAHAN_GROUP) {
        float gx = 0.f, gy = 0.f, gz = 0.f;
        const int ke = min(k0 + STEPS_KAHAN_GROUP, jn);
        for (int k = k0; k < ke; ++k) {
          const float4 A = sA[k];
          const float4 B = sB[k];
          const float dx = (I.xh - A.x) + (I.xl - B.x);
          const float dy = (I.yh - A.y) + (I.yl - B.y);
          // wrap the hi difference before adding the lo words, so a separation
          // just below L keeps its small wrapped value (the window edge depends
          // on the sign of dz)
          float dz = I.zh - A.z;
          dz = (dz - rintf(dz)) + (I.zl - B.z);
          const float dR2 = fmaf(dx, dx, dy * dy);
          const float hh = I.h + B.w;
          // images with |k| <= hh + 1/2 can be inside the support when dR < hh;
          // kw = -1: no lane's pair is softened, every image is Newtonian
          const int kl = dR2 < hh * hh ? (int)(hh + 0.5f) : -1;
          const int kw = __reduce_max_sync(0xffffffffu, kl);
          float sr, szz;
          pair_images_fp32(dR2, dz, hh, n_cut, fnc, kw, sr, szz);
          const float mj = (k == self) ? 0.0f : A.w;
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
    const long long slot = (long long)b + c;
    double* dst = part + slot * 3 * kBI;
    dst[threadIdx.x] = (double)sx + (double)cx * (KAHAN ? -1.0 : 0.0);
    dst[kBI + threadIdx.x] = (double)sy + (double)cy * (KAHAN ? -1.0 : 0.0);
    dst[2 * kBI + threadIdx.x] = (double)sz + (double)cz * (KAHAN ? -1.0 : 0.0);
    u += t1 - t0;
  }
}

}  // namespace steps
