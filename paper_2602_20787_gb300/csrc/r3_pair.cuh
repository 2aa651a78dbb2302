// FP32 pair kernel of the R^3 topology (arXiv 2602.20787, Sect. 2.1, eq.
// NewtonianForce): the softened Newtonian pair force, one image per pair.
//
// With one image per pair, the per-pair work is the whole cost. Two j share every
// packed FP32x2 operation: the shared-memory tile stores j pairs interleaved,
// so one 128-bit load yields the packed (j0, j1) operands directly:
//   H[s] = (x_hi, y_hi) of j = 2s, 2s+1 as two packed pairs,
//   Lo[s] = (x_lo, y_lo), Z[s] = (z_hi, z_lo), MH[s] = (m, h/L).
// F(r^2, h_i + h_j)/r depends on the symmetric r^2 and softening sum only, so a
// pair and its reverse stay exactly antisymmetric. The spline runs only when some
// lane of the warp has one of its two j inside the softening support (the
// three-branch select of spline_value_r2); the self pair (r = 0) always takes it
// and gives the finite centre. The stream-K split and the partial layout are
// those of pair_fp32_kernel.
#pragma once
#include <cstdint>

#include "pair_fp32.cuh"

namespace steps {

#ifndef STEPS_R3_GROUP
#define STEPS_R3_GROUP 16  // j per plain FP32 group before the compensated update
#endif
static_assert(kBJ % STEPS_R3_GROUP == 0 && STEPS_R3_GROUP % 2 == 0, "whole groups of j pairs per tile");

struct R3Tile {
  ulonglong2 H[kBJ / 2], Lo[kBJ / 2], Z[kBJ / 2], MH[kBJ / 2];
};

// Tile t of the packed j-set into the interleaved layout (padded with massless
// far particles, as load_tile).
__device__ __forceinline__ void load_tile_r3(const float4* __restrict__ jA, const float4* __restrict__ jB, int n,
                                             int t, R3Tile& T) {
  const int jl = t * kBJ + threadIdx.x;
  float4 a = make_float4(4096.0f, 4096.0f, 0.0f, 0.0f), b = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
  if (jl < n) {
    a = jA[jl];
    b = jB[jl];
  }
  const int s = threadIdx.x >> 1, p = threadIdx.x & 1;
  float* h = reinterpret_cast<float*>(&T.H[s]);
  float* l = reinterpret_cast<float*>(&T.Lo[s]);
  float* z = reinterpret_cast<float*>(&T.Z[s]);
  float* mh = reinterpret_cast<float*>(&T.MH[s]);
  h[p] = a.x;
  h[2 + p] = a.y;
  l[p] = b.x;
  l[2 + p] = b.y;
  z[p] = a.z;
  z[2 + p] = b.z;
  mh[p] = a.w;
  mh[2 + p] = b.w;
}

template <bool KAHAN>
__device__ __forceinline__ void pair_tile_r3(const IParticle& I, const R3Tile& T, float& sx, float& sy, float& sz,
                                             float& cx, float& cy, float& cz) {
  float xh, yh, xl, yl;
  upk(I.xyh, xh, yh);
  upk(I.xyl, xl, yl);
  const u64 XH = pk(xh, xh), YH = pk(yh, yh), ZH = pk(I.zh, I.zh);
  const u64 XL = pk(xl, xl), YL = pk(yl, yl), ZL = pk(I.zl, I.zl);
  const u64 HI = pk(I.h, I.h);
#pragma unroll 1
  for (int s0 = 0; s0 < kBJ / 2; s0 += STEPS_R3_GROUP / 2) {
    u64 GX = pk(0.f, 0.f), GY = pk(0.f, 0.f), GZ = pk(0.f, 0.f);
#pragma unroll 2
    for (int s = s0; s < s0 + STEPS_R3_GROUP / 2; ++s) {
      const ulonglong2 h = T.H[s], l = T.Lo[s], z = T.Z[s], mh = T.MH[s];
      const u64 DX = add2(sub2(XH, h.x), sub2(XL, l.x));
      const u64 DY = add2(sub2(YH, h.y), sub2(YL, l.y));
      const u64 DZ = add2(sub2(ZH, z.x), sub2(ZL, z.y));
      const u64 R2 = fma2(DX, DX, fma2(DY, DY, mul2(DZ, DZ)));
      const u64 HH = add2(HI, mh.y);
      float ra, rb, ha, hb;
      upk(R2, ra, rb);
      upk(HH, ha, hb);
      const u64 RI = pk(rsq(fmaxf(ra, 1e-30f)), rsq(fmaxf(rb, 1e-30f)));
      u64 F = mul2(mul2(RI, RI), RI);
      if (__any_sync(0xffffffffu, ra < ha * ha || rb < hb * hb)) {
        const float iha = rcp_approx(ha), ihb = rcp_approx(hb);
        const u64 IH = pk(iha, ihb);
        F = spline_value_r2(R2, RI, F, IH, pk(-iha, -ihb), mul2(mul2(IH, IH), IH));
      }
      const u64 MF = mul2(mh.x, F);
      GX = fma2(DX, MF, GX);
      GY = fma2(DY, MF, GY);
      GZ = fma2(DZ, MF, GZ);
    }
    float a, b;
    upk(GX, a, b);
    acc<KAHAN>(sx, cx, a + b);
    upk(GY, a, b);
    acc<KAHAN>(sy, cy, a + b);
    upk(GZ, a, b);
    acc<KAHAN>(sz, cz, a + b);
  }
}

// part layout: [slot][3][kBI] doubles, slot = i-block + CTA (as pair_fp32_kernel).
template <bool KAHAN>
__global__ void __launch_bounds__(kBI, 8)
pair_r3_kernel(const float4* __restrict__ jA, const float4* __restrict__ jB, int n, long long U, int NT, int C,
               double* __restrict__ part, int b0 = 0) {
  __shared__ R3Tile T;
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
      load_tile_r3(jA, jB, n, t, T);
      __syncthreads();
      pair_tile_r3<KAHAN>(I, T, sx, sy, sz, cx, cy, cz);
    }
    double* dst = part + ((long long)lb + c) * 3 * kBI;
    dst[threadIdx.x] = (double)sx - (KAHAN ? (double)cx : 0.0);
    dst[kBI + threadIdx.x] = (double)sy - (KAHAN ? (double)cy : 0.0);
    dst[2 * kBI + threadIdx.x] = (double)sz - (KAHAN ? (double)cz : 0.0);
    u += t1 - t0;
  }
}

}  // namespace steps
