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
// lanes may have inside the support (|k| < h + 1/2). Of those, the few that
// may reach the inner core (u < 1/2) on some lane use a branch-free packed
// evaluation of all three spline branches; the others lie in the outer shell
// or beyond on every lane and use the cheaper factored outer form; the
// remaining images a lean packed Newtonian loop. Each costs one rsqrt per
// image, and all loop bounds are warp-uniform, so no lane diverges.
//
// Per-pair overhead. Everything outside the image loop is issue slots taken
// from the FP32 pipes the MUFU leaves free, and the MUFU itself takes only the
// image rsqrts and one rcp: the wrap of dz and the softening bound are
// integer-valued roundings done with a 2^23 magic constant on the FMA pipe
// (no F2I/FRND), x and y go through packed FP32x2, and the j-tile is padded to
// kBJ with massless far particles so the j loop has a constant trip count and
// no guard. The self pair needs no test: it has dx = dy = 0, a finite spline
// centre and an image walk symmetric in +-k, so it adds exact zeros.
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
#define STEPS_KAHAN_GROUP 8   // pair forces summed plainly in groups of this many j before the Kahan update
#endif
#ifndef STEPS_SPLINE_UNROLL
#define STEPS_SPLINE_UNROLL 2 // unroll of the spline-capable image loop
#endif
constexpr int kSplineUnroll = STEPS_SPLINE_UNROLL;
#ifndef STEPS_NCUT_FIXED
#define STEPS_NCUT_FIXED 1    // compile the windows N_cut = 16 and 64 unrolled beside the general one
#endif
#ifndef STEPS_PLAIN_MIN_BLOCKS
#define STEPS_PLAIN_MIN_BLOCKS 8  // resident CTAs per SM the plain kernels are compiled for (registers)
#endif

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
__device__ __forceinline__ u64 sub2(u64 a, u64 b) {
  u64 r;
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
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

// The i-particle of a thread: (x, y) hi and lo words as packed pairs.
struct IParticle {
  u64 xyh, xyl;
  float zh, zl, h;
};

__device__ __forceinline__ IParticle load_i(const float4* __restrict__ jA, const float4* __restrict__ jB, int i) {
  const float4 a = jA[i];
  const float4 q = jB[i];
  IParticle I;
  I.xyh = pk(a.x, a.y);
  I.xyl = pk(q.x, q.y);
  I.zh = a.z;
  I.zl = q.z;
  I.h = q.w;
  return I;
}

// j-tile t into shared memory; slots past n get a massless particle far off
// the axis (zero softening), whose pairs are finite and add exact zeros.
__device__ __forceinline__ void load_tile(const float4* __restrict__ jA, const float4* __restrict__ jB, int n, int t,
                                          float4* sA, float4* sB) {
  const int jl = t * kBJ + threadIdx.x;
  if (jl < n) {
    sA[threadIdx.x] = jA[jl];
    sB[threadIdx.x] = jB[jl];
  } else {
    sA[threadIdx.x] = make_float4(4096.0f, 4096.0f, 0.0f, 0.0f);
    sB[threadIdx.x] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
  }
}

constexpr float kRound23 = 12582912.0f;  // 1.5 * 2^23: x + c - c rounds |x| < 2^22 to an integer
constexpr float kTwo23 = 8388608.0f;     // 2^23: bits(2^23 + x) - bits(2^23) = rn(x) for 0 <= x < 2^23
constexpr int kTwo23Bits = 0x4B000000;

// Geometry of the pair (i, j) in units of L: separation (dx, dy, dz) with dz
// wrapped into [-1/2, 1/2] (hi words wrapped before the lo words are added, so
// a separation just below L keeps its small wrapped value), dR^2 = dx^2 + dy^2,
// hh = h_i + h_j, and the warp-uniform bound kw on the image pairs +-k that may
// lie inside the softening support. An image k has |dz + k| >= |k| - 1/2, so it
// can be inside only if dR < hh and |k| < hh + 1/2; rn(hh) is an upper bound
// of that largest |k|, and kw is its maximum over the warp (-1: no lane's pair
// is softened). Both roundings are exact integer-valued FP32 additions.
__device__ __forceinline__ void pair_separation(const IParticle& I, const float4& A, const float4& B, float& dx,
                                                float& dy, float& dz, float& dR2, float& hh) {
  const u64 D = add2(sub2(I.xyh, pk(A.x, A.y)), sub2(I.xyl, pk(B.x, B.y)));
  upk(D, dx, dy);
  dR2 = fmaf(dx, dx, dy * dy);
  const float d = I.zh - A.z;
  dz = (d - __fsub_rn(__fadd_rn(d, kRound23), kRound23)) + (I.zl - B.z);
  hh = I.h + B.w;
}
__device__ __forceinline__ void pair_geometry(const IParticle& I, const float4& A, const float4& B, float& dx, float& dy,
                                              float& dz, float& dR2, float& hh, int& kw) {
  pair_separation(I, A, B, dx, dy, dz, dR2, hh);
  const int kl = dR2 < hh * hh ? __float_as_int(__fadd_rn(hh, kTwo23)) : kTwo23Bits - 1;
  kw = __reduce_max_sync(0xffffffffu, kl) - kTwo23Bits;
}

// F(r,h)/r of eq. Force_spline_kernel, packed over two images, in the form
// used wherever u = r/h >= 1/2 may hold: the M4 enclosed-mass fraction of the
// outer shell factored about u = 1 is 1 - V^4 (16 - 25.6 V + (32/3) V^2) with
// V = max(0, 1 - u), so F/r = r^-3 (1 - V^4 R(V)), and V = 0 makes it exactly
// r^-3 for u >= 1. RR = r (= r^2 rsqrt(r^2)), N3 = r^-3, NIH = (-1/h, -1/h).
__device__ __forceinline__ u64 spline_outer_value(u64 RR, u64 N3, u64 NIH) {
  float va, vb;
  upk(fma2(RR, NIH, pk(1.0f, 1.0f)), va, vb);
  const u64 V = pk(fmaxf(va, 0.0f), fmaxf(vb, 0.0f));
  const u64 V2 = mul2(V, V);
  const u64 NR = fma2(fma2(V, pk(-10.6666666667f, -10.6666666667f), pk(25.6f, 25.6f)), V, pk(-16.0f, -16.0f));
  return mul2(N3, fma2(mul2(V2, V2), NR, pk(1.0f, 1.0f)));
}

// Every image's F/r is a function of (r^2, h) alone, whichever of the three
// evaluations below computes it: the inner polynomial where u < 1/2, else
// spline_outer_value (which is r^-3 for u >= 1). So a pair and its reverse,
// evaluated by different warps with different tiers, get bit-identical image
// values, and the pair forces stay exactly antisymmetric.

// All branches, for images that may have u < 1/2 on some lane. The inner
// branch is h^-3 (32/3 - 38.4 u^2 + 32 u^3), selected per lane. r^2 is floored
// at 1e-30 so that a coincident pair gives a finite inner value.
// The select itself, from r^2, its floored rsqrt RI and r^-3 = RI^3 (also the
// R^3 kernel's softened branch).
__device__ __forceinline__ u64 spline_value_r2(u64 R2, u64 RI, u64 N3, u64 IH, u64 NIH, u64 IH3) {
  const u64 RR = mul2(R2, RI);
  const u64 U = mul2(RR, IH);
  const u64 inner = mul2(fma2(mul2(U, U), fma2(U, pk(32.0f, 32.0f), pk(-38.4f, -38.4f)),
                               pk(10.6666666667f, 10.6666666667f)), IH3);
  const u64 outer = spline_outer_value(RR, N3, NIH);
  float ua, ub, ia, ib, oa, ob;
  upk(U, ua, ub);
  upk(inner, ia, ib);
  upk(outer, oa, ob);
  return pk(ua < 0.5f ? ia : oa, ub < 0.5f ? ib : ob);
}

__device__ __forceinline__ u64 spline_over_r2(u64 O, u64 DR2, u64 IH, u64 NIH, u64 IH3) {
  const u64 R2 = fma2(O, O, DR2);
  float a, b;
  upk(R2, a, b);
  const u64 RI = pk(rsq(fmaxf(a, 1e-30f)), rsq(fmaxf(b, 1e-30f)));
  return spline_value_r2(R2, RI, mul2(mul2(RI, RI), RI), IH, NIH, IH3);
}

// Images with u >= 1/2 on every lane (outer shell or beyond): no select.
__device__ __forceinline__ u64 spline_outer_over_r2(u64 O, u64 DR2, u64 NIH) {
  const u64 R2 = fma2(O, O, DR2);
  float a, b;
  upk(R2, a, b);
  const u64 RI = pk(rsq(fmaxf(a, 1e-30f)), rsq(fmaxf(b, 1e-30f)));
  const u64 N3 = mul2(mul2(RI, RI), RI);
  return spline_outer_value(mul2(R2, RI), N3, NIH);
}

// The next Newtonian image pair (O + (1, -1)): 1/r^3 into SR, o/r^3 into SZ.
__device__ __forceinline__ void newton_pair(u64& O, u64 STEP, u64 DR2, u64& SR, u64& SZ) {
  O = add2(O, STEP);
  const u64 R2 = fma2(O, O, DR2);
  float ra, rb;
  upk(R2, ra, rb);
  const u64 RI = pk(rsq(ra), rsq(rb));
  const u64 R3 = mul2(mul2(RI, RI), RI);
  SR = add2(SR, R3);
  SZ = fma2(O, R3, SZ);
}

// Image sums of one pair in units of L: sr = sum F(r)/r, sz = sum o F(r)/r over
// the 2 Ncut images of the window (2 Ncut - 1 when dz == 0).
//   kw: warp-uniform number of image pairs (dz +- k, k = 1..kw) that may lie
//       inside the softening support of some lane's pair. Three tiers, all
//       with warp-uniform bounds: the centre/edge pair and the pairs that may
//       reach the inner core (u < 1/2) on some lane use spline_over_r2; the
//       other pairs up to kw use the outer-shell form; the rest the Newtonian
//       loop (1/r^3), which is exact there because |dz +- k| >= k - 1/2 > h.
//   EDGE = false leaves the edge image out (the near part |k| < n_cut only).
template <bool EDGE = true, int NC = 0>  // NC > 0: the window fixed at compile time (n_cut is then NC)
__device__ __forceinline__ void pair_images_fp32(float dR2, float dz, float hh, int n_cut_rt, float fnc, int kw,
                                                 float& sr, float& sz) {
  const int n_cut = NC > 0 ? NC : n_cut_rt;
  const u64 DR2 = pk(dR2, dR2);
  const u64 STEP = pk(1.0f, -1.0f);
  // centre image (k = 0) and edge image (dz - sign(dz) Ncut, absent at dz == 0)
  u64 O = pk(dz, dz - copysignf(fnc, dz));
  const u64 W = pk(1.0f, EDGE && dz != 0.0f ? 1.0f : 0.0f);
  // The centre/edge pair (CR, CZ) is kept apart from the +-k series (SR, SZ)
  // until the end: the reverse pair (j, i) walks the same images with its
  // lanes swapped, so both get the same sr and opposite sz, bit for bit.
  u64 CR, CZ;
  u64 SR = pk(0.0f, 0.0f), SZ = pk(0.0f, 0.0f);
  int k = 1;
  if (kw >= 0) {
    // some lane of the warp has its pair inside the softening support
    const float ih = rcp_approx(hh);
    const u64 NIH = pk(-ih, -ih);
    int k1 = 0;  // image pairs 1 .. k1 may reach the inner core (u < 1/2)
    const bool core = 4.0f * dR2 < hh * hh;
    if (__any_sync(0xffffffffu, core)) {
      // the full three-branch spline where some lane can have u < 1/2: the
      // centre, and pairs k with |k| < hh/2 + 1/2 (bounded by rn(hh/2))
      const int kl = core ? __float_as_int(__fadd_rn(0.5f * hh, kTwo23)) : kTwo23Bits;
      k1 = min(__reduce_max_sync(0xffffffffu, kl) - kTwo23Bits, n_cut - 1);
      const u64 IH = pk(ih, ih);
      const float ih3 = ih * ih * ih;
      const u64 IH3 = pk(ih3, ih3);
      CR = mul2(spline_over_r2(O, DR2, IH, NIH, IH3), W);
      CZ = mul2(O, CR);
      O = pk(dz, dz);
      for (; k <= k1; ++k) {
        O = add2(O, STEP);
        const u64 F = spline_over_r2(O, DR2, IH, NIH, IH3);
        SR = add2(SR, F);
        SZ = fma2(O, F, SZ);
      }
    } else {
      CR = mul2(spline_outer_over_r2(O, DR2, NIH), W);
      CZ = mul2(O, CR);
      O = pk(dz, dz);
    }
    // outer shell only (u >= 1/2 on every lane) up to the support bound
    const int kg = min(kw, n_cut - 1);
#pragma unroll(kSplineUnroll)
    for (; k <= kg; ++k) {
      O = add2(O, STEP);
      const u64 F = spline_outer_over_r2(O, DR2, NIH);
      SR = add2(SR, F);
      SZ = fma2(O, F, SZ);
    }
  } else {
    const u64 R2 = fma2(O, O, DR2);
    float ra, rb;
    upk(R2, ra, rb);
    const u64 RI = pk(rsq(ra), rsq(rb));
    CR = mul2(mul2(mul2(RI, RI), RI), W);
    CZ = mul2(O, CR);
    O = pk(dz, dz);
  }
  // Newtonian image pairs k .. n_cut - 1, outward. With the window fixed at
  // compile time and no softened pair beyond the centre (k == 1, the common
  // case), one straight run; else the first (count mod 4) enter a straight run
  // part-way (no remainder loop) and the rest go in fours.
  const int cnt = n_cut - k;
  if (NC > 0 && k == 1) {
#pragma unroll
    for (int q = 1; q < NC; ++q) newton_pair(O, STEP, DR2, SR, SZ);
  } else {
  switch (cnt & 3) {
    case 3: newton_pair(O, STEP, DR2, SR, SZ);  // fall through
    case 2: newton_pair(O, STEP, DR2, SR, SZ);  // fall through
    case 1: newton_pair(O, STEP, DR2, SR, SZ);  // fall through
    default: break;
  }
#pragma unroll 1
  for (int q = cnt >> 2; q > 0; --q) {
    newton_pair(O, STEP, DR2, SR, SZ);
    newton_pair(O, STEP, DR2, SR, SZ);
    newton_pair(O, STEP, DR2, SR, SZ);
    newton_pair(O, STEP, DR2, SR, SZ);
  }
  }
  float s0, s1, z0, z1, c0, c1, d0, d1;
  upk(SR, s0, s1);
  upk(SZ, z0, z1);
  upk(CR, c0, c1);
  upk(CZ, d0, d1);
  sr = (s0 + s1) + (c0 + c1);
  sz = (z0 + z1) + (d0 + d1);
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

#ifndef STEPS_J_UNROLL
#define STEPS_J_UNROLL 2      // unroll of the j loop inside a Kahan group
#endif
constexpr int kJUnroll = STEPS_J_UNROLL;
static_assert(kBJ % STEPS_KAHAN_GROUP == 0, "a j-tile holds whole Kahan groups");

// All pairs of i with the kBJ j of a (padded) shared-memory tile: pair forces
// are summed plainly over groups of STEPS_KAHAN_GROUP j, and each group sum
// enters the compensated per-i sum.
template <bool KAHAN>
__device__ __forceinline__ void pair_tile_fp32(const IParticle& I, const float4* sA, const float4* sB, int n_cut,
                                               float fnc, float& sx, float& sy, float& sz, float& cx, float& cy,
                                               float& cz) {
#pragma unroll 1
  for (int k0 = 0; k0 < kBJ; k0 += STEPS_KAHAN_GROUP) {
    float gx = 0.f, gy = 0.f, gz = 0.f;
#pragma unroll(kJUnroll)
    for (int k = k0; k < k0 + STEPS_KAHAN_GROUP; ++k) {
      const float4 A = sA[k];
      const float4 B = sB[k];
      float dx, dy, dz, dR2, hh;
      int kw;
      pair_geometry(I, A, B, dx, dy, dz, dR2, hh, kw);
      float sr, szz;
      pair_images_fp32(dR2, dz, hh, n_cut, fnc, kw, sr, szz);
      const float msr = A.w * sr;
      gx = fmaf(dx, msr, gx);
      gy = fmaf(dy, msr, gy);
      gz = fmaf(A.w, szz, gz);
    }
    acc<KAHAN>(sx, cx, gx);
    acc<KAHAN>(sy, cy, gy);
    acc<KAHAN>(sz, cz, gz);
  }
}

// part layout: [slot][3][kBI] doubles, slot = i-block + CTA. The units cover
// the i-blocks [b0, b0 + U / NT) (all of them unless the rows are sharded), and
// slots count i-blocks from b0.
template <bool KAHAN>
__global__ void __launch_bounds__(kBI, 8)
pair_fp32_kernel(const float4* __restrict__ jA, const float4* __restrict__ jB, int n, int n_cut,
                 long long U, int NT, int C, double* __restrict__ part, int b0 = 0) {
  __shared__ float4 sA[kBJ];
  __shared__ float4 sB[kBJ];
  const int c = blockIdx.x;
  const long long u0 = (long long)c * U / C;
  const long long u1 = (long long)(c + 1) * U / C;
  const float fnc = (float)n_cut;
  long long u = u0;
  while (u < u1) {
    const int lb = (int)(u / NT);  // i-block of the evaluated range [b0, b0 + U / NT)
    const int b = b0 + lb;
    const int t0 = (int)(u % NT);
    const long long rem = u1 - u;
    const int t1 = (int)min((long long)NT, (long long)t0 + rem);
    const int i = b * kBI + threadIdx.x;
    const IParticle I = load_i(jA, jB, min(i, n - 1));
    float sx = 0.f, sy = 0.f, sz = 0.f, cx = 0.f, cy = 0.f, cz = 0.f;
    for (int t = t0; t < t1; ++t) {
      __syncthreads();
      load_tile(jA, jB, n, t, sA, sB);
      __syncthreads();
      pair_tile_fp32<KAHAN>(I, sA, sB, n_cut, fnc, sx, sy, sz, cx, cy, cz);
    }
    const long long slot = (long long)lb + c;
    double* dst = part + slot * 3 * kBI;
    dst[threadIdx.x] = (double)sx + (double)cx * (KAHAN ? -1.0 : 0.0);
    dst[kBI + threadIdx.x] = (double)sy + (double)cy * (KAHAN ? -1.0 : 0.0);
    dst[2 * kBI + threadIdx.x] = (double)sz + (double)cz * (KAHAN ? -1.0 : 0.0);
    u += t1 - t0;
  }
}

}  // namespace steps
