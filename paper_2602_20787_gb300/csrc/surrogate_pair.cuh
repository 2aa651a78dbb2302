// Pair kernel with the learned far-image surrogate (this project's method; the
// window of eq. ForceCylindrical is unchanged, only how its far part is
// evaluated). Per pair: the near images |k| <= n0 are summed exactly as in
// pair_fp32.cuh; the tail is B1 + E * (MLP(u) * sc + mu) (see
// surrogate_train.cuh), plus the exact spline correction of tail images that
// lie inside the softening support.
//
// The MLP runs on the tensor cores with mma.sync (FP16 operands, FP32
// accumulation) over the 32 pairs of a warp (one per lane, same j): two m16
// tiles, rows assigned so that the quad of lanes 4g..4g+3 owns rows g and g+8
// of both tiles, i.e. its own four pairs. The accumulator fragment of one
// layer is, after ReLU and packing to f16x2, the A fragment of the next, so
// activations never leave registers; only the three inputs are exchanged
// within a quad (shuffles) and the two outputs are read back from the quad's
// first lane. Weights live in registers as B fragments, biases seed the
// accumulators.
#pragma once
#include <cstdint>

#include "pair_fp32.cuh"

namespace steps {

// Per-lane B fragments and accumulator seeds, prepared on the host from the
// FP32 weights (W1 as m16n8k8 fragments, W2 and W3 as m16n8k16 fragments).
struct SurrLane {
  uint32_t w1[4];   // n-block nb: {W1[8nb+g][2t], W1[8nb+g][2t+1]} (input 2 at t = 1, zero beyond)
  uint32_t w2[16];  // [kb][nb][2]
  uint32_t w3[4];   // [kb][2], rows 0, 1 of W3 only
  float b1[8];      // [nb][2]: b1[8nb+2t], b1[8nb+2t+1]
  float b2[8];
  float b3[2];
  float pad[6];
};
static_assert(sizeof(SurrLane) == 48 * 4, "SurrLane layout");

// Word w of lane L's SurrLane lives at wt[w * 32 + L] in shared memory
// (word-major), so a warp reading one word touches 32 distinct banks.
constexpr int kSurrWords = sizeof(SurrLane) / 4;
struct SurrW {
  const uint32_t* p;  // wt + lane
  __device__ __forceinline__ uint32_t u(int w) const { return p[w * 32]; }
  __device__ __forceinline__ float f(int w) const { return __uint_as_float(p[w * 32]); }
};
constexpr int kW1 = 0, kW2 = 4, kW3 = 20, kB1 = 24, kB2 = 32, kB3 = 40;

// Stage the 32 lanes' fragments word-major into shared memory (all threads of
// the block take part; ends with a barrier).
__device__ __forceinline__ void stage_surr_weights(const SurrLane* __restrict__ wl, uint32_t* wt) {
  const uint32_t* src = reinterpret_cast<const uint32_t*>(wl);
  for (int k = threadIdx.x; k < 32 * kSurrWords; k += blockDim.x) {
    const int lane = k / kSurrWords, w = k % kSurrWords;
    wt[w * 32 + lane] = src[k];
  }
  __syncthreads();
}

struct SurrConst {
  float mu0, mu1, sc0, sc1;
  float inv_dR_max, dR_max;
  int n0;
};

__device__ __forceinline__ void mma_k8(float d[4], uint32_t a0, uint32_t a1, uint32_t b0, const float c[4]) {
  asm("mma.sync.aligned.m16n8k8.row.col.f32.f16.f16.f32 {%0,%1,%2,%3}, {%4,%5}, {%6}, {%7,%8,%9,%10};"
      : "=f"(d[0]), "=f"(d[1]), "=f"(d[2]), "=f"(d[3])
      : "r"(a0), "r"(a1), "r"(b0), "f"(c[0]), "f"(c[1]), "f"(c[2]), "f"(c[3]));
}
__device__ __forceinline__ void mma_k16(float d[4], const uint32_t a[4], uint32_t b0, uint32_t b1, const float c[4]) {
  asm("mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%10,%11,%12,%13};"
      : "=f"(d[0]), "=f"(d[1]), "=f"(d[2]), "=f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1), "f"(c[0]), "f"(c[1]), "f"(c[2]), "f"(c[3]));
}
// ReLU and pack two FP32 values as f16x2 (lo in the lower half)
__device__ __forceinline__ uint32_t relu_pack(float lo, float hi) {
  uint32_t r;
  asm("cvt.rn.relu.f16x2.f32 %0, %1, %2;" : "=r"(r) : "f"(hi), "f"(lo));
  return r;
}
__device__ __forceinline__ uint32_t pack_h2(float lo, float hi) {
  uint32_t r;
  asm("cvt.rn.f16x2.f32 %0, %1, %2;" : "=r"(r) : "f"(hi), "f"(lo));
  return r;
}

// The MLP for NJ x 32 pairs of the warp (NJ values of j, one pair per lane
// each); every lane passes its own pairs' inputs and receives their outputs.
// The 2 NJ m-tiles are independent chains of mma, which the scheduler
// interleaves. Must be called by all 32 lanes with uniform control flow.
template <int NJ>
__device__ __forceinline__ void mlp_warp(const SurrW& W, const float (&u)[NJ][3], float (&y)[NJ][2]) {
  const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
  uint32_t in[NJ][4];
#pragma unroll
  for (int jj = 0; jj < NJ; ++jj) {
    const uint32_t p01 = pack_h2(u[jj][0], u[jj][1]), p2 = pack_h2(u[jj][2], 0.0f);
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const uint32_t s01 = __shfl_sync(0xffffffffu, p01, 4 * g + q);
      const uint32_t s2 = __shfl_sync(0xffffffffu, p2, 4 * g + q);
      in[jj][q] = t == 0 ? s01 : (t == 1 ? s2 : 0u);
    }
  }
  float out[NJ][2][4];
#pragma unroll
  for (int jj = 0; jj < NJ; ++jj) {
#pragma unroll
    for (int mt = 0; mt < 2; ++mt) {
      // layer 1: [16 pairs x 8 inputs] x [8 x 32]
      float d1[4][4];
#pragma unroll
      for (int nb = 0; nb < 4; ++nb) {
        const float b0 = W.f(kB1 + 2 * nb), b1v = W.f(kB1 + 2 * nb + 1);
        const float c[4] = {b0, b1v, b0, b1v};
        mma_k8(d1[nb], in[jj][2 * mt], in[jj][2 * mt + 1], W.u(kW1 + nb), c);
      }
      uint32_t a2[2][4];
#pragma unroll
      for (int kb = 0; kb < 2; ++kb) {
        a2[kb][0] = relu_pack(d1[2 * kb][0], d1[2 * kb][1]);
        a2[kb][1] = relu_pack(d1[2 * kb][2], d1[2 * kb][3]);
        a2[kb][2] = relu_pack(d1[2 * kb + 1][0], d1[2 * kb + 1][1]);
        a2[kb][3] = relu_pack(d1[2 * kb + 1][2], d1[2 * kb + 1][3]);
      }
      // layer 2: [16 x 32] x [32 x 32]
      float d2[4][4];
#pragma unroll
      for (int nb = 0; nb < 4; ++nb) {
        const float b0 = W.f(kB2 + 2 * nb), b1v = W.f(kB2 + 2 * nb + 1);
        const float c[4] = {b0, b1v, b0, b1v};
        mma_k16(d2[nb], a2[0], W.u(kW2 + nb * 2), W.u(kW2 + nb * 2 + 1), c);
        mma_k16(d2[nb], a2[1], W.u(kW2 + (4 + nb) * 2), W.u(kW2 + (4 + nb) * 2 + 1), d2[nb]);
      }
      uint32_t a3[2][4];
#pragma unroll
      for (int kb = 0; kb < 2; ++kb) {
        a3[kb][0] = relu_pack(d2[2 * kb][0], d2[2 * kb][1]);
        a3[kb][1] = relu_pack(d2[2 * kb][2], d2[2 * kb][3]);
        a3[kb][2] = relu_pack(d2[2 * kb + 1][0], d2[2 * kb + 1][1]);
        a3[kb][3] = relu_pack(d2[2 * kb + 1][2], d2[2 * kb + 1][3]);
      }
      // layer 3: [16 x 32] x [32 x 8] (columns 0, 1 used)
      const float c3[4] = {W.f(kB3), W.f(kB3 + 1), W.f(kB3), W.f(kB3 + 1)};
      mma_k16(out[jj][mt], a3[0], W.u(kW3), W.u(kW3 + 1), c3);
      mma_k16(out[jj][mt], a3[1], W.u(kW3 + 2), W.u(kW3 + 3), out[jj][mt]);
    }
  }
  // outputs of rows g, g+8 of both tiles sit in lane 4g (columns 0, 1)
  const int src = 4 * g;
  const int mt = t >> 1, hi = t & 1;
#pragma unroll
  for (int jj = 0; jj < NJ; ++jj) {
    float v[2][4];
#pragma unroll
    for (int m = 0; m < 2; ++m)
#pragma unroll
      for (int e = 0; e < 4; ++e) v[m][e] = __shfl_sync(0xffffffffu, out[jj][m][e], src);
    y[jj][0] = mt == 0 ? (hi ? v[0][2] : v[0][0]) : (hi ? v[1][2] : v[1][0]);
    y[jj][1] = mt == 0 ? (hi ? v[0][3] : v[0][1]) : (hi ? v[1][3] : v[1][1]);
  }
}

// FP32 base of one side of the tail (cells [lo, hi]): SR and SZ parts and the
// near-end reciprocal distance.
__device__ __forceinline__ void side_base_fp32(float R2, float lo, float hi, float& sr, float& sz, float& il_out) {
  const float il = rsq(fmaf(lo, lo, R2)), ih = rsq(fmaf(hi, hi, R2));
  const float il2 = il * il, ih2 = ih * ih;
  const float IR = (hi - lo) * (hi + lo) * il2 * ih2 * rcp_approx(fmaf(hi, ih, lo * il));
  const float IZ = il - ih;
  const float il5 = il2 * il2 * il, ih5 = ih2 * ih2 * ih;
  const float dRl = -3.0f * lo * il5, dRh = -3.0f * hi * ih5;
  const float dZl = il2 * il - 3.0f * lo * lo * il5, dZh = ih2 * ih - 3.0f * hi * hi * ih5;
  sr = IR - (dRh - dRl) * (1.0f / 24.0f);
  sz = IZ - (dZh - dZl) * (1.0f / 24.0f);
  il_out = il;
}

// Per-pair state of the surrogate evaluation between its stages.
struct SurrPair {
  float sr, sz;          // near-image sums so far
  float br, bz, er, ez;  // tail base and envelope
  float sg;              // sign(dz)
  float u[3];            // network inputs
  float ih, ih3;         // 1/h, 1/h^3 (when some lane is softened)
};

// Stage A: near images |k| <= n0 exactly (as in pair_fp32.cuh), the tail base,
// the envelope and the network inputs. kw: warp-uniform spline bound.
__device__ __forceinline__ void surr_stage_a(float dR2, float dz, float hh, int n_cut, int kw, const SurrConst& S,
                                             SurrPair& P) {
  const u64 DR2 = pk(dR2, dR2);
  const u64 STEP = pk(1.0f, -1.0f);
  const int n0 = S.n0;
  u64 SR, SZ, O;
  int k = 1;
  P.ih = 0.f;
  P.ih3 = 0.f;
  if (kw >= 0) {
    P.ih = rcp_approx(hh);
    P.ih3 = P.ih * P.ih * P.ih;
    const u64 IH = pk(P.ih, P.ih), IH3 = pk(P.ih3, P.ih3);
    O = pk(dz, dz);
    const u64 F = mul2(spline_over_r2(O, DR2, IH, IH3), pk(1.0f, 0.0f));
    SR = F;
    SZ = mul2(O, F);
    const int kg = min(kw, n0);
#pragma unroll(kSplineUnroll)
    for (; k <= kg; ++k) {
      O = add2(O, STEP);
      const u64 G = spline_over_r2(O, DR2, IH, IH3);
      SR = add2(SR, G);
      SZ = fma2(O, G, SZ);
    }
  } else {
    const float r2 = fmaf(dz, dz, dR2);
    const float ri = rsq(r2);
    const float r3 = ri * ri * ri;
    SR = pk(r3, 0.0f);
    SZ = pk(dz * r3, 0.0f);
    O = pk(dz, dz);
  }
#pragma unroll 4
  for (; k <= n0; ++k) {
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
  P.sr = s0 + s1;
  P.sz = z0 + z1;
  // tail base and envelope (|dz|; z part gets sign(dz))
  const float adz = fabsf(dz), A = (float)n0 + 0.5f;
  const float kneg = adz > 0.0f ? (float)n_cut : (float)(n_cut - 1);
  float br1, bz1, il1, br2, bz2, il2;
  side_base_fp32(dR2, A + adz, (float)(n_cut - 1) + 0.5f + adz, br1, bz1, il1);
  side_base_fp32(dR2, A - adz, kneg + 0.5f - adz, br2, bz2, il2);
  const float e = il1 * il1;
  P.er = e * e * e;
  P.ez = e * e * il1;
  P.br = br1 + br2;
  P.bz = bz1 - bz2;
  P.sg = dz > 0.0f ? 1.0f : (dz < 0.0f ? -1.0f : 0.0f);
  const float dR = dR2 * rsq(fmaxf(dR2, 1e-30f));
  P.u[0] = 2.0f * fminf(dR, S.dR_max) * S.inv_dR_max - 1.0f;
  P.u[1] = 4.0f * adz - 1.0f;
  P.u[2] = 2.0f * fminf(hh, A) / A - 1.0f;
}

// Stage C: tail = base + envelope x network output, plus the exact spline
// correction of tail images inside some lane's softening support.
__device__ __forceinline__ void surr_stage_c(float dR2, float dz, int n_cut, int kw, const SurrConst& S,
                                             const SurrPair& P, float y0, float y1, float& sr, float& sz) {
  const int n0 = S.n0;
  sr = P.sr + P.br + P.er * fmaf(y0, S.sc0, S.mu0);
  sz = P.sz + P.sg * (P.bz + P.ez * fmaf(y1, S.sc1, S.mu1));
  if (kw > n0) {
    const u64 DR2 = pk(dR2, dR2);
    const u64 STEP = pk(1.0f, -1.0f);
    const u64 IH = pk(P.ih, P.ih), IH3 = pk(P.ih3, P.ih3);
    const int kt = min(kw, n_cut - 1);
    u64 CR = pk(0.f, 0.f), CZ = pk(0.f, 0.f);
    u64 O = pk(dz + (float)n0, dz - (float)n0);
    for (int kk = n0 + 1; kk <= kt; ++kk) {
      O = add2(O, STEP);
      const u64 R2 = fma2(O, O, DR2);
      float ra, rb;
      upk(R2, ra, rb);
      const u64 RI = pk(rsq(ra), rsq(rb));
      const u64 N3 = mul2(mul2(RI, RI), RI);
      const u64 D = fma2(N3, pk(-1.0f, -1.0f), spline_over_r2(O, DR2, IH, IH3));
      CR = add2(CR, D);
      CZ = fma2(O, D, CZ);
    }
    if (kw >= n_cut) {  // the edge image as well
      const float oe = dz - copysignf((float)n_cut, dz);
      const u64 OE = pk(oe, oe);
      const float r2 = fmaf(oe, oe, dR2);
      const float ri = rsq(r2);
      float fa, fb;
      upk(spline_over_r2(OE, DR2, IH, IH3), fa, fb);
      const float d = (dz != 0.0f ? 1.0f : 0.0f) * (fa - ri * ri * ri);
      CR = add2(CR, pk(d, 0.f));
      CZ = add2(CZ, pk(oe * d, 0.f));
    }
    float c0, c1, d0, d1;
    upk(CR, c0, c1);
    upk(CZ, d0, d1);
    sr += c0 + c1;
    sz += d0 + d1;
  }
}

// Geometry of the pair (i, j) shared by both forms.
__device__ __forceinline__ void pair_geometry(const IParticle& I, const float4& A, const float4& B, float& dx, float& dy,
                                              float& dz, float& dR2, float& hh, int& kw) {
  dx = (I.xh - A.x) + (I.xl - B.x);
  dy = (I.yh - A.y) + (I.yl - B.y);
  dz = I.zh - A.z;
  dz = (dz - rintf(dz)) + (I.zl - B.z);
  dR2 = fmaf(dx, dx, dy * dy);
  hh = I.h + B.w;
  const int kl = dR2 < hh * hh ? (int)(hh + 0.5f) : -1;
  kw = __reduce_max_sync(0xffffffffu, kl);
}

// One j-tile of pairs for one i (shared by the stream-K and the subset kernels).
// The surrogate form handles two j per network call.
template <bool KAHAN, bool SURR>
__device__ __forceinline__ void pair_tile(const IParticle& I, const float4* sA, const float4* sB, int jn, int self,
                                          int n_cut, float fnc, const SurrW& W, const SurrConst& S, float& sx,
                                          float& sy, float& sz, float& cx, float& cy, float& cz) {
  constexpr int STEPJ = SURR ? 2 : 1;
  for (int k0 = 0; k0 < jn; k0 += STEPS_KAHAN_GROUP) {
    float gx = 0.f, gy = 0.f, gz = 0.f;
    const int ke = min(k0 + STEPS_KAHAN_GROUP, jn);
    for (int k = k0; k < ke; k += STEPJ) {
      float dx[STEPJ], dy[STEPJ], dz[STEPJ], dR2[STEPJ], hh[STEPJ], mj[STEPJ], sr[STEPJ], szz[STEPJ];
      int kw[STEPJ];
#pragma unroll
      for (int jj = 0; jj < STEPJ; ++jj) {
        // a second j past the tile end repeats the first with zero mass
        const int kk = min(k + jj, ke - 1);
        const float4 A = sA[kk];
        const float4 B = sB[kk];
        pair_geometry(I, A, B, dx[jj], dy[jj], dz[jj], dR2[jj], hh[jj], kw[jj]);
        mj[jj] = (kk == self || k + jj >= ke) ? 0.0f : A.w;
      }
      if (SURR) {
        SurrPair P[STEPJ];
        float u[STEPJ][3], y[STEPJ][2];
#pragma unroll
        for (int jj = 0; jj < STEPJ; ++jj) {
          surr_stage_a(dR2[jj], dz[jj], hh[jj], n_cut, kw[jj], S, P[jj]);
          u[jj][0] = P[jj].u[0];
          u[jj][1] = P[jj].u[1];
          u[jj][2] = P[jj].u[2];
        }
        mlp_warp<STEPJ>(W, u, y);
#pragma unroll
        for (int jj = 0; jj < STEPJ; ++jj)
          surr_stage_c(dR2[jj], dz[jj], n_cut, kw[jj], S, P[jj], y[jj][0], y[jj][1], sr[jj], szz[jj]);
      } else {
#pragma unroll
        for (int jj = 0; jj < STEPJ; ++jj) pair_images_fp32(dR2[jj], dz[jj], hh[jj], n_cut, fnc, kw[jj], sr[jj], szz[jj]);
      }
#pragma unroll
      for (int jj = 0; jj < STEPJ; ++jj) {
        const float msr = mj[jj] * sr[jj];
        gx = fmaf(dx[jj], msr, gx);
        gy = fmaf(dy[jj], msr, gy);
        gz = fmaf(mj[jj], szz[jj], gz);
      }
    }
    acc<KAHAN>(sx, cx, gx);
    acc<KAHAN>(sy, cy, gy);
    acc<KAHAN>(sz, cz, gz);
  }
}

// Stream-K kernel with the surrogate tail (same work split and partial layout
// as pair_fp32_kernel).
#ifndef STEPS_SURR_MIN_BLOCKS
#define STEPS_SURR_MIN_BLOCKS 4  // co-resident CTAs per SM asked of the register allocator
#endif

template <bool KAHAN>
__global__ void __launch_bounds__(kBI, STEPS_SURR_MIN_BLOCKS)
pair_fp32_surr_kernel(const float4* __restrict__ jA, const float4* __restrict__ jB, int n, int n_cut, long long U,
                      int NT, int C, const SurrLane* __restrict__ wl, SurrConst S, double* __restrict__ part) {
  __shared__ float4 sA[kBJ];
  __shared__ float4 sB[kBJ];
  // weight fragments stay in shared memory (word-major, conflict-free) and are
  // read where the mma needs them, which leaves registers for resident warps
  __shared__ uint32_t sWT[32 * kSurrWords];
  stage_surr_weights(wl, sWT);
  const SurrW W{sWT + (threadIdx.x & 31)};
  const int c = blockIdx.x;
  const long long u0 = (long long)c * U / C;
  const long long u1 = (long long)(c + 1) * U / C;
  const float fnc = (float)n_cut;
  long long u = u0;
  while (u < u1) {
    const int b = (int)(u / NT);
    const int t0 = (int)(u % NT);
    const int t1 = (int)min((long long)NT, (long long)t0 + (u1 - u));
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
      pair_tile<KAHAN, true>(I, sA, sB, min(kBJ, n - t * kBJ), i - t * kBJ, n_cut, fnc, W, S, sx, sy, sz, cx, cy,
                             cz);
    }
    double* dst = part + ((long long)b + c) * 3 * kBI;
    dst[threadIdx.x] = (double)sx - (KAHAN ? (double)cx : 0.0);
    dst[kBI + threadIdx.x] = (double)sy - (KAHAN ? (double)cy : 0.0);
    dst[2 * kBI + threadIdx.x] = (double)sz - (KAHAN ? (double)cz : 0.0);
    u += t1 - t0;
  }
}

// Subset kernel (acceptance checks): CTA (bx, by) takes listed i-particles
// [bx * kBI, +kBI) against j-tiles [by * tpc, (by + 1) * tpc); partials
// part[by][3][ni]. The listed indices are internal and may repeat.
template <bool KAHAN, bool SURR>
__global__ void __launch_bounds__(kBI, 3)
pair_fp32_subset_kernel(const float4* __restrict__ jA, const float4* __restrict__ jB, int n, int n_cut,
                        const int64_t* __restrict__ idx, int ni, int tpc, const SurrLane* __restrict__ wl, SurrConst S,
                        double* __restrict__ part) {
  __shared__ float4 sA[kBJ];
  __shared__ float4 sB[kBJ];
  __shared__ uint32_t sWT[32 * kSurrWords];
  if (SURR) stage_surr_weights(wl, sWT);
  const SurrW W{sWT + (threadIdx.x & 31)};
  const int q = blockIdx.x * kBI + threadIdx.x;
  const int i = (int)idx[min(q, ni - 1)];
  IParticle I;
  {
    const float4 a = jA[i];
    const float4 b = jB[i];
    I.xh = a.x; I.yh = a.y; I.zh = a.z; I.xl = b.x; I.yl = b.y; I.zl = b.z; I.h = b.w;
  }
  const int NT = (n + kBJ - 1) / kBJ;
  const int t0 = blockIdx.y * tpc, t1 = min(NT, t0 + tpc);
  float sx = 0.f, sy = 0.f, sz = 0.f, cx = 0.f, cy = 0.f, cz = 0.f;
  for (int t = t0; t < t1; ++t) {
    __syncthreads();
    const int jl = t * kBJ + threadIdx.x;
    if (jl < n) {
      sA[threadIdx.x] = jA[jl];
      sB[threadIdx.x] = jB[jl];
    }
    __syncthreads();
    pair_tile<KAHAN, SURR>(I, sA, sB, min(kBJ, n - t * kBJ), i - t * kBJ, n_cut, (float)n_cut, W, S, sx, sy, sz, cx,
                           cy, cz);
  }
  if (q < ni) {
    double* dst = part + (long long)blockIdx.y * 3 * ni;
    dst[q] = (double)sx - (KAHAN ? (double)cx : 0.0);
    dst[ni + q] = (double)sy - (KAHAN ? (double)cy : 0.0);
    dst[2 * ni + q] = (double)sz - (KAHAN ? (double)cz : 0.0);
  }
}

}  // namespace steps
