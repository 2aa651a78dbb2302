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
// activations never leave registers. The three inputs reach the quad through
// a small per-warp shared buffer. The output layer adds the two tiles'
// products into one accumulator, the even tile's in columns 0..3 and the odd
// tile's in columns 4..7, each output repeated twice, so every lane already
// holds its own pair's outputs. Weights are B fragments read from shared memory
// once per call per layer; the hidden bias seeds the accumulators.
#pragma once
#include <cstdint>

#include "pair_fp32.cuh"

namespace steps {

// Per-lane B fragments and accumulator seeds, prepared on the host from the
// FP32 weights (W1 as m16n8k8 fragments, W2 and W3 as m16n8k16 fragments).
// The first layer's bias rides in the weights: the network's input vector
// carries a constant 1 as its fourth component, whose weight column is b1. The
// output bias is folded into the output shift on the host (mu + sc b3). The
// hidden bias b2 is laid out as the mma's C operand (c0..c3 of lane (g, t) hold
// columns 2t, 2t + 1 of rows g and g + 8), so one 128-bit load yields a C
// operand with no register moves.
struct SurrLane {
  uint32_t w1[4];   // n-block nb: {W1[8nb+g][2t], W1[8nb+g][2t+1]}; t = 1: {W1[.][2], b1[8nb+g]}; zero beyond
  uint32_t w2[16];  // [nb][kb][2]
  uint32_t w3e[4];  // [kb][2]: output column g of the even m-tile's product (lanes g < 4; zero for g >= 4)
  uint32_t w3o[4];  // [kb][2]: output column g of the odd m-tile's product (lanes g >= 4; zero for g < 4)
  float c2[16];     // [nb][4]: b2[8nb+2t], b2[8nb+2t+1], b2[8nb+2t], b2[8nb+2t+1]
};
static_assert(sizeof(SurrLane) == 44 * 4, "SurrLane layout");

// Lane L's SurrLane lives at wt[L * kSurrStride ...] in shared memory. A row
// stride of 44 words (12 mod 32) puts the 16-byte loads of a quarter warp (8
// lanes) on 32 distinct banks. Each layer's fragments are read once per
// network call with 128-bit volatile shared loads: kept out of the register
// file across the j loop, they leave room for resident warps.
constexpr int kSurrWords = sizeof(SurrLane) / 4;
constexpr int kSurrStride = kSurrWords;
static_assert(kSurrStride % 32 == 4 || kSurrStride % 32 == 12 || kSurrStride % 32 == 20 || kSurrStride % 32 == 28,
              "conflict-free 16-byte loads");
struct SurrW {
  const uint32_t* p;  // wt + lane * kSurrStride (16-byte aligned)
  __device__ __forceinline__ uint4 ld4(int w) const {
    uint4 v;
    asm volatile("ld.shared.v4.b32 {%0, %1, %2, %3}, [%4];"
                 : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
                 : "r"((uint32_t)__cvta_generic_to_shared(p + w)));
    return v;
  }
  __device__ __forceinline__ float4 ldc(int w) const {
    const uint4 v = ld4(w);
    return make_float4(__uint_as_float(v.x), __uint_as_float(v.y), __uint_as_float(v.z), __uint_as_float(v.w));
  }
};
constexpr int kW1 = 0, kW2 = 4, kW3E = 20, kW3O = 24, kC2 = 28;

// Stage the 32 lanes' fragments into shared memory (all threads of the block
// take part; ends with a barrier).
__device__ __forceinline__ void stage_surr_weights(const SurrLane* __restrict__ wl, uint32_t* wt) {
  const uint32_t* src = reinterpret_cast<const uint32_t*>(wl);
  for (int k = threadIdx.x; k < 32 * kSurrWords; k += blockDim.x) {
    const int lane = k / kSurrWords, w = k % kSurrWords;
    wt[lane * kSurrStride + w] = src[k];
  }
  __syncthreads();
}

struct SurrConst {
  float mu0, mu1, sc0, sc1;
  float inv_dR_max, dR_max;
  int n0;
  // derived on the host (surr_const_finish): A = n0 + 1/2, 2 / A, 2 / dR_max,
  // and the far end of the finite window, n_cut - 1/2
  float A, two_over_A, two_inv_dR_max, fnh;
};

__host__ __device__ __forceinline__ void surr_const_finish(SurrConst& S, int n_cut) {
  S.A = (float)S.n0 + 0.5f;
  S.two_over_A = 2.0f / S.A;
  S.two_inv_dR_max = 2.0f * S.inv_dR_max;
  S.fnh = (float)n_cut - 0.5f;
}

__device__ __forceinline__ void mma_k8(float d[4], uint32_t a0, uint32_t a1, uint32_t b0, const float4& c) {
  asm("mma.sync.aligned.m16n8k8.row.col.f32.f16.f16.f32 {%0,%1,%2,%3}, {%4,%5}, {%6}, {%7,%8,%9,%10};"
      : "=f"(d[0]), "=f"(d[1]), "=f"(d[2]), "=f"(d[3])
      : "r"(a0), "r"(a1), "r"(b0), "f"(c.x), "f"(c.y), "f"(c.z), "f"(c.w));
}
__device__ __forceinline__ void mma_k16(float d[4], const uint32_t a[4], uint32_t b0, uint32_t b1, const float4& c) {
  asm("mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%10,%11,%12,%13};"
      : "=f"(d[0]), "=f"(d[1]), "=f"(d[2]), "=f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1), "f"(c.x), "f"(c.y), "f"(c.z), "f"(c.w));
}
// d += A B (the accumulator stays in place)
__device__ __forceinline__ void mma_k16_acc(float d[4], const uint32_t a[4], uint32_t b0, uint32_t b1) {
  asm("mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
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

__device__ __forceinline__ float f32(uint32_t v) { return __uint_as_float(v); }

// The MLP for NJ x 32 pairs of the warp (NJ values of j, one pair per lane
// each); every lane passes its own pairs' inputs and receives their outputs.
// Layer by layer over all 2 NJ m-tiles, so each layer's fragments are read from
// shared memory once per call and the tiles' mma chains are independent work
// for the scheduler. Must be called by all 32 lanes with uniform control flow.
// Per-warp exchange buffer of the network inputs: [NJ][slot t][kInStride]
// words; slot 0 holds the (u0, u1) f16x2 word of each lane, slot 1 the (u2, 1)
// word (the constant 1 carries the first layer's bias), slots 2 and 3 stay
// zero (columns 4..7 of the A operand). Lane (g, t) reads its A fragment,
// words 4g .. 4g+3 of slot t, with one 16-byte load; a slot stride of 40 words
// keeps those loads and the stores free of bank conflicts.
constexpr int kInStride = 40;
constexpr int kInWords = 4 * kInStride;

template <int NJ>
__device__ __forceinline__ void mlp_zero_inputs(uint32_t* buf) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int jj = 0; jj < NJ; ++jj) {
    buf[jj * kInWords + 2 * kInStride + lane] = 0u;
    buf[jj * kInWords + 3 * kInStride + lane] = 0u;
  }
}

template <int NJ>
__device__ __forceinline__ void mlp_warp(const SurrW& W, uint32_t* buf, const float (&u)[NJ][3],
                                         float (&y)[NJ][2]) {
  constexpr int NT = 2 * NJ;  // m16 tiles: tile 2 jj + mt
  const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
  uint32_t in[NJ][4];
  __syncwarp();  // the previous call's reads are done
#pragma unroll
  for (int jj = 0; jj < NJ; ++jj) {
    buf[jj * kInWords + lane] = pack_h2(u[jj][0], u[jj][1]);
    buf[jj * kInWords + kInStride + lane] = pack_h2(u[jj][2], 1.0f);
  }
  __syncwarp();
#pragma unroll
  for (int jj = 0; jj < NJ; ++jj) {
    const uint4 v = *reinterpret_cast<const uint4*>(buf + jj * kInWords + t * kInStride + 4 * g);
    in[jj][0] = v.x;
    in[jj][1] = v.y;
    in[jj][2] = v.z;
    in[jj][3] = v.w;
  }
  // layer 1: [16 pairs x 8 inputs] x [8 x 32] per tile (input 3 is the
  // constant 1, so the product already holds the bias)
  uint32_t a2[NT][2][4];
  {
    const uint4 w1 = W.ld4(kW1);
    const uint32_t wv[4] = {w1.x, w1.y, w1.z, w1.w};
    const float4 zero = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
    for (int tl = 0; tl < NT; ++tl) {
      float d1[4][4];
#pragma unroll
      for (int nb = 0; nb < 4; ++nb)
        mma_k8(d1[nb], in[tl >> 1][2 * (tl & 1)], in[tl >> 1][2 * (tl & 1) + 1], wv[nb], zero);
#pragma unroll
      for (int kb = 0; kb < 2; ++kb) {
        a2[tl][kb][0] = relu_pack(d1[2 * kb][0], d1[2 * kb][1]);
        a2[tl][kb][1] = relu_pack(d1[2 * kb][2], d1[2 * kb][3]);
        a2[tl][kb][2] = relu_pack(d1[2 * kb + 1][0], d1[2 * kb + 1][1]);
        a2[tl][kb][3] = relu_pack(d1[2 * kb + 1][2], d1[2 * kb + 1][3]);
      }
    }
  }
  // layer 2: [16 x 32] x [32 x 32] per tile, one n-block of outputs at a
  // time over all tiles (its fragments [kb][2] and bias seeds are read once
  // per call); each n-block's result is packed at once into the next layer's
  // A fragment: n-block nb fills words 2 (nb & 1), +1 of k-block nb >> 1
  uint32_t a3[NT][2][4];
#pragma unroll
  for (int nb = 0; nb < 4; ++nb) {
    const uint4 w = W.ld4(kW2 + 4 * nb);
    const float4 cb = W.ldc(kC2 + 4 * nb);
#pragma unroll
    for (int tl = 0; tl < NT; ++tl) {
      float d2[4];
      mma_k16(d2, a2[tl][0], w.x, w.y, cb);
      mma_k16_acc(d2, a2[tl][1], w.z, w.w);
      a3[tl][nb >> 1][2 * (nb & 1)] = relu_pack(d2[0], d2[1]);
      a3[tl][nb >> 1][2 * (nb & 1) + 1] = relu_pack(d2[2], d2[3]);
    }
  }
  // layer 3: per value of j, [16 x 32] x [32 x 8] for the even tile plus the
  // same for the odd tile into one accumulator: the even tile's weights fill
  // columns 0..3 and the odd tile's columns 4..7 (output n & 1 in column n),
  // the other columns' weights being zero. The output bias is in mu.
  float out[NJ][4];
  {
    const uint4 we = W.ld4(kW3E);
    const uint4 wo = W.ld4(kW3O);
    const float4 zero = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
    for (int jj = 0; jj < NJ; ++jj) {
      mma_k16(out[jj], a3[2 * jj][0], we.x, we.y, zero);
      mma_k16_acc(out[jj], a3[2 * jj][1], we.z, we.w);
      mma_k16_acc(out[jj], a3[2 * jj + 1][0], wo.x, wo.y);
      mma_k16_acc(out[jj], a3[2 * jj + 1][1], wo.z, wo.w);
    }
  }
  // lane (g, t) holds columns 2t, 2t + 1 (outputs 0, 1) of rows g and g + 8 of
  // tile t >> 1; its own pair is row g + 8 (t & 1)
  const bool hi = (t & 1) != 0;
#pragma unroll
  for (int jj = 0; jj < NJ; ++jj) {
    y[jj][0] = hi ? out[jj][2] : out[jj][0];
    y[jj][1] = hi ? out[jj][3] : out[jj][1];
  }
}

// FP32 base of both sides of the tail at once (lane a: the side beyond +n0,
// lane b: the side beyond -n0), each over the cells [lo, hi]. With
// i(x) = (x^2 + dR^2)^(-1/2), per side: the integrals
// (hi^2 - lo^2) il^2 ih^2 / (hi ih + lo il) (of i^3, written without
// cancellation) and il - ih (of x i^3), minus 1/24 of the end-point derivative
// differences, d/dx i^3 = -3 x i^5 and d/dx (x i^3) = i^3 - 3 x^2 i^5. Returns
// the SR parts of both sides added, the SZ parts subtracted (the z part is odd
// in dz), and the near-end il of side a. The packed work stays packed; the
// constants enter through scalar FMAs with immediate operands, so that no
// constant pair has to be assembled in registers.
__device__ __forceinline__ void tail_base_fp32(float R2, float lo_a, float lo_b, float hi_a, float hi_b, float& br,
                                               float& bz, float& il_a) {
  const u64 LO = pk(lo_a, lo_b), HI = pk(hi_a, hi_b);
  const u64 IL = pk(rsq(fmaf(lo_a, lo_a, R2)), rsq(fmaf(lo_b, lo_b, R2)));
  const u64 IH = pk(rsq(fmaf(hi_a, hi_a, R2)), rsq(fmaf(hi_b, hi_b, R2)));
  const u64 IL2 = mul2(IL, IL), IH2 = mul2(IH, IH);
  float e, f;
  upk(fma2(HI, IH, mul2(LO, IL)), e, f);
  const u64 IR = mul2(mul2(mul2(sub2(HI, LO), add2(HI, LO)), mul2(IL2, IH2)), pk(rcp_approx(e), rcp_approx(f)));
  const u64 P = mul2(LO, mul2(mul2(IL2, IL2), IL));  // lo il^5
  const u64 Q = mul2(HI, mul2(mul2(IH2, IH2), IH));  // hi ih^5
  const u64 D3 = sub2(mul2(IH2, IH), mul2(IL2, IL));
  const u64 E = sub2(mul2(HI, Q), mul2(LO, P));
  float qp_a, qp_b, ir_a, ir_b, d3_a, d3_b, e_a, e_b, d_a, d_b, il_b;
  upk(sub2(Q, P), qp_a, qp_b);
  upk(IR, ir_a, ir_b);
  upk(D3, d3_a, d3_b);
  upk(E, e_a, e_b);
  upk(sub2(IL, IH), d_a, d_b);
  upk(IL, il_a, il_b);
  br = fmaf(qp_a, 0.125f, ir_a) + fmaf(qp_b, 0.125f, ir_b);
  bz = fmaf(e_a, 0.125f, fmaf(d3_a, -1.0f / 24.0f, d_a)) - fmaf(e_b, 0.125f, fmaf(d3_b, -1.0f / 24.0f, d_b));
}

// The same base with both far ends at infinity (the Ncut -> infinity window):
// per side Int_lo^inf i^3 = 1/(r (r + lo)) = il^2 / (1 + lo il) and
// Int_lo^inf x i^3 = il, plus the near end's term (-3 lo il^5 and
// il^3 - 3 lo^2 il^5, over 24).
__device__ __forceinline__ void tail_base_inf_fp32(float R2, float lo_a, float lo_b, float& br, float& bz,
                                                   float& il_a) {
  const u64 LO = pk(lo_a, lo_b);
  const u64 IL = pk(rsq(fmaf(lo_a, lo_a, R2)), rsq(fmaf(lo_b, lo_b, R2)));
  const u64 IL2 = mul2(IL, IL), IL3 = mul2(IL2, IL);
  float e, f;
  upk(fma2(LO, IL, pk(1.0f, 1.0f)), e, f);
  const u64 IR = mul2(IL2, pk(rcp_approx(e), rcp_approx(f)));
  const u64 P = mul2(LO, mul2(IL2, IL3));  // lo il^5
  const u64 T = fma2(mul2(LO, P), pk(-3.0f, -3.0f), IL3);  // il^3 - 3 lo^2 il^5
  float p_a, p_b, ir_a, ir_b, t_a, t_b, il_b;
  upk(P, p_a, p_b);
  upk(IR, ir_a, ir_b);
  upk(T, t_a, t_b);
  upk(IL, il_a, il_b);
  br = fmaf(p_a, -0.125f, ir_a) + fmaf(p_b, -0.125f, ir_b);
  bz = fmaf(t_a, 1.0f / 24.0f, il_a) - fmaf(t_b, 1.0f / 24.0f, il_b);
}

// F/r of one image from its r^2: the scalar form of spline_value_r2 (all three
// branches, core selected per lane) or, with FULL false, of the outer-shell
// form spline_outer_value (exactly r^-3 for u >= 1). ih = 1 / hh.
template <bool FULL>
__device__ __forceinline__ float spline_scalar(float r2, float ih, float ih3) {
  const float ri = rsq(fmaxf(r2, 1e-30f));
  const float rr = r2 * ri;
  const float n3 = ri * ri * ri;
  const float v = fmaxf(fmaf(rr, -ih, 1.0f), 0.0f);
  const float v2 = v * v;
  const float nr = fmaf(fmaf(v, -10.6666666667f, 25.6f), v, -16.0f);
  const float outer = n3 * fmaf(v2 * v2, nr, 1.0f);
  if (!FULL) return outer;
  const float u = rr * ih;
  const float inner = fmaf(u * u, fmaf(u, 32.0f, -38.4f), 10.6666666667f) * ih3;
  return u < 0.5f ? inner : outer;
}

// Near images |k| <= n0 of a pair for the modelled-tail forms: the centre
// image k = 0 on its own (no edge image rides along), then the pairs +-k
// walked outward packed, with the warp-uniform spline tiers of
// pair_images_fp32.
template <int N0 = 0>  // N0 > 0: the near range fixed at compile time (n0 is then N0)
__device__ __forceinline__ void near_images_fp32(float dR2, float dz, float hh, int n0_rt, int kw, float& sr,
                                                 float& sz) {
  const int n0 = N0 > 0 ? N0 : n0_rt;
  const u64 DR2 = pk(dR2, dR2);
  const u64 STEP = pk(1.0f, -1.0f);
  u64 O = pk(dz, dz);
  u64 SR = pk(0.0f, 0.0f), SZ = pk(0.0f, 0.0f);
  float cr;  // the centre image's F/r
  const float c2 = fmaf(dz, dz, dR2);
  int k = 1;
  if (kw >= 0) {
    const float ih = rcp_approx(hh);
    const u64 NIH = pk(-ih, -ih);
    const bool core = 4.0f * dR2 < hh * hh;
    if (__any_sync(0xffffffffu, core)) {
      const int kl = core ? __float_as_int(__fadd_rn(0.5f * hh, kTwo23)) : kTwo23Bits;
      const int k1 = min(__reduce_max_sync(0xffffffffu, kl) - kTwo23Bits, n0);
      const float ih3 = ih * ih * ih;
      const u64 IH = pk(ih, ih), IH3 = pk(ih3, ih3);
      cr = spline_scalar<true>(c2, ih, ih3);
      for (; k <= k1; ++k) {
        O = add2(O, STEP);
        const u64 F = spline_over_r2(O, DR2, IH, NIH, IH3);
        SR = add2(SR, F);
        SZ = fma2(O, F, SZ);
      }
    } else {
      cr = spline_scalar<false>(c2, ih, 0.0f);
    }
    const int kg = min(kw, n0);
    for (; k <= kg; ++k) {
      O = add2(O, STEP);
      const u64 F = spline_outer_over_r2(O, DR2, NIH);
      SR = add2(SR, F);
      SZ = fma2(O, F, SZ);
    }
  } else {
    const float ri = rsq(c2);
    cr = ri * ri * ri;
  }
  // Newtonian pairs k .. n0: the first (count mod 4) enter a straight run
  // part-way, the rest go in fours
  const int cnt = n0 + 1 - k;
  if (N0 > 0 && k == 1) {  // no softened pair: the whole fixed range, unrolled
#pragma unroll
    for (int q = 0; q < N0; ++q) newton_pair(O, STEP, DR2, SR, SZ);
    float s0, s1, z0, z1;
    upk(SR, s0, s1);
    upk(SZ, z0, z1);
    sr = (s0 + s1) + cr;
    sz = (z0 + z1) + dz * cr;
    return;
  }
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
  float s0, s1, z0, z1;
  upk(SR, s0, s1);
  upk(SZ, z0, z1);
  sr = (s0 + s1) + cr;
  sz = (z0 + z1) + dz * cr;
}

#ifndef STEPS_SURR_N0_FIXED
#define STEPS_SURR_N0_FIXED 1  // compile the n0 = 4 near range unrolled beside the general one
#endif

// Per-pair state carried across the network: the image sums are affine in
// the network outputs, sr = a0 + b0 y0 and sz = a1 + b1 y1 (near images, tail
// base, envelope, sign(dz) and the output scaling folded in), plus the inputs.
struct SurrPair {
  float a0, b0, a1, b1;
  float u[3];  // network inputs
};

// Stage A: near images |k| <= n0 exactly (the tiered image walk of
// pair_fp32.cuh without the edge image), the tail base, the envelope and the
// network inputs. kw: warp-uniform spline bound. INF: the infinite window.
// RAW: the frame of the tail: 0 the base and envelope (the learned tail and
// the residual tables, n0 >= 1), 1 none (the nearest-image table, n0 = 0, holds
// the tail sums themselves), -1 chosen at run time from S.n0.
template <bool INF = false, int RAW = 0>
__device__ __forceinline__ void surr_stage_a(float dR2, float dz, float hh, int n_cut, int kw, const SurrConst& S,
                                             SurrPair& P) {
  (void)n_cut;  // the finite window's far end comes in S.fnh
  float sr, sz;
#if STEPS_SURR_N0_FIXED
  if (S.n0 == 4)  // the near range of the learned-tail workloads, unrolled
    near_images_fp32<4>(dR2, dz, hh, 4, kw, sr, sz);
  else
#endif
    near_images_fp32(dR2, dz, hh, S.n0, kw, sr, sz);
  // tail base and envelope (|dz|; z part gets sign(dz))
  const float adz = fabsf(dz), A = S.A;
  float br, bz, il1;
  if (RAW > 0 || (RAW < 0 && S.n0 == 0)) {
    br = 0.0f;
    bz = 0.0f;
    il1 = 1.0f;
  } else if (INF) {
    tail_base_inf_fp32(dR2, A + adz, A - adz, br, bz, il1);
  } else {
    // far ends: + side (n_cut - 1) + 1/2 + |dz|; - side at n_cut + 1/2 - |dz| when
    // dz != 0 (the edge image n_cut belongs to it), else n_cut - 1/2
    const float hb = (adz > 0.0f ? S.fnh + 1.0f : S.fnh) - adz;
    tail_base_fp32(dR2, A + adz, A - adz, S.fnh + adz, hb, br, bz, il1);
  }
  const float e = il1 * il1;
  const float er = e * e * e;
  const float sg = dz > 0.0f ? 1.0f : (dz < 0.0f ? -1.0f : 0.0f);
  const float ez = sg * (e * e * il1);  // sign(dz) E_z: the z part of the tail is odd in dz
  // tail = base + E (y sc + mu)
  P.a0 = fmaf(er, S.mu0, sr + br);
  P.b0 = er * S.sc0;
  P.a1 = fmaf(ez, S.mu1, fmaf(sg, bz, sz));
  P.b1 = ez * S.sc1;
  const float dR = dR2 * rsq(fmaxf(dR2, 1e-30f));
  P.u[0] = fmaf(fminf(dR, S.dR_max), S.two_inv_dR_max, -1.0f);
  P.u[1] = fmaf(adz, 4.0f, -1.0f);
  P.u[2] = fmaf(fminf(hh, A), S.two_over_A, -1.0f);
}

// Stage A of a pair that no lane of the warp has inside its softening support
// (kw < 0), with the near range n0 = 4 fixed: the same arithmetic as
// surr_stage_a on that path (centre image, then the four image pairs +-k
// packed, then the tail base, envelope and inputs), written without a branch so
// that a caller can place it in one straight run with the network.
template <bool INF = false>
__device__ __forceinline__ void surr_stage_a_far4(float dR2, float dz, float hh, const SurrConst& S, SurrPair& P) {
  const float adz = fabsf(dz), A = S.A;
  const float dR = dR2 * rsq(fmaxf(dR2, 1e-30f));
  P.u[0] = fmaf(fminf(dR, S.dR_max), S.two_inv_dR_max, -1.0f);
  P.u[1] = fmaf(adz, 4.0f, -1.0f);
  P.u[2] = fmaf(fminf(hh, A), S.two_over_A, -1.0f);
  // near images |k| <= 4, all Newtonian
  const u64 DR2 = pk(dR2, dR2);
  const u64 STEP = pk(1.0f, -1.0f);
  u64 O = pk(dz, dz);
  u64 SR = pk(0.0f, 0.0f), SZ = pk(0.0f, 0.0f);
  const float ri = rsq(fmaf(dz, dz, dR2));
  const float cr = ri * ri * ri;
#pragma unroll
  for (int q = 0; q < 4; ++q) newton_pair(O, STEP, DR2, SR, SZ);
  float s0, s1, z0, z1;
  upk(SR, s0, s1);
  upk(SZ, z0, z1);
  const float sr = (s0 + s1) + cr;
  const float sz = (z0 + z1) + dz * cr;
  // tail base and envelope, as in surr_stage_a
  float br, bz, il1;
  if (INF) {
    tail_base_inf_fp32(dR2, A + adz, A - adz, br, bz, il1);
  } else {
    const float hb = (adz > 0.0f ? S.fnh + 1.0f : S.fnh) - adz;
    tail_base_fp32(dR2, A + adz, A - adz, S.fnh + adz, hb, br, bz, il1);
  }
  const float e = il1 * il1;
  const float er = e * e * e;
  const float sg = dz > 0.0f ? 1.0f : (dz < 0.0f ? -1.0f : 0.0f);
  const float ez = sg * (e * e * il1);
  P.a0 = fmaf(er, S.mu0, sr + br);
  P.b0 = er * S.sc0;
  P.a1 = fmaf(ez, S.mu1, fmaf(sg, bz, sz));
  P.b1 = ez * S.sc1;
}

// Stage C: tail = base + envelope x network output, plus the exact spline
// correction of tail images inside some lane's softening support.
// The separation is recomputed from the tile (same arithmetic, same values)
// on that rare path rather than kept live across the network. INF: the
// infinite window (no window bound, no edge image).
template <bool INF = false>
__device__ __forceinline__ void surr_stage_c(const IParticle& I, const float4& A, const float4& B, int n_cut, int kw,
                                             const SurrConst& S, const SurrPair& P, float y0, float y1, float& sr,
                                             float& sz) {
  const int n0 = S.n0;
  sr = fmaf(P.b0, y0, P.a0);
  sz = fmaf(P.b1, y1, P.a1);
  if (kw > n0) {
    float dx, dy, dz, dR2, hh;
    pair_separation(I, A, B, dx, dy, dz, dR2, hh);
    const u64 DR2 = pk(dR2, dR2);
    const u64 STEP = pk(1.0f, -1.0f);
    const float ih = rcp_approx(hh), ih3 = ih * ih * ih;
    const u64 IH = pk(ih, ih), NIH = pk(-ih, -ih), IH3 = pk(ih3, ih3);
    const int kt = INF ? kw : min(kw, n_cut - 1);
    u64 CR = pk(0.f, 0.f), CZ = pk(0.f, 0.f);
    u64 O = pk(dz + (float)n0, dz - (float)n0);
    for (int kk = n0 + 1; kk <= kt; ++kk) {
      O = add2(O, STEP);
      const u64 R2 = fma2(O, O, DR2);
      float ra, rb;
      upk(R2, ra, rb);
      const u64 RI = pk(rsq(ra), rsq(rb));
      const u64 N3 = mul2(mul2(RI, RI), RI);
      const u64 D = fma2(N3, pk(-1.0f, -1.0f), spline_over_r2(O, DR2, IH, NIH, IH3));
      CR = add2(CR, D);
      CZ = fma2(O, D, CZ);
    }
    if (!INF && kw >= n_cut) {  // the edge image as well
      const float oe = dz - copysignf((float)n_cut, dz);
      const u64 OE = pk(oe, oe);
      const float r2 = fmaf(oe, oe, dR2);
      const float ri = rsq(r2);
      float fa, fb;
      upk(spline_over_r2(OE, DR2, IH, NIH, IH3), fa, fb);
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

#ifndef STEPS_SURR_NJ
#define STEPS_SURR_NJ 2  // values of j per network call (independent mma chains per warp)
#endif
static_assert(STEPS_KAHAN_GROUP % STEPS_SURR_NJ == 0, "a Kahan group holds whole network calls");

// One j-tile of pairs for one i (shared by the stream-K and the subset kernels).
// The surrogate form handles two j per network call; INF: the infinite window.
template <bool KAHAN, bool SURR, bool INF = false>
__device__ __forceinline__ void pair_tile(const IParticle& I, const float4* sA, const float4* sB, int jn, int self,
                                          int n_cut, float fnc, const SurrW& W, uint32_t* ibuf, const SurrConst& S,
                                          float& sx,
                                          float& sy, float& sz, float& cx, float& cy, float& cz) {
  constexpr int STEPJ = SURR ? STEPS_SURR_NJ : 1;
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
          surr_stage_a<INF>(dR2[jj], dz[jj], hh[jj], n_cut, kw[jj], S, P[jj]);
          u[jj][0] = P[jj].u[0];
          u[jj][1] = P[jj].u[1];
          u[jj][2] = P[jj].u[2];
        }
        mlp_warp<STEPJ>(W, ibuf, u, y);
#pragma unroll
        for (int jj = 0; jj < STEPJ; ++jj) {
          const int kk = min(k + jj, ke - 1);
          surr_stage_c<INF>(I, sA[kk], sB[kk], n_cut, kw[jj], S, P[jj], y[jj][0], y[jj][1], sr[jj], szz[jj]);
        }
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

template <bool KAHAN, bool INF = false>
__global__ void __launch_bounds__(kBI, STEPS_SURR_MIN_BLOCKS)
pair_fp32_surr_kernel(const float4* __restrict__ jA, const float4* __restrict__ jB, int n, int n_cut, long long U,
                      int NT, int C, const SurrLane* __restrict__ wl, SurrConst S, double* __restrict__ part,
                      int b0 = 0) {
  __shared__ float4 sA[kBJ];
  __shared__ float4 sB[kBJ];
  // weight fragments stay in shared memory (word-major, conflict-free) and are
  // read where the mma needs them, which leaves registers for resident warps
  __shared__ __align__(16) uint32_t sWT[32 * kSurrStride];
  __shared__ __align__(16) uint32_t sIn[kBI / 32][STEPS_SURR_NJ * kInWords];
  uint32_t* ibuf = sIn[threadIdx.x >> 5];
  mlp_zero_inputs<STEPS_SURR_NJ>(ibuf);
  stage_surr_weights(wl, sWT);
  const SurrW W{sWT + (threadIdx.x & 31) * kSurrStride};
  const int c = blockIdx.x;
  const long long u0 = (long long)c * U / C;
  const long long u1 = (long long)(c + 1) * U / C;
  const float fnc = (float)n_cut;
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
      pair_tile<KAHAN, true, INF>(I, sA, sB, kBJ, i - t * kBJ, n_cut, fnc, W, ibuf, S, sx, sy, sz, cx, cy,
                                  cz);
    }
    double* dst = part + ((long long)lb + c) * 3 * kBI;
    dst[threadIdx.x] = (double)sx - (KAHAN ? (double)cx : 0.0);
    dst[kBI + threadIdx.x] = (double)sy - (KAHAN ? (double)cy : 0.0);
    dst[2 * kBI + threadIdx.x] = (double)sz - (KAHAN ? (double)cz : 0.0);
    u += t1 - t0;
  }
}

// Subset kernel (acceptance checks): CTA (bx, by) takes listed i-particles
// [bx * kBI, +kBI) against j-tiles [by * tpc, (by + 1) * tpc); partials
// part[by][3][ni]. The listed indices are internal and may repeat. INF: the
// surrogate of the infinite window.
template <bool KAHAN, bool SURR, bool INF = false>
__global__ void __launch_bounds__(kBI, 3)
pair_fp32_subset_kernel(const float4* __restrict__ jA, const float4* __restrict__ jB, int n, int n_cut,
                        const int64_t* __restrict__ idx, int ni, int tpc, const SurrLane* __restrict__ wl, SurrConst S,
                        double* __restrict__ part) {
  __shared__ float4 sA[kBJ];
  __shared__ float4 sB[kBJ];
  __shared__ __align__(16) uint32_t sWT[32 * kSurrStride];
  __shared__ __align__(16) uint32_t sIn[kBI / 32][SURR ? STEPS_SURR_NJ * kInWords : 4];
  uint32_t* ibuf = sIn[threadIdx.x >> 5];
  if (SURR) {
    mlp_zero_inputs<STEPS_SURR_NJ>(ibuf);
    stage_surr_weights(wl, sWT);
  }
  const SurrW W{sWT + (threadIdx.x & 31) * kSurrStride};
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
    pair_tile<KAHAN, SURR, INF>(I, sA, sB, kBJ, i - t * kBJ, n_cut, (float)n_cut, W, ibuf, S, sx, sy, sz, cx,
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
