// Symmetric evaluation of the pair sum (Newton's third law). The window of
// eq. ForceCylindrical is symmetric: the reverse pair (j, i) sees the images of
// (i, j) mirrored, with the same dR and h_i + h_j, so its sums are sr(j, i) =
// sr(i, j) and sz(j, i) = -sz(i, j), and the force j feels from i is the
// opposite of the force i feels from j up to the two masses. Each unordered
// pair is therefore evaluated once: with v = (dx sr, dy sr, sz),
//   S_i += m_j v,   S_j -= m_i v,
// where S is the sum that the FP32 pair kernels produce per particle (scaled by
// -G / L^2 in the finalize step).
//
// Work split. The (i-block b, j-tile t) units with t >= b (the upper triangle of
// the block grid, NB (NB + 1) / 2 units) are laid out b-major, and every CTA
// takes an equal contiguous range, as in the stream-K split of pair_fp32.cuh.
// A diagonal unit (t == b) evaluates all ordered pairs of its block for the i
// side only (the self pair adds exact zeros); an off-diagonal unit evaluates
// its 128 x 128 pairs once and adds each to both sides.
//
// The j side. In each group of 32 j-slots of a tile, lane l pairs its i with
// slot (l + s) mod 32 at step s, so every slot meets every lane once in 32
// steps. A lane keeps the running sum of m_i v for the slot it holds and passes
// it to lane l - 1 after each step (JRing: one shuffle per component and step);
// after the group lane l holds the warp's whole sum of slot (l + 31) mod 32 and
// writes it to the warp's row of a shared array. (STEPS_SYM_RING = 0 keeps all
// lanes on one slot and reduces each slot over the warp with shuffles instead.)
// After the tile, thread q adds the four warps' sums of j-slot q in warp order.
//
// Accumulation. The i-side sum of a CTA's range (FP32, Kahan-compensated as in
// the row kernels) and the j-side sum of a unit are converted to 64-bit fixed
// point, value * 2^S rounded to an integer, and added with integer atomics into
// one accumulator per particle and component. Integer addition is associative,
// so the result does not depend on the order in which CTAs finish: the force
// evaluation stays deterministic and bit-reproducible. 2^S is chosen on the host
// from a bound on |S_i| (total mass times the largest softened force); a value
// beyond 2^62 / 2^S sets an error bit instead of wrapping.
#pragma once
#include <cstdint>

#include "pair_fp32.cuh"
#include "surrogate_pair.cuh"
#include "tail_table.cuh"

namespace steps {

constexpr int kErrFixRange = 32;  // a pair sum left the range of the fixed-point accumulators
constexpr int kErrIndex = 64;     // (index-checked builds) an index left its buffer

// Index-checked builds (STEPS_DEBUG_INDEX=1) check every computed index of the
// symmetric kernels' shared and global accesses against its buffer; an index
// outside is recorded in g_index_err and clamped into the buffer, so that
// control flow (and every warp-collective call) stays the same. The host folds
// the record into the device error word (kErrIndex). Release builds compile
// the checks away.
#ifndef STEPS_DEBUG_INDEX
#define STEPS_DEBUG_INDEX 0
#endif
#if STEPS_DEBUG_INDEX
__device__ unsigned int g_index_err;
#endif

__device__ __forceinline__ long long checked_index(long long v, long long size) {
#if STEPS_DEBUG_INDEX
  if (v < 0 || v >= size) {
    atomicOr(&g_index_err, 1u);
    return v < 0 ? 0 : size - 1;
  }
#else
  (void)size;
#endif
  return v;
}
constexpr int kJRow = 3 * kBJ;    // floats of one warp's j-side row: [kBJ][3]

// Fixed-point accumulators (two's complement in unsigned words, unit
// 1 / scale) and the error word. Unsharded (world == 0): acc[3][n]. When the
// rows are sharded across world ranks (balanced contiguous ranges of 128-row
// blocks: the first `extra` ranks own base + 1 blocks, the others base),
// acc[world][3][chunk], rank-major, so that a reduce-scatter over the ranks
// hands each rank the sums of its own rows.
struct FixAcc {
  unsigned long long* acc;
  int n;
  double scale;
  int* err;
  int world, base, extra, chunk;
};

__device__ __forceinline__ long long fix_index(const FixAcc& F, int c, int i) {
  if (F.world == 0) return (long long)c * F.n + i;
  const int b = i / kBI, big = F.extra * (F.base + 1);
  const int r = b < big ? b / (F.base + 1) : F.extra + (b - big) / F.base;
  const int first = (r < F.extra ? r * (F.base + 1) : big + (r - F.extra) * F.base) * kBI;
  return ((long long)r * 3 + c) * F.chunk + (i - first);
}

__device__ __forceinline__ void fix_add(const FixAcc& F, int c, int i, double v) {
  const double q = v * F.scale;
  if (!(fabs(q) < 4.0e18)) {  // beyond 2^62 (or not finite): flag it, never wrap
    atomicOr(F.err, kErrFixRange);
    return;
  }
  const long long size = F.world == 0 ? 3LL * F.n : 3LL * F.world * F.chunk;
  atomicAdd(F.acc + checked_index(fix_index(F, c, i), size), (unsigned long long)__double2ll_rn(q));
}

// Offset of row b of the upper triangle (units t = b .. NB - 1 per row).
__host__ __device__ __forceinline__ long long tri_off(int b, int NB) {
  return (long long)b * NB - (long long)b * (b - 1) / 2;
}

// The row b of unit u (tri_off(b) <= u < tri_off(b + 1)).
__device__ __forceinline__ int tri_row(long long u, int NB) {
  const double h = 2.0 * NB + 1.0;
  int b = (int)(0.5 * (h - sqrt(fmax(h * h - 8.0 * (double)u, 0.0))));
  b = max(0, min(b, NB - 1));
  while (b > 0 && tri_off(b, NB) > u) --b;
  while (b + 1 < NB && tri_off(b + 1, NB) <= u) ++b;
  return b;
}

// Warp sums of the j-side vectors of two j (w0 for j-slot k, w1 for k + 1)
// into the warp's shared row (lanes 0 and 16 write).
__device__ __forceinline__ void jside_pair(const float (&w0)[3], const float (&w1)[3], float* row, int k) {
  const int lane = threadIdx.x & 31;
  const bool hi = (lane & 16) != 0;
  float r[3];
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    const float send = hi ? w0[c] : w1[c];
    float keep = hi ? w1[c] : w0[c];
    keep += __shfl_xor_sync(0xffffffffu, send, 16);
    keep += __shfl_xor_sync(0xffffffffu, keep, 8);
    keep += __shfl_xor_sync(0xffffffffu, keep, 4);
    keep += __shfl_xor_sync(0xffffffffu, keep, 2);
    keep += __shfl_xor_sync(0xffffffffu, keep, 1);
    r[c] = keep;
  }
  if ((lane & 15) == 0) {
    float* d = row + 3 * checked_index(k + (hi ? 1 : 0), kBJ);
    d[0] = r[0];
    d[1] = r[1];
    d[2] = r[2];
  }
}

// The j-side vector m_i v of one pair.
__device__ __forceinline__ void jside_vec(float mi, float dx, float dy, float sr, float sz, float (&w)[3]) {
  const float misr = mi * sr;
  w[0] = dx * misr;
  w[1] = dy * misr;
  w[2] = mi * sz;
}

#ifndef STEPS_SYM_RING
#define STEPS_SYM_RING 1  // 1: the j side is carried around the warp (JRing); 0: reduced per two j (jside_pair)
#endif

// The j-slot that this lane pairs with at step k of a tile. With the ring, in
// each group of 32 slots lane l takes slot (l + k) mod 32 at step k, so every
// slot meets every lane once in 32 steps; otherwise all lanes take slot k.
__device__ __forceinline__ int jslot(int k) {
#if STEPS_SYM_RING
  return (int)checked_index((k & ~31) | ((k + (int)threadIdx.x) & 31), kBJ);
#else
  return (int)checked_index(k, kBJ);
#endif
}

// The j side carried around the warp: a lane keeps the running sum of the slot
// it holds, adds its pair's vector, and takes over the sum of lane l + 1 (the
// slot it holds at the next step). After the last step of a group no shift is
// made: lane l then holds the whole warp's sum of slot (l + 31) mod 32, one
// shuffle per component and step instead of a 32-lane reduction per slot.
struct JRing {
  float a[3] = {0.f, 0.f, 0.f};
  __device__ __forceinline__ void take(const float (&w)[3], bool shift) {
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      a[c] += w[c];
      if (shift) a[c] = __shfl_sync(0xffffffffu, a[c], (threadIdx.x + 1) & 31);
    }
  }
  // k: the group's last step
  __device__ __forceinline__ void flush(float* row, int k) {
    float* d = row + 3 * jslot(k);
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      d[c] = a[c];
      a[c] = 0.f;
    }
  }
};

// The j side of the two steps k, k + 1 (k even) into the warp's row.
__device__ __forceinline__ void jside_two(JRing& ring, const float (&w0)[3], const float (&w1)[3], float* row,
                                          int k) {
#if STEPS_SYM_RING
  const bool last = ((k + 2) & 31) == 0;
  ring.take(w0, true);
  ring.take(w1, !last);
  if (last) ring.flush(row, k + 1);
#else
  (void)ring;
  jside_pair(w0, w1, row, k);
#endif
}

// ---- tile functions: all pairs of one i with the kBJ j of a shared tile -------
// They add m_j v to the i-side Kahan sums and, when sym is set (an
// off-diagonal unit), write the warp's j-side sums of every j-slot to row.

#ifndef STEPS_PLAIN_JUNROLL
#define STEPS_PLAIN_JUNROLL 1  // unroll of the two-j steps of a Kahan group (plain image sum)
#endif
constexpr int kPlainJUnroll = STEPS_PLAIN_JUNROLL;

// Plain image sum (pair_fp32.cuh), two j per step.
template <bool KAHAN>
__device__ __forceinline__ void sym_tile_plain(const IParticle& I, float mi, const float4* sA, const float4* sB,
                                               bool sym, float* row, int n_cut, float fnc, float& sx, float& sy,
                                               float& sz, float& cx, float& cy, float& cz) {
  JRing ring;
#pragma unroll 1
  for (int k0 = 0; k0 < kBJ; k0 += STEPS_KAHAN_GROUP) {
    float gx = 0.f, gy = 0.f, gz = 0.f;
#pragma unroll(kPlainJUnroll)
    for (int k = k0; k < k0 + STEPS_KAHAN_GROUP; k += 2) {
      float w[2][3];
#pragma unroll
      for (int jj = 0; jj < 2; ++jj) {
        const int q = jslot(k + jj);
        const float4 A = sA[q];
        const float4 B = sB[q];
        float dx, dy, dz, dR2, hh;
        int kw;
        pair_geometry(I, A, B, dx, dy, dz, dR2, hh, kw);
        float sr, szz;
#if STEPS_NCUT_FIXED
        if (n_cut == 16)
          pair_images_fp32<true, 16>(dR2, dz, hh, 16, fnc, kw, sr, szz);
        else if (n_cut == 64)
          pair_images_fp32<true, 64>(dR2, dz, hh, 64, fnc, kw, sr, szz);
        else
#endif
          pair_images_fp32(dR2, dz, hh, n_cut, fnc, kw, sr, szz);
        const float msr = A.w * sr;
        gx = fmaf(dx, msr, gx);
        gy = fmaf(dy, msr, gy);
        gz = fmaf(A.w, szz, gz);
        jside_vec(mi, dx, dy, sr, szz, w[jj]);
      }
      if (sym) jside_two(ring, w[0], w[1], row, k);
    }
    acc<KAHAN>(sx, cx, gx);
    acc<KAHAN>(sy, cy, gy);
    acc<KAHAN>(sz, cz, gz);
  }
}

// One network call of the learned tail for the NJ steps k .. k + NJ - 1 (slots
// jslot(k + jj)): the i-side group sums and the j-side vectors w. FAR4 (near
// range n0 = 4): stage A of every pair is first taken as if no lane's pair were
// inside its softening support (surr_stage_a_far4, no branch), so that the
// geometry, stage A and the network form one straight run in which the
// scheduler interleaves the tensor-core chain with the FP32 and MUFU work. A
// step where some lane's pair is inside its support (kw >= 0, warp-uniform)
// redoes stage A of that pair with the spline tiers after the network, from
// the same separation, which gives the tiered call's values bit for bit.
template <int NJ, bool INF, bool FAR4>
__device__ __forceinline__ void surr_call(const IParticle& I, float mi, const float4* sA, const float4* sB, int k,
                                          int self, int n_cut, const SurrW& W, uint32_t* ibuf, const SurrConst& S,
                                          float& gx, float& gy, float& gz, float (*w)[3]) {
  float dx[NJ], dy[NJ], mj[NJ];
  int kw[NJ];
  SurrPair P[NJ];
  float u[NJ][3], y[NJ][2];
  int q[NJ];
#pragma unroll
  for (int jj = 0; jj < NJ; ++jj) {
    q[jj] = jslot(k + jj);
    const float4 A = sA[q[jj]];
    const float4 B = sB[q[jj]];
    float dz, dR2, hh;
    pair_geometry(I, A, B, dx[jj], dy[jj], dz, dR2, hh, kw[jj]);
    mj[jj] = (q[jj] == self) ? 0.0f : A.w;
    if (FAR4)
      surr_stage_a_far4<INF>(dR2, dz, hh, S, P[jj]);
    else
      surr_stage_a<INF>(dR2, dz, hh, n_cut, kw[jj], S, P[jj]);
    u[jj][0] = P[jj].u[0];
    u[jj][1] = P[jj].u[1];
    u[jj][2] = P[jj].u[2];
  }
  mlp_warp<NJ>(W, ibuf, u, y);
  if (FAR4) {
#pragma unroll
    for (int jj = 0; jj < NJ; ++jj) {
      if (kw[jj] >= 0) {
        float ddx, ddy, dz, dR2, hh;
        pair_separation(I, sA[q[jj]], sB[q[jj]], ddx, ddy, dz, dR2, hh);
        surr_stage_a<INF>(dR2, dz, hh, n_cut, kw[jj], S, P[jj]);
      }
    }
  }
#pragma unroll
  for (int jj = 0; jj < NJ; ++jj) {
    float sr, szz;
    surr_stage_c<INF>(I, sA[q[jj]], sB[q[jj]], n_cut, kw[jj], S, P[jj], y[jj][0], y[jj][1], sr, szz);
    const float msr = mj[jj] * sr;
    gx = fmaf(dx[jj], msr, gx);
    gy = fmaf(dy[jj], msr, gy);
    gz = fmaf(mj[jj], szz, gz);
    jside_vec(mi, dx[jj], dy[jj], sr, szz, w[jj]);
  }
}

#ifndef STEPS_SURR_UNROLL
#define STEPS_SURR_UNROLL 1  // unroll of the two-j steps of a Kahan group (learned tail)
#endif
constexpr int kSurrUnroll = STEPS_SURR_UNROLL;

// Learned tail (surrogate_pair.cuh): STEPS_SURR_NJ j per network call, the
// j side reduced two j at a time. FAR4: the straight-run calls (near range
// n0 = 4), which the host takes when every softening support lies within half
// a period (h_i + h_j < L / 2): only the centre image of a pair can then be
// softened, and the steps that redo a pair stay rare. Loads with wider
// supports take the tiered calls throughout.
template <bool KAHAN, bool INF, bool FAR4>
__device__ __forceinline__ void sym_tile_surr(const IParticle& I, float mi, const float4* sA, const float4* sB,
                                              bool sym, float* row, int self, int n_cut, const SurrW& W,
                                              uint32_t* ibuf, const SurrConst& S, float& sx, float& sy, float& sz,
                                              float& cx, float& cy, float& cz) {
  static_assert(STEPS_SURR_NJ == 1 || STEPS_SURR_NJ == 2, "one or two j per network call");
  JRing ring;
#pragma unroll 1
  for (int k0 = 0; k0 < kBJ; k0 += STEPS_KAHAN_GROUP) {
    float gx = 0.f, gy = 0.f, gz = 0.f;
#pragma unroll(kSurrUnroll)
    for (int k = k0; k < k0 + STEPS_KAHAN_GROUP; k += 2) {
      float w[2][3];
      if (STEPS_SURR_NJ == 2) {
        surr_call<2, INF, FAR4>(I, mi, sA, sB, k, self, n_cut, W, ibuf, S, gx, gy, gz, w);
      } else {
        surr_call<1, INF, FAR4>(I, mi, sA, sB, k, self, n_cut, W, ibuf, S, gx, gy, gz, w);
        surr_call<1, INF, FAR4>(I, mi, sA, sB, k + 1, self, n_cut, W, ibuf, S, gx, gy, gz, w + 1);
      }
      if (sym) jside_two(ring, w[0], w[1], row, k);
    }
    acc<KAHAN>(sx, cx, gx);
    acc<KAHAN>(sy, cy, gy);
    acc<KAHAN>(sz, cz, gz);
  }
}

// Correction-table tail (tail_table.cuh), two j per step; READ: the table read
// (the exact reads belong to the nearest-image table, n0 = 0, stored raw).
// FAR4: as for the learned tail, the straight-run stage A of both pairs and
// their table reads form one run (the fetches are issued as soon as the inputs
// exist and return while the near images and the base are computed); a pair
// whose step is softened is redone with the spline tiers after the reads.
template <bool KAHAN, bool INF, int READ, bool FAR4>
__device__ __forceinline__ void sym_tile_table(const IParticle& I, float mi, const float4* sA, const float4* sB,
                                               bool sym, float* row, int self, int n_cut, const SurrConst& S,
                                               const TableTail& T, float& sx, float& sy, float& sz, float& cx,
                                               float& cy, float& cz) {
  constexpr int RAW = READ >= kReadCicExact ? 1 : 0;
  static_assert(!(FAR4 && RAW), "the straight run belongs to the residual tables (n0 = 4)");
  JRing ring;
#pragma unroll 1
  for (int k0 = 0; k0 < kBJ; k0 += STEPS_KAHAN_GROUP) {
    float gx = 0.f, gy = 0.f, gz = 0.f;
#pragma unroll 1
    for (int k = k0; k < k0 + STEPS_KAHAN_GROUP; k += 2) {
      float w[2][3];
      if (FAR4) {
        int q[2], kw[2];
        float dx[2], dy[2];
        SurrPair P[2];
        float2 r[2];
#pragma unroll
        for (int jj = 0; jj < 2; ++jj) {
          q[jj] = jslot(k + jj);
          float dz, dR2, hh;
          pair_geometry(I, sA[q[jj]], sB[q[jj]], dx[jj], dy[jj], dz, dR2, hh, kw[jj]);
          surr_stage_a_far4<INF>(dR2, dz, hh, S, P[jj]);
          r[jj] = table_read<READ>(T, P[jj].u[0], P[jj].u[1]);
        }
#pragma unroll
        for (int jj = 0; jj < 2; ++jj) {
          const float4 A = sA[q[jj]];
          const float4 B = sB[q[jj]];
          if (kw[jj] >= 0) {
            float ddx, ddy, dz, dR2, hh;
            pair_separation(I, A, B, ddx, ddy, dz, dR2, hh);
            surr_stage_a<INF>(dR2, dz, hh, n_cut, kw[jj], S, P[jj]);
          }
          float sr, szz;
          surr_stage_c<INF>(I, A, B, n_cut, kw[jj], S, P[jj], r[jj].x, r[jj].y, sr, szz);
          const float mj = (q[jj] == self) ? 0.0f : A.w;
          const float msr = mj * sr;
          gx = fmaf(dx[jj], msr, gx);
          gy = fmaf(dy[jj], msr, gy);
          gz = fmaf(mj, szz, gz);
          jside_vec(mi, dx[jj], dy[jj], sr, szz, w[jj]);
        }
      } else {
#pragma unroll
        for (int jj = 0; jj < 2; ++jj) {
          const int q = jslot(k + jj);
          const float4 A = sA[q];
          const float4 B = sB[q];
          float dx, dy, dz, dR2, hh;
          int kw;
          pair_geometry(I, A, B, dx, dy, dz, dR2, hh, kw);
          SurrPair P;
          surr_stage_a<INF, RAW>(dR2, dz, hh, n_cut, kw, S, P);
          const float2 r = table_read<READ>(T, P.u[0], P.u[1]);
          float sr, szz;
          surr_stage_c<INF>(I, A, B, n_cut, kw, S, P, r.x, r.y, sr, szz);
          const float mj = (q == self) ? 0.0f : A.w;
          const float msr = mj * sr;
          gx = fmaf(dx, msr, gx);
          gy = fmaf(dy, msr, gy);
          gz = fmaf(mj, szz, gz);
          jside_vec(mi, dx, dy, sr, szz, w[jj]);
        }
      }
      if (sym) jside_two(ring, w[0], w[1], row, k);
    }
    acc<KAHAN>(sx, cx, gx);
    acc<KAHAN>(sy, cy, gy);
    acc<KAHAN>(sz, cz, gz);
  }
}

// ---- the stream-K driver over the upper triangle -----------------------------
// tile(I, mi, sym, self, row, sx .. cz) evaluates one staged tile. sJ: the
// warps' j-side rows, [kBI / 32][kJRow] floats.
template <bool KAHAN, class Tile>
__device__ __forceinline__ void sym_stream_k(const float4* __restrict__ jA, const float4* __restrict__ jB, int n,
                                             int NB, long long Ua, long long U, int C, float4* sA, float4* sB,
                                             float* sJ, const FixAcc& F, Tile tile) {
  // the units [Ua, Ua + U) (all of them, or a rank's share), split over C CTAs
  const int c = blockIdx.x;
  const long long u0 = Ua + (long long)c * U / C;
  const long long u1 = Ua + (long long)(c + 1) * U / C;
  float* row = sJ + (threadIdx.x >> 5) * kJRow;
  long long u = u0;
  while (u < u1) {
    const int b = (int)checked_index(tri_row(u, NB), NB);
    const int t0 = (int)checked_index(b + (u - tri_off(b, NB)), NB);
    const int t1 = (int)min((long long)NB, (long long)t0 + (u1 - u));
    const int i = b * kBI + threadIdx.x;
    const IParticle I = load_i(jA, jB, min(i, n - 1));
    const float mi = i < n ? jA[i].w : 0.0f;  // rows past n add nothing to the j side
    float sx = 0.f, sy = 0.f, sz = 0.f, cx = 0.f, cy = 0.f, cz = 0.f;
    for (int t = t0; t < t1; ++t) {
      __syncthreads();
      load_tile(jA, jB, n, t, sA, sB);
      __syncthreads();
      const bool sym = t != b;
      tile(I, mi, sA, sB, sym, i - t * kBJ, row, sx, sy, sz, cx, cy, cz);
      if (sym) {
        __syncthreads();  // every warp's row is written
        const int j = t * kBJ + threadIdx.x;
        if (j < n) {
          float s0 = 0.f, s1 = 0.f, s2 = 0.f;
#pragma unroll
          for (int w = 0; w < kBI / 32; ++w) {
            const float* q = sJ + w * kJRow + 3 * threadIdx.x;
            s0 += q[0];
            s1 += q[1];
            s2 += q[2];
          }
          fix_add(F, 0, j, -(double)s0);
          fix_add(F, 1, j, -(double)s1);
          fix_add(F, 2, j, -(double)s2);
        }
      }
    }
    if (i < n) {
      fix_add(F, 0, i, (double)sx - (KAHAN ? (double)cx : 0.0));
      fix_add(F, 1, i, (double)sy - (KAHAN ? (double)cy : 0.0));
      fix_add(F, 2, i, (double)sz - (KAHAN ? (double)cz : 0.0));
    }
    u += t1 - t0;
  }
}

// ---- kernels ---------------------------------------------------------------
template <bool KAHAN>
__global__ void __launch_bounds__(kBI, STEPS_PLAIN_MIN_BLOCKS)
pair_sym_kernel(const float4* __restrict__ jA, const float4* __restrict__ jB, int n, int n_cut, int NB, long long Ua,
                long long U, int C, FixAcc F) {
  __shared__ float4 sA[kBJ];
  __shared__ float4 sB[kBJ];
  __shared__ float sJ[kBI / 32 * kJRow];
  const float fnc = (float)n_cut;
  sym_stream_k<KAHAN>(jA, jB, n, NB, Ua, U, C, sA, sB, sJ, F,
                      [&](const IParticle& I, float mi, const float4* a, const float4* bb, bool sym, int /*self*/,
                          float* row, float& sx, float& sy, float& sz, float& cx, float& cy, float& cz) {
                        sym_tile_plain<KAHAN>(I, mi, a, bb, sym, row, n_cut, fnc, sx, sy, sz, cx, cy, cz);
                      });
}

template <bool KAHAN, bool INF, bool FAR4 = false>
__global__ void __launch_bounds__(kBI, STEPS_SURR_MIN_BLOCKS)
pair_sym_surr_kernel(const float4* __restrict__ jA, const float4* __restrict__ jB, int n, int n_cut, int NB,
                     long long Ua, long long U, int C, const SurrLane* __restrict__ wl, SurrConst S, FixAcc F) {
  __shared__ float4 sA[kBJ];
  __shared__ float4 sB[kBJ];
  __shared__ float sJ[kBI / 32 * kJRow];
  __shared__ __align__(16) uint32_t sWT[32 * kSurrStride];
  __shared__ __align__(16) uint32_t sIn[kBI / 32][STEPS_SURR_NJ * kInWords];
  uint32_t* ibuf = sIn[threadIdx.x >> 5];
  mlp_zero_inputs<STEPS_SURR_NJ>(ibuf);
  stage_surr_weights(wl, sWT);
  const SurrW W{sWT + (threadIdx.x & 31) * kSurrStride};
  sym_stream_k<KAHAN>(jA, jB, n, NB, Ua, U, C, sA, sB, sJ, F,
                      [&](const IParticle& I, float mi, const float4* a, const float4* bb, bool sym, int self,
                          float* row, float& sx, float& sy, float& sz, float& cx, float& cy, float& cz) {
                        sym_tile_surr<KAHAN, INF, FAR4>(I, mi, a, bb, sym, row, self, n_cut, W, ibuf, S, sx, sy,
                                                        sz, cx, cy, cz);
                      });
}

template <bool KAHAN, bool INF, int READ, bool FAR4 = false>
__global__ void __launch_bounds__(kBI, STEPS_TABLE_MIN_BLOCKS)
pair_sym_table_kernel(const float4* __restrict__ jA, const float4* __restrict__ jB, int n, int n_cut, int NB,
                      long long Ua, long long U, int C, TableTail T, SurrConst S, FixAcc F) {
  __shared__ float4 sA[kBJ];
  __shared__ float4 sB[kBJ];
  __shared__ float sJ[kBI / 32 * kJRow];
  sym_stream_k<KAHAN>(jA, jB, n, NB, Ua, U, C, sA, sB, sJ, F,
                      [&](const IParticle& I, float mi, const float4* a, const float4* bb, bool sym, int self,
                          float* row, float& sx, float& sy, float& sz, float& cx, float& cy, float& cz) {
                        sym_tile_table<KAHAN, INF, READ, FAR4>(I, mi, a, bb, sym, row, self, n_cut, S, T, sx, sy, sz,
                                                         cx, cy, cz);
                      });
}

}  // namespace steps
