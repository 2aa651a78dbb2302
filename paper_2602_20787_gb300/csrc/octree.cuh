// Octree force (arXiv 2602.20787, Sect. 2.4 "Octree"): a Barnes-Hut tree of
// the S1xR2 volume, re-drawn in a random frame at every force evaluation.
//
// Frame. x' = c x - s y, y' = s x + c y (c, s = cos, sin phi), z' = z + zeta
// (minus L when >= L). The root is a cube of side S = 2 max(L, 2 R_sim) centred
// at (0, 0, L/2); normalised coordinates u = (x'/S + 1/2, y'/S + 1/2,
// (z' - L/2)/S + 1/2) lie in [0, 1) and are rounded to FP32. 21 bits per axis
// give a 63-bit Morton key (x bit b at key bit 3b + 2, y at 3b + 1, z at 3b).
//
// Build (all on the GPU). The keys are sorted by a stable LSD radix sort of
// eight 8-bit digits from caller order, so equal keys keep caller order. The
// tree is built level by level from the root: an active node's eight child
// ranges are found by binary search in the sorted keys, and one scan numbers
// the non-empty children (consecutively per parent) and the next level's
// active nodes (more than `leaf` particles, depth < 21). Moments are summed
// bottom-up in FP64, level by level: mass, centre of mass (x, y in the
// particles' frame, z in the tree frame and shifted back by zeta) and the
// largest softening. Each node is packed as a pseudo-particle in the layout of
// the pair kernels (hi/lo position over L, mass, h/L).
//
// Walk. One warp per group of 32 consecutive particles in key order, all lanes
// on one shared stack. A node is opened for the group when any lane opens it:
// s^2 >= theta^2 d^2, or |d| - (sqrt(3)/2) s <= hu_i + hu_max (d: offset of u
// from the node centre with z wrapped to the nearest image, hu = h / S). The
// test is evaluated in FP32 with exactly rounded operations in the order
// written, so it is reproducible off the GPU. An accepted node, or the
// particles of an opened leaf, are appended to the warp's interaction list in
// shared memory; full lists are evaluated by all 32 lanes with the pair form
// of the correction-table tail over the infinite window (near images
// |k| <= n0 exact, the rest from the table), exactly as the direct kernel
// evaluates a j-tile.
#pragma once
#include <cstdint>

#include "tail_table.cuh"

namespace steps {

constexpr int kTreeDepth = 21;
constexpr int kSortThreads = 256;
constexpr int kSortRounds = 8;
constexpr int kSortTile = kSortThreads * kSortRounds;  // keys per sort tile
#ifndef STEPS_TREE_WARPS
#define STEPS_TREE_WARPS 4    // groups (warps) per CTA of the walk
#endif
#ifndef STEPS_TREE_LIST
#define STEPS_TREE_LIST 128   // interaction-list entries per warp (>= 64)
#endif
constexpr int kWalkWarps = STEPS_TREE_WARPS;
constexpr int kWalkStack = 160;                        // >= 7 * 21 + 1 pushes of a depth-first walk
constexpr int kWalkList = STEPS_TREE_LIST;
static_assert(kWalkList >= 64, "a list must take a node and a 32-particle chunk after a flush check");

struct TreeFrame {
  double c, s, zeta, L, halfL, invS;
};

struct TreeCrit {
  float Lu, hLu, th2;  // period and half period in root units (infinite for R^3), theta^2
};

// The R^3 frame (Sect. 2.4): the domain centre moved to cen, the frame rotated
// by the matrix R (row-major), root side S = 4 R_sim centred at cen.
struct TreeFrame3 {
  double cen[3], R[9], invS;
};

__device__ __forceinline__ uint64_t spread3(uint32_t v) {
  uint64_t x = v & 0x1fffffu;
  x = (x | (x << 32)) & 0x1f00000000ffffull;
  x = (x | (x << 16)) & 0x1f0000ff0000ffull;
  x = (x | (x << 8)) & 0x100f00f00f00f00full;
  x = (x | (x << 4)) & 0x10c30c30c30c30c3ull;
  x = (x | (x << 2)) & 0x1249249249249249ull;
  return x;
}

__device__ __forceinline__ uint32_t compact3(uint64_t x) {
  x &= 0x1249249249249249ull;
  x = (x | (x >> 2)) & 0x10c30c30c30c30c3ull;
  x = (x | (x >> 4)) & 0x100f00f00f00f00full;
  x = (x | (x >> 8)) & 0x1f0000ff0000ffull;
  x = (x | (x >> 16)) & 0x1f00000000ffffull;
  x = (x | (x >> 32)) & 0x1fffffull;
  return (uint32_t)x;
}

// Tree-frame coordinates of the particles (internal order): u4[i] = (u, hu);
// the key and the internal index go to caller position perm[i], the input
// order of the stable sort. zt[i] = z' in the tree frame.
static __global__ void tree_frame_kernel(const double* __restrict__ x, const double* __restrict__ y,
                                         const double* __restrict__ z, const double* __restrict__ h,
                                         const int* __restrict__ perm, int n, TreeFrame F, float4* __restrict__ u4,
                                         double* __restrict__ zt, uint64_t* __restrict__ key,
                                         int* __restrict__ val, int* __restrict__ err) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const double xr = __fma_rn(F.c, x[i], -__dmul_rn(F.s, y[i]));
    const double yr = __fma_rn(F.s, x[i], __dmul_rn(F.c, y[i]));
    double zr = __dadd_rn(z[i], F.zeta);
    if (zr >= F.L) zr = __dsub_rn(zr, F.L);
    const float ux = __double2float_rn(__fma_rn(xr, F.invS, 0.5));
    const float uy = __double2float_rn(__fma_rn(yr, F.invS, 0.5));
    const float uz = __double2float_rn(__fma_rn(__dsub_rn(zr, F.halfL), F.invS, 0.5));
    const float hu = __double2float_rn(__dmul_rn(h[i], F.invS));
    const bool inside = ux >= 0.0f && ux < 1.0f && uy >= 0.0f && uy < 1.0f && uz >= 0.0f && uz < 1.0f;
    if (!inside) atomicOr(err, kErrTreeRange);
    const float cx = inside ? ux : 0.0f, cy = inside ? uy : 0.0f, cz = inside ? uz : 0.0f;
    const uint32_t qx = (uint32_t)__fmul_rn(cx, 2097152.0f), qy = (uint32_t)__fmul_rn(cy, 2097152.0f),
                   qz = (uint32_t)__fmul_rn(cz, 2097152.0f);
    u4[i] = make_float4(ux, uy, uz, hu);
    zt[i] = zr;
    const int c = perm[i];
    key[c] = (spread3(qx) << 2) | (spread3(qy) << 1) | spread3(qz);
    val[c] = i;
  }
}

// The same for the R^3 frame: u = R (x - cen) / S + 1/2, with the explicit
// fma/mul sequence; zt[i] = z[i] (no period).
static __global__ void tree_frame_r3_kernel(const double* __restrict__ x, const double* __restrict__ y,
                                            const double* __restrict__ z, const double* __restrict__ h,
                                            const int* __restrict__ perm, int n, TreeFrame3 F,
                                            float4* __restrict__ u4, double* __restrict__ zt,
                                            uint64_t* __restrict__ key, int* __restrict__ val, int* __restrict__ err) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const double dx = __dsub_rn(x[i], F.cen[0]), dy = __dsub_rn(y[i], F.cen[1]), dz = __dsub_rn(z[i], F.cen[2]);
    const double xr = __fma_rn(F.R[0], dx, __fma_rn(F.R[1], dy, __dmul_rn(F.R[2], dz)));
    const double yr = __fma_rn(F.R[3], dx, __fma_rn(F.R[4], dy, __dmul_rn(F.R[5], dz)));
    const double zr = __fma_rn(F.R[6], dx, __fma_rn(F.R[7], dy, __dmul_rn(F.R[8], dz)));
    const float ux = __double2float_rn(__fma_rn(xr, F.invS, 0.5));
    const float uy = __double2float_rn(__fma_rn(yr, F.invS, 0.5));
    const float uz = __double2float_rn(__fma_rn(zr, F.invS, 0.5));
    const float hu = __double2float_rn(__dmul_rn(h[i], F.invS));
    const bool inside = ux >= 0.0f && ux < 1.0f && uy >= 0.0f && uy < 1.0f && uz >= 0.0f && uz < 1.0f;
    if (!inside) atomicOr(err, kErrTreeRange);
    const float cx = inside ? ux : 0.0f, cy = inside ? uy : 0.0f, cz = inside ? uz : 0.0f;
    const uint32_t qx = (uint32_t)__fmul_rn(cx, 2097152.0f), qy = (uint32_t)__fmul_rn(cy, 2097152.0f),
                   qz = (uint32_t)__fmul_rn(cz, 2097152.0f);
    u4[i] = make_float4(ux, uy, uz, hu);
    zt[i] = z[i];
    const int c = perm[i];
    key[c] = (spread3(qx) << 2) | (spread3(qy) << 1) | spread3(qz);
    val[c] = i;
  }
}

// ---- stable LSD radix sort of (key, value), 8-bit digits -------------------
// hist[d][tile]: count of digit d in each tile of kSortTile keys.
static __global__ void __launch_bounds__(kSortThreads)
radix_hist_kernel(const uint64_t* __restrict__ key, int n, int shift, int ntiles, unsigned* __restrict__ hist) {
  __shared__ unsigned hcount[256];
  hcount[threadIdx.x] = 0;
  __syncthreads();
  const int base = blockIdx.x * kSortTile;
  for (int r = 0; r < kSortRounds; ++r) {
    const int q = base + r * kSortThreads + threadIdx.x;
    if (q < n) atomicAdd(&hcount[(unsigned)(key[q] >> shift) & 255u], 1u);
  }
  __syncthreads();
  hist[(size_t)threadIdx.x * ntiles + blockIdx.x] = hcount[threadIdx.x];
}

// Exclusive scan of m counts by one CTA of 1024 threads (each takes a
// contiguous chunk). total (may be null) gets the sum.
static __global__ void __launch_bounds__(1024)
scan_exclusive_kernel(const unsigned* __restrict__ in, unsigned* __restrict__ out, int m, unsigned* total) {
  __shared__ unsigned part[1024];
  const int chunk = (m + 1023) / 1024;
  const int b = threadIdx.x * chunk, e = min(m, b + chunk);
  unsigned s = 0;
  for (int k = b; k < e; ++k) s += in[k];
  part[threadIdx.x] = s;
  __syncthreads();
  for (int off = 1; off < 1024; off <<= 1) {  // Hillis-Steele inclusive scan of the chunk sums
    const unsigned v = threadIdx.x >= off ? part[threadIdx.x - off] : 0u;
    __syncthreads();
    part[threadIdx.x] += v;
    __syncthreads();
  }
  unsigned run = part[threadIdx.x] - s;
  for (int k = b; k < e; ++k) {
    const unsigned v = in[k];
    out[k] = run;
    run += v;
  }
  if (total && threadIdx.x == 1023) *total = part[1023];
}

// Stable scatter: the keys of a tile are taken in order, kSortThreads per
// round; within a round a key's rank among equal digits comes from its warp
// (match) and the warps before it, across rounds from a running count.
static __global__ void __launch_bounds__(kSortThreads)
radix_scatter_kernel(const uint64_t* __restrict__ kin, const int* __restrict__ vin, int n, int shift, int ntiles,
                     const unsigned* __restrict__ offs, uint64_t* __restrict__ kout, int* __restrict__ vout) {
  constexpr int kWarps = kSortThreads / 32;
  __shared__ unsigned run[256];
  __shared__ unsigned wcnt[kWarps][256];
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  run[threadIdx.x] = offs[(size_t)threadIdx.x * ntiles + blockIdx.x];
  const unsigned lt = (1u << lane) - 1u;
  for (int r = 0; r < kSortRounds; ++r) {
    for (int k = 0; k < kWarps; ++k) wcnt[k][threadIdx.x] = 0;
    __syncthreads();
    const int q = blockIdx.x * kSortTile + r * kSortThreads + threadIdx.x;
    const bool valid = q < n;
    const uint64_t kv = valid ? kin[q] : 0ull;
    const int vv = valid ? vin[q] : 0;
    const unsigned dig = valid ? ((unsigned)(kv >> shift) & 255u) : 256u;
    const unsigned peers = __match_any_sync(0xffffffffu, dig);
    const unsigned rank = __popc(peers & lt);
    if (valid && rank == 0) wcnt[w][dig] = __popc(peers);
    __syncthreads();
    {
      unsigned acc = run[threadIdx.x];
      for (int k = 0; k < kWarps; ++k) {
        const unsigned cnt = wcnt[k][threadIdx.x];
        wcnt[k][threadIdx.x] = acc;
        acc += cnt;
      }
      run[threadIdx.x] = acc;
    }
    __syncthreads();
    if (valid) {
      const unsigned pos = wcnt[w][dig] + rank;
      kout[pos] = kv;
      vout[pos] = vv;
    }
    __syncthreads();
  }
}

// ---- level-by-level build ---------------------------------------------------
// Node records: link = (first child or -1, children, first, end sorted
// positions), geo = (centre, side) in root units, pre = key prefix.
// Thread per (active node, child digit): the child's sorted range.
static __global__ void tree_children_kernel(const int* __restrict__ active, int n_active, int level,
                                            const uint64_t* __restrict__ key, const int4* __restrict__ link,
                                            const uint64_t* __restrict__ pre, int* __restrict__ cnt,
                                            int* __restrict__ beg) {
  const int slot = blockIdx.x * blockDim.x + threadIdx.x;
  if (slot >= 8 * n_active) return;
  const int node = active[slot >> 3], c = slot & 7;
  const int4 lk = link[node];
  const int sh = 3 * (kTreeDepth - 1 - level);
  const uint64_t target = (pre[node] << 3) | (uint64_t)c;
  int lo = lk.z, hi = lk.w;  // first q with key[q] >> sh >= target
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if ((key[mid] >> sh) < target) lo = mid + 1;
    else hi = mid;
  }
  int lo2 = lo, hi2 = lk.w;  // first q with key[q] >> sh > target
  while (lo2 < hi2) {
    const int mid = (lo2 + hi2) >> 1;
    if ((key[mid] >> sh) <= target) lo2 = mid + 1;
    else hi2 = mid;
  }
  cnt[slot] = lo2 - lo;
  beg[slot] = lo;
}

// One CTA: numbers the non-empty child slots (new nodes from id `base`, in
// slot order, so each parent's children are consecutive) and the next active
// nodes; writes the children, links the parents, and stores the two totals.
static __global__ void __launch_bounds__(1024)
tree_link_kernel(const int* __restrict__ active, int n_active, int level, int leaf, int base,
                 const int* __restrict__ cnt, const int* __restrict__ beg, int* __restrict__ pos,
                 int4* __restrict__ link, float4* __restrict__ geo, uint64_t* __restrict__ pre,
                 int* __restrict__ next_active, int* __restrict__ totals) {
  __shared__ int s1[1024], s2[1024];
  const int m = 8 * n_active;
  const int chunk = (m + 1023) / 1024;
  const int b = threadIdx.x * chunk, e = min(m, b + chunk);
  const bool deeper = level + 1 < kTreeDepth;
  int c1 = 0, c2 = 0;
  for (int k = b; k < e; ++k) {
    c1 += cnt[k] > 0;
    c2 += deeper && cnt[k] > leaf;
  }
  s1[threadIdx.x] = c1;
  s2[threadIdx.x] = c2;
  __syncthreads();
  for (int off = 1; off < 1024; off <<= 1) {
    const int v1 = threadIdx.x >= off ? s1[threadIdx.x - off] : 0;
    const int v2 = threadIdx.x >= off ? s2[threadIdx.x - off] : 0;
    __syncthreads();
    s1[threadIdx.x] += v1;
    s2[threadIdx.x] += v2;
    __syncthreads();
  }
  int p1 = s1[threadIdx.x] - c1, p2 = s2[threadIdx.x] - c2;
  const float side = ldexpf(1.0f, -(level + 1));
  for (int k = b; k < e; ++k) {
    pos[k] = p1;
    const int ck = cnt[k];
    if (ck > 0) {
      const int id = base + p1;
      const uint64_t pf = (pre[active[k >> 3]] << 3) | (uint64_t)(k & 7);
      pre[id] = pf;
      link[id] = make_int4(-1, 0, beg[k], beg[k] + ck);
      const uint32_t ix = compact3(pf >> 2), iy = compact3(pf >> 1), iz = compact3(pf);
      geo[id] = make_float4(__fmul_rn((float)ix + 0.5f, side), __fmul_rn((float)iy + 0.5f, side),
                            __fmul_rn((float)iz + 0.5f, side), side);
      ++p1;
      if (deeper && ck > leaf) next_active[p2++] = id;
    }
  }
  __syncthreads();
  for (int a = threadIdx.x; a < n_active; a += 1024) {
    const int first = pos[8 * a];
    const int last = 8 * a + 7;
    const int nch = pos[last] + (cnt[last] > 0) - first;
    int4 lk = link[active[a]];
    lk.x = base + first;
    lk.y = nch;
    link[active[a]] = lk;
  }
  if (threadIdx.x == 1023) {
    totals[0] = s1[1023];
    totals[1] = s2[1023];
  }
}

// Moments of the nodes [n0, n1) of one level, children first: a leaf sums its
// particles (sorted order), an inner node its children (FP64). mom = (M,
// sum m x, sum m y, sum m z'); hmax: largest h; hmf: largest hu.
static __global__ void tree_moments_kernel(int n0, int n1, const int4* __restrict__ link,
                                           const int* __restrict__ sidx, const double* __restrict__ x,
                                           const double* __restrict__ y, const double* __restrict__ zt,
                                           const double* __restrict__ m, const double* __restrict__ h,
                                           const float4* __restrict__ u4, double4_32a* __restrict__ mom,
                                           double* __restrict__ hmax, float* __restrict__ hmf) {
  const int id = n0 + blockIdx.x * blockDim.x + threadIdx.x;
  if (id >= n1) return;
  const int4 lk = link[id];
  double M = 0.0, sx = 0.0, sy = 0.0, sz = 0.0, hm = 0.0;
  float hu = 0.0f;
  if (lk.y == 0) {
    for (int q = lk.z; q < lk.w; ++q) {
      const int i = sidx[q];
      const double mi = m[i];
      M += mi;
      sx = fma(mi, x[i], sx);
      sy = fma(mi, y[i], sy);
      sz = fma(mi, zt[i], sz);
      hm = fmax(hm, h[i]);
      hu = fmaxf(hu, u4[i].w);
    }
  } else {
    for (int k = lk.x; k < lk.x + lk.y; ++k) {
      const double4_32a c = mom[k];
      M += c.x;
      sx += c.y;
      sy += c.z;
      sz += c.w;
      hm = fmax(hm, hmax[k]);
      hu = fmaxf(hu, hmf[k]);
    }
  }
  mom[id] = make_double4_32a(M, sx, sy, sz);
  hmax[id] = hm;
  hmf[id] = hu;
}

// Pseudo-particles of all nodes in the pair kernels' layout (periodic: z of
// the centre of mass shifted back by zeta into [0, L)).
static __global__ void tree_pack_kernel(int nn, const double4_32a* __restrict__ mom, const double* __restrict__ hmax,
                                        double zeta, double L, double invL, int periodic, float4* __restrict__ nA,
                                        float4* __restrict__ nB) {
  for (int id = blockIdx.x * blockDim.x + threadIdx.x; id < nn; id += gridDim.x * blockDim.x) {
    const double4_32a c = mom[id];
    double zc = c.w / c.x - zeta;
    if (periodic && zc < 0.0) zc += L;
    pack_one(c.y / c.x, c.z / c.x, zc, c.x, hmax[id], id, invL, nA, nB);
  }
}

// Particles in key order in the pair kernels' layout (coalesced leaf reads),
// with their tree-frame coordinates.
static __global__ void tree_gather_kernel(const float4* __restrict__ jA, const float4* __restrict__ jB,
                                          const float4* __restrict__ u4, const int* __restrict__ sidx, int n,
                                          float4* __restrict__ sA, float4* __restrict__ sB,
                                          float4* __restrict__ u4s) {
  for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < n; q += gridDim.x * blockDim.x) {
    const int i = sidx[q];
    sA[q] = jA[i];
    sB[q] = jB[i];
    u4s[q] = u4[i];
  }
}

// ---- walk ---------------------------------------------------------------------
// The opening test of one lane (FP32, exactly rounded, in the order written).
__device__ __forceinline__ bool tree_opens(const float4& u, const float4& g, float hm, const TreeCrit& C) {
  const float dx = __fsub_rn(u.x, g.x);
  const float dy = __fsub_rn(u.y, g.y);
  float dz = __fsub_rn(u.z, g.z);
  if (dz > C.hLu) dz = __fsub_rn(dz, C.Lu);
  else if (dz < -C.hLu) dz = __fadd_rn(dz, C.Lu);
  const float d2 = __fadd_rn(__fadd_rn(__fmul_rn(dx, dx), __fmul_rn(dy, dy)), __fmul_rn(dz, dz));
  if (__fmul_rn(g.w, g.w) >= __fmul_rn(C.th2, d2)) return true;
  const float clear = __fsub_rn(__fsqrt_rn(d2), __fmul_rn(0.8660254f, g.w));
  return clear <= __fadd_rn(u.w, hm);
}

// All lanes against the nl entries of the warp's list: the pair form of the
// correction-table tail over the infinite window (entry `self` of a lane,
// its own particle, has zero mass).
template <bool KAHAN>
__device__ __forceinline__ void tree_eval(const IParticle& I, int me, const float4* __restrict__ A_,
                                          const float4* __restrict__ B_, const int* __restrict__ id_, int nl,
                                          const SurrConst& S, const TableTail& T, float& sx, float& sy, float& sz,
                                          float& cx, float& cy, float& cz) {
#pragma unroll 1
  for (int k0 = 0; k0 < nl; k0 += STEPS_KAHAN_GROUP) {
    float gx = 0.f, gy = 0.f, gz = 0.f;
#pragma unroll 2
    for (int k = k0; k < k0 + STEPS_KAHAN_GROUP; ++k) {
      const int kc = min(k, nl - 1);
      const float4 A = A_[kc];
      const float4 B = B_[kc];
      float dx, dy, dz, dR2, hh;
      int kw;
      pair_geometry(I, A, B, dx, dy, dz, dR2, hh, kw);
      SurrPair P;
      surr_stage_a<true, -1>(dR2, dz, hh, 0, kw, S, P);
      const float2 r = table_read(T, P.u[0], P.u[1]);
      float sr, szz;
      surr_stage_c<true>(I, A, B, 0, kw, S, P, r.x, r.y, sr, szz);
      const float mj = (k < nl && id_[kc] != me) ? A.w : 0.0f;
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

// The R^3 form of the list evaluation (eq. NewtonianForce, one image): two
// entries per packed FP32x2 op, the spline only when some lane is softened.
template <bool KAHAN>
__device__ __forceinline__ void tree_eval_r3(const IParticle& I, int me, const float4* __restrict__ A_,
                                             const float4* __restrict__ B_, const int* __restrict__ id_, int nl,
                                             float& sx, float& sy, float& sz, float& cx, float& cy, float& cz) {
  float xh, yh, xl, yl;
  upk(I.xyh, xh, yh);
  upk(I.xyl, xl, yl);
  const u64 XH = pk(xh, xh), YH = pk(yh, yh), ZH = pk(I.zh, I.zh);
  const u64 XL = pk(xl, xl), YL = pk(yl, yl), ZL = pk(I.zl, I.zl);
  const u64 HI = pk(I.h, I.h);
#pragma unroll 1
  for (int k0 = 0; k0 < nl; k0 += 8) {
    u64 GX = pk(0.f, 0.f), GY = pk(0.f, 0.f), GZ = pk(0.f, 0.f);
#pragma unroll 1
    for (int k = k0; k < k0 + 8; k += 2) {
      const int ka = min(k, nl - 1), kb = min(k + 1, nl - 1);
      const float4 A0 = A_[ka], A1 = A_[kb], B0 = B_[ka], B1 = B_[kb];
      const float m0 = (k < nl && id_[ka] != me) ? A0.w : 0.0f;
      const float m1 = (k + 1 < nl && id_[kb] != me) ? A1.w : 0.0f;
      const u64 DX = add2(sub2(XH, pk(A0.x, A1.x)), sub2(XL, pk(B0.x, B1.x)));
      const u64 DY = add2(sub2(YH, pk(A0.y, A1.y)), sub2(YL, pk(B0.y, B1.y)));
      const u64 DZ = add2(sub2(ZH, pk(A0.z, A1.z)), sub2(ZL, pk(B0.z, B1.z)));
      const u64 R2 = fma2(DX, DX, fma2(DY, DY, mul2(DZ, DZ)));
      const u64 HH = add2(HI, pk(B0.w, B1.w));
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
      const u64 MF = mul2(pk(m0, m1), F);
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

#ifndef STEPS_TREE_MIN_BLOCKS
#define STEPS_TREE_MIN_BLOCKS 4  // co-resident CTAs per SM asked of the register allocator
#endif

// One warp per group of 32 particles in key order (sA/sB, u4s: key order);
// out = [3][n] pair sums in internal order (sidx maps key order to internal).
// R3: the R^3 pair force (no images, no table).
template <bool KAHAN, bool R3 = false>
__global__ void __launch_bounds__(kWalkWarps * 32, STEPS_TREE_MIN_BLOCKS)
tree_walk_kernel(const float4* __restrict__ sA, const float4* __restrict__ sB, const float4* __restrict__ u4s,
                 const int* __restrict__ sidx, int n, const int4* __restrict__ link, const float4* __restrict__ geo,
                 const float* __restrict__ hmf, const float4* __restrict__ nA, const float4* __restrict__ nB,
                 TreeCrit C, TableTail T, SurrConst S, double* __restrict__ out,
                 unsigned long long* __restrict__ inter, int* __restrict__ err) {
  __shared__ int stk[kWalkWarps][kWalkStack];
  __shared__ float4 lA[kWalkWarps][kWalkList];
  __shared__ float4 lB[kWalkWarps][kWalkList];
  __shared__ int lid[kWalkWarps][kWalkList];
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int g = blockIdx.x * kWalkWarps + w;
  if (g * 32 >= n) return;  // the whole warp leaves; the walk uses warp-level synchronisation only
  const int q = g * 32 + lane;
  const bool valid = q < n;
  const int qc = min(q, n - 1);
  const IParticle I = load_i(sA, sB, qc);
  const float4 u = u4s[qc];
  const int me = valid ? q : -1;
  const int nvalid = min(32, n - g * 32);
  int* st = stk[w];
  float4* A_ = lA[w];
  float4* B_ = lB[w];
  int* id_ = lid[w];
  float sx = 0.f, sy = 0.f, sz = 0.f, cx = 0.f, cy = 0.f, cz = 0.f;
  unsigned long long count = 0;
  bool overflow = false;
  if (lane == 0) st[0] = 0;
  __syncwarp();
  int top = 1, nl = 0;
  while (top > 0) {
    const int node = st[--top];
    const float4 gm = geo[node];
    const int4 lk = link[node];
    const float hm = hmf[node];
    const bool open = __any_sync(0xffffffffu, valid && tree_opens(u, gm, hm, C));
    __syncwarp();  // every lane has read st[top] before it is reused
    if (open && lk.y > 0) {
      if (top + lk.y > kWalkStack) {
        overflow = true;
        break;
      }
      if (lane < lk.y) st[top + lane] = lk.x + lane;
      __syncwarp();
      top += lk.y;
      continue;
    }
    if (!open) {
      if (lane == 0) {
        A_[nl] = nA[node];
        B_[nl] = nB[node];
        id_[nl] = -1;
      }
      ++nl;
    } else {
      for (int b0 = lk.z; b0 < lk.w; b0 += 32) {
        const int c = min(32, lk.w - b0);
        if (nl + c > kWalkList) {
          __syncwarp();
          if (R3)
            tree_eval_r3<KAHAN>(I, me, A_, B_, id_, nl, sx, sy, sz, cx, cy, cz);
          else
            tree_eval<KAHAN>(I, me, A_, B_, id_, nl, S, T, sx, sy, sz, cx, cy, cz);
          count += (unsigned long long)nl * nvalid;
          nl = 0;
          __syncwarp();
        }
        if (lane < c) {
          A_[nl + lane] = sA[b0 + lane];
          B_[nl + lane] = sB[b0 + lane];
          id_[nl + lane] = b0 + lane;
        }
        nl += c;
      }
    }
    if (nl > kWalkList - 33) {
      __syncwarp();
      if (R3)
        tree_eval_r3<KAHAN>(I, me, A_, B_, id_, nl, sx, sy, sz, cx, cy, cz);
      else
        tree_eval<KAHAN>(I, me, A_, B_, id_, nl, S, T, sx, sy, sz, cx, cy, cz);
      count += (unsigned long long)nl * nvalid;
      nl = 0;
      __syncwarp();
    }
  }
  __syncwarp();
  if (nl > 0) {
    if (R3)
      tree_eval_r3<KAHAN>(I, me, A_, B_, id_, nl, sx, sy, sz, cx, cy, cz);
    else
      tree_eval<KAHAN>(I, me, A_, B_, id_, nl, S, T, sx, sy, sz, cx, cy, cz);
    count += (unsigned long long)nl * nvalid;
  }
  if (lane == 0) {
    atomicAdd(inter, count);
    if (overflow) atomicOr(err, kErrTreeStack);
  }
  if (valid) {
    const int i = sidx[q];
    out[i] = (double)sx - (KAHAN ? (double)cx : 0.0);
    out[(long long)n + i] = (double)sy - (KAHAN ? (double)cy : 0.0);
    out[2 * (long long)n + i] = (double)sz - (KAHAN ? (double)cz : 0.0);
  }
}

}  // namespace steps
