// Unit-rate measurement for the roofline of the pair kernels (not part of the
// library): MUFU rsqrt/ex2/rcp, FFMA, packed FFMA2, FMNMX, the pair kernel's
// image pattern (scalar and packed) and mma.sync m16n8k16 f16->f32, each run as
// one full wave of independent dependency chains. Rates are computed from CUDA
// event time (clock64 does not tick at the SM clock on this part), and reported
// per SM per clock at the SM clock passed on the command line (MHz; default the
// device's maximum).
// Build and run: nvcc -gencode arch=compute_103a,code=sm_103a -O3 unit_rates.cu -o unit_rates && ./unit_rates [MHz]
// Every kernel writes one float per thread into out[gridDim.x*blockDim.x] and
// one cycle count per block into cyc[gridDim.x]; no other memory access.
#include <cstdio>
#include <cstdint>
#include <cstdlib>
#include <cuda_runtime.h>

#define CH 8
#define CK(x) do { cudaError_t e = (x); if (e != cudaSuccess) { printf("CUDA %s at %d\n", cudaGetErrorString(e), __LINE__); return 1; } } while (0)

__device__ __forceinline__ float rsq(float x) { float y; asm volatile("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x)); return y; }
__device__ __forceinline__ float ex2(float x) { float y; asm volatile("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x)); return y; }
__device__ __forceinline__ float rcp(float x) { float y; asm volatile("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x)); return y; }
__device__ __forceinline__ unsigned long long f2(float a, float b) { unsigned long long r; asm("mov.b64 %0, {%1,%2};" : "=l"(r) : "f"(a), "f"(b)); return r; }
__device__ __forceinline__ float2 u2(unsigned long long r) { float a, b; asm("mov.b64 {%0,%1}, %2;" : "=f"(a), "=f"(b) : "l"(r)); return make_float2(a, b); }

template <int MODE>
__global__ void kern(float* out, long long* cyc, int iters, float a, float b) {
  float v[CH];
  unsigned long long p[CH];
#pragma unroll
  for (int c = 0; c < CH; ++c) { v[c] = 1.0f + 0.001f * (threadIdx.x + c); p[c] = f2(v[c], v[c] + 0.5f); }
  __syncthreads();
  long long t0 = clock64();
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int c = 0; c < CH; ++c) {
      if (MODE == 0) {            // MUFU rsqrt only
        v[c] = rsq(v[c] + 0.0f);
      } else if (MODE == 1) {     // FFMA only (4 per chain step)
        v[c] = fmaf(v[c], a, b); v[c] = fmaf(v[c], a, b); v[c] = fmaf(v[c], a, b); v[c] = fmaf(v[c], a, b);
      } else if (MODE == 2) {     // packed FFMA2 only (4 per chain step)
        unsigned long long A = f2(a, a), B = f2(b, b);
        asm volatile("fma.rn.f32x2 %0, %0, %1, %2;" : "+l"(p[c]) : "l"(A), "l"(B));
        asm volatile("fma.rn.f32x2 %0, %0, %1, %2;" : "+l"(p[c]) : "l"(A), "l"(B));
        asm volatile("fma.rn.f32x2 %0, %0, %1, %2;" : "+l"(p[c]) : "l"(A), "l"(B));
        asm volatile("fma.rn.f32x2 %0, %0, %1, %2;" : "+l"(p[c]) : "l"(A), "l"(B));
      } else if (MODE == 3) {     // image pattern: 6 FP32 + 1 MUFU
        float o = v[c] + a;
        float r2 = fmaf(o, o, b);
        float ri = rsq(r2);
        float r3 = ri * ri * ri;
        v[c] = v[c] + r3;
        v[c] = fmaf(o, r3, v[c]) * 0.5f;
      } else if (MODE == 4) {     // ex2 only
        v[c] = ex2(v[c] * -0.5f);
      } else if (MODE == 5) {     // FMNMX-heavy: 4 fmaxf per step
        v[c] = fmaxf(v[c], a); v[c] = fminf(v[c], b); v[c] = fmaxf(v[c], a * 0.5f); v[c] = fminf(v[c], b + 1.f);
      } else if (MODE == 6) {     // rcp only
        v[c] = rcp(v[c] + 0.0f);
      } else if (MODE == 7) {     // packed image pattern: 2 images per chain step, 6 packed + 2 MUFU
        unsigned long long A = f2(a, a + 1.0f), B = f2(b, b), o, r2, r3, t;
        asm volatile("add.rn.f32x2 %0, %1, %2;" : "=l"(o) : "l"(p[c]), "l"(A));
        asm volatile("fma.rn.f32x2 %0, %1, %1, %2;" : "=l"(r2) : "l"(o), "l"(B));
        float2 q = u2(r2);
        float2 ri = make_float2(rsq(q.x), rsq(q.y));
        unsigned long long R = f2(ri.x, ri.y);
        asm volatile("mul.rn.f32x2 %0, %1, %1;" : "=l"(t) : "l"(R));
        asm volatile("mul.rn.f32x2 %0, %1, %2;" : "=l"(r3) : "l"(t), "l"(R));
        asm volatile("add.rn.f32x2 %0, %0, %1;" : "+l"(p[c]) : "l"(r3));
        asm volatile("fma.rn.f32x2 %0, %1, %2, %0;" : "+l"(p[c]) : "l"(o), "l"(r3));
      }
    }
  }
  long long t1 = clock64();
  float s = 0.f;
#pragma unroll
  for (int c = 0; c < CH; ++c) { float2 q = u2(p[c]); s += v[c] + q.x + q.y; }
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
  if (threadIdx.x == 0) cyc[blockIdx.x] = t1 - t0;
}

// mma.sync m16n8k16 f16 inputs, f32 accumulate: 4 independent accumulators per warp
__global__ void kmma(float* out, long long* cyc, int iters) {
  unsigned a0 = 0x3c003c00u ^ threadIdx.x, a1 = a0, a2 = a0, a3 = a0, b0 = 0x3c003c00u, b1 = b0;
  float d[4][4];
#pragma unroll
  for (int c = 0; c < 4; ++c) for (int e = 0; e < 4; ++e) d[c][e] = 0.f;
  __syncthreads();
  long long t0 = clock64();
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int c = 0; c < 4; ++c)
      asm volatile("mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};"
                   : "+f"(d[c][0]), "+f"(d[c][1]), "+f"(d[c][2]), "+f"(d[c][3])
                   : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
  }
  long long t1 = clock64();
  float s = 0.f;
  for (int c = 0; c < 4; ++c) for (int e = 0; e < 4; ++e) s += d[c][e];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
  if (threadIdx.x == 0) cyc[blockIdx.x] = t1 - t0;
}

int main(int argc, char** argv) {
  cudaDeviceProp pr; CK(cudaGetDeviceProperties(&pr, 0));
  int sms = pr.multiProcessorCount;
  int khz = 0;
  cudaDeviceGetAttribute(&khz, cudaDevAttrClockRate, 0);
  const double mhz = argc > 1 ? atof(argv[1]) : khz / 1000.0;
  printf("device %s SMs %d cc %d.%d, rates per SM per clock at %.0f MHz\n", pr.name, sms, pr.major, pr.minor, mhz);
  const int bs = 256, maxblocks = 4096;
  float* out; long long* cyc;
  CK(cudaMalloc(&out, sizeof(float) * bs * maxblocks));
  CK(cudaMalloc(&cyc, sizeof(long long) * maxblocks));
  long long hc[4096];
  struct T { const char* name; void* f; double ops; } tests[] = {
    {"mufu_rsqrt", (void*)kern<0>, 1.0 * CH},
    {"ffma", (void*)kern<1>, 4.0 * CH},
    {"ffma2(lanes x2)", (void*)kern<2>, 8.0 * CH},
    {"image 6fp32+1mufu (per image)", (void*)kern<3>, 1.0 * CH},
    {"mufu_ex2", (void*)kern<4>, 1.0 * CH},
    {"fmnmx", (void*)kern<5>, 4.0 * CH},
    {"mufu_rcp", (void*)kern<6>, 1.0 * CH},
    {"image packed (per image)", (void*)kern<7>, 2.0 * CH},
  };
  for (int pass = 0; pass < 2; ++pass)
  for (auto& t : tests) {
    int nb = 0;
    CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, t.f, bs, 0));
    int grid = sms * nb; if (grid > maxblocks) grid = maxblocks;
    int iters = 4096;
    void* args[] = {&out, &cyc, &iters, nullptr, nullptr};
    float a = 0.999f, b = 0.0001f;
    args[3] = &a; args[4] = &b;
    cudaEvent_t e0, e1; cudaEventCreate(&e0); cudaEventCreate(&e1);
    CK(cudaEventRecord(e0));
    CK(cudaLaunchKernel(t.f, dim3(grid), dim3(bs), args, 0, 0));
    CK(cudaEventRecord(e1));
    CK(cudaDeviceSynchronize());
    float ms; cudaEventElapsedTime(&ms, e0, e1);
    CK(cudaMemcpy(hc, cyc, sizeof(long long) * grid, cudaMemcpyDeviceToHost));
    double mc = 0; for (int i = 0; i < grid; ++i) mc += hc[i]; mc /= grid;
    double ops_block = t.ops * iters * bs;
    double per_sm_clk = ops_block * nb / mc;
    double total = t.ops * iters * (double)bs * grid;
    if (pass == 1)
      printf("%-34s %.3e ops/s  %7.2f lane-ops/SM/clk  %.3f ms\n", t.name, total / (ms * 1e-3),
             total / (ms * 1e-3) / (sms * mhz * 1e6), ms);
  }
  for (int pass = 0; pass < 2; ++pass) {
    int nb = 0;
    CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kmma, bs, 0));
    int grid = sms * nb; if (grid > maxblocks) grid = maxblocks;
    int iters = 8192;
    cudaEvent_t e0, e1; cudaEventCreate(&e0); cudaEventCreate(&e1);
    CK(cudaEventRecord(e0));
    kmma<<<grid, bs>>>(out, cyc, iters);
    CK(cudaGetLastError());
    CK(cudaEventRecord(e1));
    CK(cudaDeviceSynchronize());
    float ms; cudaEventElapsedTime(&ms, e0, e1);
    CK(cudaMemcpy(hc, cyc, sizeof(long long) * grid, cudaMemcpyDeviceToHost));
    double mc = 0; for (int i = 0; i < grid; ++i) mc += hc[i]; mc /= grid;
    double flops_block = 2.0 * 16 * 8 * 16 * 4 * (double)iters * (bs / 32);
    if (pass == 1)
      printf("%-34s %.3e flop/s  %7.1f flop/SM/clk  %.3f ms\n", "mma.sync m16n8k16 f16->f32",
             flops_block * grid / (ms * 1e-3), flops_block * grid / (ms * 1e-3) / (sms * mhz * 1e6), ms);
  }
  cudaFree(out); cudaFree(cyc);
  return 0;
}
