// Allocation-free pair accelerations (declared in include/steps_cyl.h as
// steps_cyl_pair_accel_noalloc).
//
// Some callers cannot allocate device memory: a host whose device memory is
// owned and budgeted by another allocator (a caching allocator or a fixed
// arena reserved at start-up), a loop that must not take cudaMalloc's implicit
// device-wide synchronisation, or a plug-in that is only allowed to allocate
// during its initialisation. For them this entry point evaluates the pair term
// with the same pack, stream-K pair and finalize kernels as a context does, but
// keeps every intermediate (the packed FP32 positions and the stream-K partial
// sums) in one file-scope __device__ array of fixed size. It never calls
// cudaMalloc, cudaFree or an allocating library routine. The call stays
// asynchronous, so it keeps no device error word: nothing would read it.
//
// The array exists once per device that loads this library and lives until the
// process exits. Host code cannot use its name as a device address: the address
// is obtained with cudaGetSymbolAddress once per device, with that device
// current, on the first call made on that device.
#include <cuda_runtime.h>

#include <algorithm>
#include <mutex>

#include "steps_cyl.h"
#include "nbody_kernels.cuh"

using namespace steps;

namespace {

constexpr int kNoallocMaxN = STEPS_NOALLOC_MAX_N;
constexpr int kNoallocMaxCtas = STEPS_NOALLOC_MAX_CTAS;
constexpr int kNoallocMaxBlocks = (kNoallocMaxN + kBI - 1) / kBI;
// byte layout of the scratch array: packed jA | packed jB | partials
constexpr size_t kPackBytes = sizeof(float4) * (size_t)kNoallocMaxN;
constexpr size_t kPartBytes = sizeof(double) * 3 * kBI * (size_t)(kNoallocMaxBlocks + kNoallocMaxCtas);
constexpr size_t kScratchBytes = 2 * kPackBytes + kPartBytes;
static_assert(kScratchBytes == STEPS_NOALLOC_SCRATCH_BYTES, "scratch size must match the header");

__device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

struct DeviceScratch {
  unsigned char* base = nullptr;  // device address of g_noalloc_scratch on this device
  int ctas = 0;                   // co-resident CTAs of the pair kernel (capped)
  bool ready = false;
};

constexpr int kMaxDevices = 64;
DeviceScratch g_dev[kMaxDevices];
std::mutex g_mutex;

// Failures are reported by the status code alone (the message text names the
// cause for a reader of this file).
inline int noalloc_fail(int code, const char* /*why*/) { return code; }

// A runtime call of this entry point failed: clear the error it left as the
// thread's last error, unless an error from the caller's earlier work was
// already pending when the call began (that one stays for the caller to see).
inline int noalloc_cuda_fail(cudaError_t pending, const char* why) {
  if (pending == cudaSuccess) cudaGetLastError();
  return noalloc_fail(STEPS_ECUDA, why);
}

// Set-up for the current device (called with that device current).
int setup_device(int dev, cudaError_t pending, DeviceScratch** out) {
  std::lock_guard<std::mutex> lock(g_mutex);
  DeviceScratch& d = g_dev[dev];
  if (!d.ready) {
    void* ptr = nullptr;
    if (cudaGetSymbolAddress(&ptr, g_noalloc_scratch) != cudaSuccess)
      return noalloc_cuda_fail(pending, "cudaGetSymbolAddress of the scratch array failed");
    int sms = 0, occ = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, pair_fp32_kernel<true>, kBI, 0) != cudaSuccess)
      return noalloc_cuda_fail(pending, "device query failed");
    d.base = static_cast<unsigned char*>(ptr);
    d.ctas = std::max(1, std::min(kNoallocMaxCtas, sms * std::max(occ, 1)));
    d.ready = true;
  }
  *out = &d;
  return STEPS_OK;
}

// True when p is device memory the kernels on device dev may dereference: an
// allocation of that device (cudaMalloc, a pool, VMM) or managed memory. Host
// memory, pinned or not, and another device's memory are refused.
// cudaPointerGetAttributes only reads the driver's records; it allocates nothing.
bool on_device(const void* p, int dev, cudaError_t pending) {
  cudaPointerAttributes at{};
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    if (pending == cudaSuccess) cudaGetLastError();
    return false;
  }
  if (at.type == cudaMemoryTypeManaged) return true;
  return at.type == cudaMemoryTypeDevice && at.device == dev;
}

}  // namespace

extern "C" int steps_cyl_pair_accel_noalloc(int64_t n, const double* x, const double* y, const double* z,
                                            const double* m, const double* h, double G, double L, int32_t n_cut,
                                            int32_t precision, double* ax, double* ay, double* az, void* stream) {
  if (n < 2 || n > kNoallocMaxN) return noalloc_fail(STEPS_EINVAL, "n must be in [2, STEPS_NOALLOC_MAX_N]");
  if (!x || !y || !z || !m || !h || !ax || !ay || !az) return noalloc_fail(STEPS_EINVAL, "NULL array");
  if (!(G > 0) || !(L > 0)) return noalloc_fail(STEPS_EINVAL, "G and L must be > 0");
  if (n_cut < 1 || n_cut > 4096) return noalloc_fail(STEPS_EINVAL, "n_cut must be in [1, 4096]");
  if (precision != STEPS_FP32_KAHAN && precision != STEPS_FP32_PLAIN)
    return noalloc_fail(STEPS_EINVAL, "precision must be STEPS_FP32_KAHAN or STEPS_FP32_PLAIN");
  const cudaError_t pending = cudaPeekAtLastError();
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return noalloc_cuda_fail(pending, "no usable current device");
  if (dev < 0 || dev >= kMaxDevices) return noalloc_fail(STEPS_ECUDA, "device ordinal beyond the table");
  const void* arrays[8] = {x, y, z, m, h, ax, ay, az};
  for (const void* p : arrays)
    if (!on_device(p, dev, pending))
      return noalloc_fail(STEPS_EINVAL, "every array must be device memory of the current device");
  DeviceScratch* d = nullptr;
  int rc = setup_device(dev, pending, &d);
  if (rc) return rc;

  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const int nn = (int)n;
  float4* jA = reinterpret_cast<float4*>(d->base);
  float4* jB = reinterpret_cast<float4*>(d->base + kPackBytes);
  double* part = reinterpret_cast<double*>(d->base + 2 * kPackBytes);
  const int NB = (nn + kBI - 1) / kBI, NT = (nn + kBJ - 1) / kBJ;
  const long long U = (long long)NB * NT;
  const int C = (int)std::min<long long>(U, d->ctas);
  const double invL = 1.0 / L;

  // every byte of the scratch array this call reads, it writes first: the
  // packed positions here, and each stream-K partial slot whole, before the
  // finalize kernel reads it
  pack_kernel<<<(nn + 255) / 256, 256, 0, st>>>(x, y, z, m, h, nn, invL, jA, jB);
  if (precision == STEPS_FP32_KAHAN)
    pair_fp32_kernel<true><<<C, kBI, 0, st>>>(jA, jB, nn, n_cut, U, NT, C, part);
  else
    pair_fp32_kernel<false><<<C, kBI, 0, st>>>(jA, jB, nn, n_cut, U, NT, C, part);
  BgParams off{};
  off.mode = STEPS_BG_OFF;
  finalize_kernel<<<(nn + 255) / 256, 256, 0, st>>>(part, nn, NT, U, C, -G * invL * invL, off, x, y, z, ax, ay, az,
                                                    0.0, nullptr, nullptr, nullptr, 1.0, nullptr, nullptr, nullptr,
                                                    nullptr);
  // a launch failure replaces the thread's last error; one equal to the error
  // pending before the call is taken as the caller's, which stays in place
  const cudaError_t after = cudaPeekAtLastError();
  if (after != cudaSuccess && after != pending) return noalloc_cuda_fail(pending, "a kernel launch failed");
  return STEPS_OK;
}
