// forces_noalloc.cu -- Coulomb accelerations without any device allocation.
//
// iontrap_forces evaluates the force kernel on a handle, and a handle owns device
// buffers that iontrap_create obtained with cudaMalloc.  Some callers cannot allocate:
// a process that hands all of its device memory to its own pool up front and forbids
// allocations behind its back, a host application that loads this library as a plugin
// and owns every device buffer itself, or a latency-critical loop that must not pay
// for cudaMalloc's implicit synchronisation.  For them, iontrap_forces_noalloc takes
// the positions and the output in the caller's device memory and keeps every piece of
// scratch the force kernel needs -- the FP32 hi/lo pair stream, the per-split partial
// sums and the arrival counters -- in one fixed array of device memory that is part of
// the library image itself (g_scratch below).  Every GPU that loads the library holds
// that array until the process exits.
//
// Limits and sharing: at most kNoAllocMaxIons ions per call (larger calls return
// IONTRAP_ETOOLARGE without launching anything).  All calls on a device share the
// one array, which keeps whatever the previous call left in it; each call clears the
// counters it relies on before it launches.  Two calls whose work overlaps on the GPU
// (different streams, or different host threads) race on the array and give wrong
// results: serialise them.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <mutex>

#include "iontrap_internal.cuh"

namespace it {
const void* step_kernel(int f64, int T, int I, int packed, int fused);
const void* prep_kernel();
}  // namespace it

using namespace it;

namespace {

constexpr long long kNoAllocMaxIons = 8192;
constexpr int kNoAllocMaxSplits = 8;
constexpr int kNoAllocThreads = 64;  // force kernel: 64 threads, one ion per thread

// Byte layout of the scratch array.
constexpr size_t kOffStep = 0;     // long long, kept 0 (pair stream buffer 0 is used)
constexpr size_t kOffErr = 8;      // int error flags
constexpr size_t kOffDone = 12;    // unsigned, completed i-blocks
constexpr size_t kOffCnt = 256;    // unsigned[i-blocks], per-i-block arrival counters
constexpr size_t kCntBytes = ((kNoAllocMaxIons / kNoAllocThreads) * sizeof(unsigned) + 255) / 256 * 256;
constexpr size_t kOffPair = kOffCnt + kCntBytes;  // float4 hi[n], lo[n]
constexpr size_t kPairBytes = (size_t)kNoAllocMaxIons * 2 * sizeof(float4);
constexpr size_t kOffPart = kOffPair + kPairBytes;  // 32-byte records, split * n + i
constexpr size_t kPartBytes = (size_t)kNoAllocMaxSplits * kNoAllocMaxIons * 32;
constexpr size_t kScratchBytes = kOffPart + kPartBytes;  // 2.25 MiB + 768 B

static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

// Device address of g_scratch per device.  In host code the name g_scratch is only a
// host-side stand-in for the symbol, so the address is looked up with that device
// current by cudaGetSymbolAddress.  The lookup is repeated on every call made outside
// stream capture, because the address belongs to the device's current context: after a
// cudaDeviceReset (or any other teardown of the primary context) the module is loaded
// again and the array may sit elsewhere.  A call made while its stream is being captured
// uses the address the last uncaptured call on that device found.
std::mutex g_mu;
constexpr int kMaxDevices = 64;
unsigned char* g_addr[kMaxDevices] = {};

int scratch_for_device(int dev, cudaStream_t stream, unsigned char** out) {
  if (dev < 0 || dev >= kMaxDevices) return IONTRAP_ECUDA;
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(stream, &cs) != cudaSuccess) return IONTRAP_ECUDA;
  std::lock_guard<std::mutex> lock(g_mu);
  if (cs == cudaStreamCaptureStatusNone) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_scratch);
    if (e != cudaSuccess || !p) return IONTRAP_ECUDA;
    g_addr[dev] = static_cast<unsigned char*>(p);
  }
  if (!g_addr[dev]) return IONTRAP_ECUDA;
  *out = g_addr[dev];
  return IONTRAP_OK;
}

}  // namespace

extern "C" int iontrap_forces_noalloc(const iontrap_species* species, int n_species,
                                      const uint8_t* d_species_of_ion, const double* d_x, int64_t n,
                                      double* d_acc, void* cuda_stream) {
  if (!species || n_species < 1 || n_species > IONTRAP_MAX_SPECIES || !d_species_of_ion || !d_x || !d_acc ||
      n < 1)
    return IONTRAP_EINVAL;
  for (int s = 0; s < n_species; ++s)
    if (!(species[s].mass_amu > 0) || !std::isfinite(species[s].mass_amu) || !std::isfinite(species[s].charge_e))
      return IONTRAP_EINVAL;
  if (n > kNoAllocMaxIons) return IONTRAP_ETOOLARGE;

  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return IONTRAP_ECUDA;
  cudaStream_t stream = static_cast<cudaStream_t>(cuda_stream);
  unsigned char* base = nullptr;
  const int st = scratch_for_device(dev, stream, &base);
  if (st) return st;

  StepArgs A{};
  A.n = n;
  float4* hi = reinterpret_cast<float4*>(base + kOffPair);
  A.hi[0] = A.hi[1] = hi;
  A.lo[0] = A.lo[1] = hi + n;
  A.x = const_cast<double*>(d_x);
  A.sp = d_species_of_ion;
  A.part = base + kOffPart;
  A.cnt = reinterpret_cast<unsigned*>(base + kOffCnt);
  A.done = reinterpret_cast<unsigned*>(base + kOffDone);
  A.step = reinterpret_cast<long long*>(base + kOffStep);
  A.err = reinterpret_cast<int*>(base + kOffErr);
  A.out = d_acc;
  A.mode = MODE_FORCES;
  const long long iblocks = (n + kNoAllocThreads - 1) / kNoAllocThreads;
  const long long splits = std::min<long long>(kNoAllocMaxSplits, std::max<long long>(1, (n + 127) / 128));
  A.jsplit = (int)((n + splits - 1) / splits);
  A.nsplit = (int)((n + A.jsplit - 1) / A.jsplit);
  const double ke = 1.0 / (4.0 * kPi * kEps0);
  for (int s = 0; s < n_species; ++s) {
    const double M = species[s].mass_amu * kAmu, z = species[s].charge_e;
    A.spc[s].coul = ke * kE * kE * z / M;
    A.spc[s].w = (float)z;
  }

  // step = 0, error flags = 0, done = 0, counters = 0; the output starts as NaN (all bits
  // set), so an ion whose sum never completes -- its i-block gave up on a bounded wait --
  // reads NaN instead of a stale value
  cudaError_t e = cudaMemsetAsync(base, 0, kOffCnt + kCntBytes, stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(d_acc, 0xFF, 3 * (size_t)n * sizeof(double), stream);
  int b = 0, f64 = 0;
  void* prep_params[] = {&A, &b, &f64};
  const unsigned prep_blocks = (unsigned)std::min<long long>((n + 255) / 256, 4096);
  if (e == cudaSuccess) e = cudaLaunchKernel(prep_kernel(), dim3(prep_blocks), dim3(256), prep_params, 0, stream);
  void* params[] = {&A};
  if (e == cudaSuccess)
    e = cudaLaunchKernel(step_kernel(0, kNoAllocThreads, 1, 0, 1), dim3((unsigned)iblocks, (unsigned)A.nsplit),
                         dim3(kNoAllocThreads), params, 0, stream);
  return e == cudaSuccess ? IONTRAP_OK : IONTRAP_ECUDA;
}
