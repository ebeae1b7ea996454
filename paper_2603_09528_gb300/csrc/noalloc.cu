// tpt_thomas_noalloc: the modal Thomas sweep with its elimination scratch in a
// fixed, file-scope device array instead of caller- or library-allocated
// memory.  It exists for callers that cannot allocate device memory when they
// call the solver: code running inside a host callback or a framework hook
// where CUDA allocation calls are not allowed, callers whose device memory is
// owned entirely by another allocator's pool, and latency-sensitive callers
// that cannot afford cudaFree's implicit device-wide synchronisation.  The
// paper has no counterpart; it is a packaging variant of the Thomas step.
#include <cuda_runtime.h>

#include <mutex>

#include "tpt_internal.h"

namespace {

// Largest field (Nx*Ny*Nz points) the fixed scratch serves: 4,194,304 points,
// 32 MiB of float64.  Every GPU that loads the library holds this array until
// the process exits.
constexpr unsigned long long kNoAllocMaxPoints = 1ull << 22;

// c' of the forward elimination, one value per point.  Host code must not pass
// this name to a kernel: in host code it is a host-side stand-in, not a device
// address.  The device address is taken once per device with
// cudaGetSymbolAddress (noalloc_scratch below).
static __device__ __align__(256) double g_thomas_scratch[kNoAllocMaxPoints];

constexpr int kMaxDevices = 64;
std::mutex g_mutex;
double* g_scratch_addr[kMaxDevices] = {nullptr};

// Device address of g_thomas_scratch on `dev`, looked up once per device with
// that device current and kept for the life of the process (a device reset
// invalidates it together with every plan, which this entry point needs).
// Returns nullptr on failure.
double* noalloc_scratch(int dev) {
  if (dev < 0 || dev >= kMaxDevices) return nullptr;
  std::lock_guard<std::mutex> lock(g_mutex);
  if (g_scratch_addr[dev]) return g_scratch_addr[dev];
  int prev = -1;
  if (cudaGetDevice(&prev) != cudaSuccess) {
    cudaGetLastError();
    prev = -1;
  }
  if (cudaSetDevice(dev) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  void* ptr = nullptr;
  const cudaError_t e = cudaGetSymbolAddress(&ptr, g_thomas_scratch);
  if (e != cudaSuccess) {
    cudaGetLastError();
    ptr = nullptr;
  }
  if (prev >= 0) cudaSetDevice(prev);
  g_scratch_addr[dev] = static_cast<double*>(ptr);
  return g_scratch_addr[dev];
}

}  // namespace

extern "C" int tpt_thomas_noalloc(tpt_plan p, const double* fhat, double* phihat, void* stream) {
  if (!p || p->dev < 0 || !p->d_scal || !fhat || !phihat) return TPT_ERR_INVALID_ARG;
  if (static_cast<unsigned long long>(tpt::npts(p)) > kNoAllocMaxPoints) return TPT_ERR_UNSUPPORTED;
  double* scratch = noalloc_scratch(p->dev);
  if (!scratch) return TPT_ERR_CUDA;
  int prev = -1;
  if (cudaGetDevice(&prev) != cudaSuccess) {
    cudaGetLastError();
    prev = -1;
  }
  if (cudaSetDevice(p->dev) != cudaSuccess) {
    cudaGetLastError();
    return TPT_ERR_CUDA;
  }
  // Every line writes its c' values before it reads them, so the scratch
  // needs no clearing between calls.
  const cudaError_t e =
      tpt::thomas_fp64(p, fhat, phihat, scratch, nullptr, static_cast<cudaStream_t>(stream));
  if (prev >= 0) cudaSetDevice(prev);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return TPT_ERR_CUDA;
  }
  return TPT_OK;
}
