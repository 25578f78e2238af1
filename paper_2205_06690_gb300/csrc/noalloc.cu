// Allocation-free variant of the exciton eigensolver (sbse_spectrum_noalloc, see include/sbse.h).
//
// Some callers cannot allocate device memory: a host framework that has reserved the whole GPU for
// its own memory pool, or code that must never trigger an allocation (and its implicit device
// synchronisation) once it is running. For them the eigensolver's scratch space (a copy of A that
// the Householder reduction overwrites, plus the tridiagonal diagonal and off-diagonal) lives in the
// file-scope device array below instead of a cudaMalloc'ed buffer. The array exists once per GPU that
// loads the library and is held until the process exits.
#include <cuda_runtime.h>

#include <string>

#include "kernels.h"
#include "sbse.h"

namespace sbse {
void set_thread_error(const std::string &msg);
}

namespace {

constexpr int kMaxN = SBSE_NOALLOC_MAX_N;
constexpr size_t kScratchDoubles = (size_t)kMaxN * kMaxN + 2 * (size_t)kMaxN;

// The shared scratch of every sbse_spectrum_noalloc call on a device. In host code this name is
// only a stand-in for the symbol: the device address comes from cudaGetSymbolAddress below.
static __device__ __align__(256) double g_eig_scratch[kScratchDoubles];

// With the calling thread's current device: the device address of the scratch array. It is looked
// up on every call (cheap once the module is loaded): an address cached per device index would go
// stale after cudaDeviceReset or differ for another context on the same device.
int scratch_for_current_device(double **out) {
  void *p = nullptr;
  const cudaError_t e = cudaGetSymbolAddress(&p, g_eig_scratch);
  if (e != cudaSuccess || !p) {
    sbse::set_thread_error(std::string("cudaGetSymbolAddress of the eigensolver scratch failed: ") +
                           cudaGetErrorString(e));
    return SBSE_ERR_CUDA;
  }
  *out = static_cast<double *>(p);
  return SBSE_OK;
}

}  // namespace

extern "C" int sbse_spectrum_noalloc(const double *a_dev, int n, int k, double *evals_dev,
                                     void *stream) {
  if (!a_dev || !evals_dev) {
    sbse::set_thread_error("a_dev and evals_dev must be device pointers");
    return SBSE_ERR_INVALID_ARG;
  }
  if (n < 1 || k < 1 || k > n) {
    sbse::set_thread_error("need 1 <= k <= n");
    return SBSE_ERR_INVALID_ARG;
  }
  if (n > kMaxN) {
    sbse::set_thread_error("n = " + std::to_string(n) + " exceeds the allocation-free limit " +
                           std::to_string(kMaxN) + "; use sbse_spectrum");
    return SBSE_ERR_SHAPE;
  }
  double *scratch = nullptr;
  int rc = scratch_for_current_device(&scratch);
  if (rc) return rc;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  // The scratch keeps the previous call's contents; nothing in it must start at zero: the copy of
  // A and the tridiagonal arrays are written in full before they are read.
  sbse::launch_eig_lowest(const_cast<double *>(a_dev), n, k, evals_dev, scratch, s);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) {
    sbse::set_thread_error(std::string("CUDA error in sbse_spectrum_noalloc: ") + cudaGetErrorString(e));
    return SBSE_ERR_CUDA;
  }
  return SBSE_OK;
}
