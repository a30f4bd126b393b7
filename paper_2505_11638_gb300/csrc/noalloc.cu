// Nystrom preconditioner apply for callers that cannot allocate device memory.
//
// Some callers cannot call cudaMalloc: applications whose device memory is owned by their
// own pool allocator (which reserves the device and forbids other allocations), and
// latency-critical loops in which cudaMalloc's implicit device-wide synchronisation is not
// acceptable.  ngd_precond_apply needs a context, and a context allocates its workspace.
// ngd_precond_apply_noalloc runs the same two kernels on caller-owned inputs and outputs and
// takes its only scratch (the ell projections U^T v) from the fixed array below, which is
// compiled into the library: every GPU that loads the library holds it until the process exits.
#include <cuda_runtime.h>

#include <mutex>

#include "linalg.cuh"

namespace {

// Scratch of ngd_precond_apply_noalloc: one double per Nystrom column, NGD_NOALLOC_MAX_ELL of
// them (8 KB).  Shared by every call in the process.
static __device__ __align__(256) double g_noalloc_w1[NGD_NOALLOC_MAX_ELL];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
double* g_scratch_addr[kMaxDevices] = {};

// Device address of the scratch array on the current device.  In host code the array's name
// only stands in for the symbol, so the address is looked up once per device with that device
// current.  Returns nullptr on failure.
double* scratch_on_current_device(cudaError_t* err) {
  int dev = 0;
  *err = cudaGetDevice(&dev);
  if (*err != cudaSuccess || dev < 0 || dev >= kMaxDevices) return nullptr;
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    *err = cudaGetSymbolAddress(&p, g_noalloc_w1);
    if (*err != cudaSuccess) return nullptr;
    g_scratch_addr[dev] = static_cast<double*>(p);
  }
  return g_scratch_addr[dev];
}

}  // namespace

extern "C" ngd_status ngd_precond_apply_noalloc(int dtype, int64_t p, int ell, const void* U, int64_t ldU,
                                                const double* lam, double mu, const double* v, double* z,
                                                void* stream) {
  if (dtype != NGD_F64 && dtype != NGD_F32) return NGD_ERR_INVALID_ARG;
  if (p < 1 || ell < 1 || ell > p || ldU < p || !U || !lam || !v || !z || v == z || !(mu >= 0.0))
    return NGD_ERR_INVALID_ARG;
  if (ell > NGD_NOALLOC_MAX_ELL) return NGD_ERR_UNSUPPORTED;
  cudaError_t err = cudaSuccess;
  double* w1 = scratch_on_current_device(&err);
  if (!w1) return NGD_ERR_CUDA;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  // k_utv writes all ell entries of the scratch before k_precond_apply reads them, so nothing
  // has to be cleared between calls.
  if (dtype == NGD_F32)
    ngd::launch_precond<float>(static_cast<const float*>(U), ldU, p, ell, lam, mu, nullptr, v, z, w1, nullptr, s);
  else
    ngd::launch_precond<double>(static_cast<const double*>(U), ldU, p, ell, lam, mu, nullptr, v, z, w1, nullptr, s);
  return cudaGetLastError() == cudaSuccess ? NGD_OK : NGD_ERR_CUDA;
}
