// Nystrom preconditioner apply for callers that cannot allocate device memory.
//
// Some callers cannot call cudaMalloc: applications whose device memory is owned by their
// own pool allocator (which reserves the device and forbids other allocations), and
// latency-critical loops in which cudaMalloc's implicit device-wide synchronisation is not
// acceptable.  ngd_precond_apply needs a context, and a context allocates its workspace.
// ngd_precond_apply_noalloc runs the same two kernels on caller-owned inputs and outputs and
// takes its only scratch (the ell projections U^T v) from the fixed array below, which is
// compiled into the library: every GPU that loads the library holds it until the process exits.
#include <cuda.h>
#include <cuda_runtime.h>

#include <mutex>

#include "linalg.cuh"

namespace {

// Scratch of ngd_precond_apply_noalloc: one double per Nystrom column, NGD_NOALLOC_MAX_ELL of
// them (8 KB).  Shared by every call in the process.
static __device__ __align__(256) double g_noalloc_w1[NGD_NOALLOC_MAX_ELL];

constexpr int kMaxDevices = NGD_NOALLOC_MAX_DEVICES;

// The array's device address belongs to the CUDA context that loaded the module: after a device
// reset (cudaDeviceReset, or the primary context released and created again) the module is
// loaded anew and the array may sit elsewhere.  The cache therefore keeps, per device, the
// driver's unique id of the context the address was looked up in.
struct ScratchSlot {
  unsigned long long ctx_id = 0;
  double* addr = nullptr;
};
std::mutex g_setup_mutex;
ScratchSlot g_slot[kMaxDevices];

using CtxGetCurrentFn = CUresult (*)(CUcontext*);
using CtxGetIdFn = CUresult (*)(CUcontext, unsigned long long*);

// Unique id of the current context (cuCtxGetId), 0 when there is none yet or the driver does not
// offer the query; then the address is looked up on every call that finds id 0.
unsigned long long current_context_id() {
  static CtxGetCurrentFn get_current = nullptr;
  static CtxGetIdFn get_id = nullptr;
  static bool resolved = false;
  if (!resolved) {
    void* a = nullptr;
    void* b = nullptr;
    cudaDriverEntryPointQueryResult qa, qb;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &a, 12000, cudaEnableDefault, &qa) == cudaSuccess &&
        qa == cudaDriverEntryPointSuccess &&
        cudaGetDriverEntryPointByVersion("cuCtxGetId", &b, 12000, cudaEnableDefault, &qb) == cudaSuccess &&
        qb == cudaDriverEntryPointSuccess) {
      get_current = reinterpret_cast<CtxGetCurrentFn>(a);
      get_id = reinterpret_cast<CtxGetIdFn>(b);
    }
    resolved = true;
  }
  if (!get_current || !get_id) return 0;
  CUcontext c = nullptr;
  unsigned long long id = 0;
  if (get_current(&c) != CUDA_SUCCESS || !c || get_id(c, &id) != CUDA_SUCCESS) return 0;
  return id;
}

// Device address of the scratch array in the current device's current context.  In host code
// the array's name only stands in for the symbol, so the address is looked up with that device
// current: once per device and context.
ngd_status scratch_on_current_device(double** out) {
  *out = nullptr;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return NGD_ERR_CUDA;
  if (dev < 0 || dev >= kMaxDevices) return NGD_ERR_UNSUPPORTED;
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  ScratchSlot& slot = g_slot[dev];
  unsigned long long id = current_context_id();
  if (!slot.addr || id == 0 || id != slot.ctx_id) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_w1) != cudaSuccess) return NGD_ERR_CUDA;
    if (id == 0) id = current_context_id();   // the lookup made the primary context current
    slot.addr = static_cast<double*>(p);
    slot.ctx_id = id;
  }
  *out = slot.addr;
  return NGD_OK;
}

}  // namespace

extern "C" ngd_status ngd_precond_apply_noalloc(int dtype, int64_t p, int ell, const void* U, int64_t ldU,
                                                const double* lam, double mu, const double* v, double* z,
                                                void* stream) {
  if (dtype != NGD_F64 && dtype != NGD_F32) return NGD_ERR_INVALID_ARG;
  if (p < 1 || ell < 1 || ell > p || ldU < p || !U || !lam || !v || !z || v == z || !(mu >= 0.0))
    return NGD_ERR_INVALID_ARG;
  if (ell > NGD_NOALLOC_MAX_ELL) return NGD_ERR_UNSUPPORTED;
  double* w1 = nullptr;
  const ngd_status st = scratch_on_current_device(&w1);
  if (st != NGD_OK) return st;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  // k_utv writes all ell entries of the scratch before k_precond_apply reads them, so nothing
  // has to be cleared between calls.
  if (dtype == NGD_F32)
    ngd::launch_precond<float>(static_cast<const float*>(U), ldU, p, ell, lam, mu, nullptr, v, z, w1, nullptr, s);
  else
    ngd::launch_precond<double>(static_cast<const double*>(U), ldU, p, ell, lam, mu, nullptr, v, z, w1, nullptr, s);
  return cudaGetLastError() == cudaSuccess ? NGD_OK : NGD_ERR_CUDA;
}
