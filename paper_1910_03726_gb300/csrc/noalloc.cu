// FCF-relaxation + fused residual for callers that cannot allocate device
// memory.  Some callers cannot call cudaMalloc (or any allocator) at the point
// where they want to relax: code that runs under a memory manager that owns
// every device byte, real-time loops where an allocation may stall or fail,
// or plug-ins that are handed pre-sized buffers.  This entry point takes the
// caller's inputs and outputs and keeps its one piece of scratch -- the
// per-interval partial sums of the residual norm -- in a fixed-size array that
// lives in the library's own device image.
#include <cuda.h>
#include <cuda_runtime.h>

#include <cstring>
#include <mutex>
#include <string>

#include "../../include/mgrit.h"
#include "device.h"

namespace mg {

void set_error(const std::string& msg);  // driver.cpp: thread-local error text

// Scratch: one partial norm per coarse interval.  Every GPU that loads the
// library holds this array until the process exits.
constexpr int kStaticMaxIntervals = MGRIT_STATIC_MAX_INTERVALS;
static __device__ __align__(256) double g_fcf_static_partial[kStaticMaxIntervals];

// Device address of the array, looked up with the device current (in host
// code the symbol itself is only a stand-in, not an address).  It is kept per
// device together with the unique ID of the CUDA context it came from, and
// looked up again when the device's current context is another one (after a
// cudaDeviceReset the module, and with it the array, is loaded anew).  The
// context ID comes from the driver's cuCtxGetCurrent and cuCtxGetId, reached
// through cudaGetDriverEntryPoint (no link against the driver library).
struct StaticAddr {
  double* addr = nullptr;
  unsigned long long ctx_id = 0;
};
static StaticAddr g_partial_addr[128];
static std::mutex g_partial_mu;

using CtxGetCurrentFn = CUresult (*)(CUcontext*);
using CtxGetIdFn = CUresult (*)(CUcontext, unsigned long long*);

static cudaError_t current_context_id(unsigned long long* id) {
  static CtxGetCurrentFn get_current = nullptr;
  static CtxGetIdFn get_id = nullptr;
  if (!get_current || !get_id) {
    cudaDriverEntryPointQueryResult q1, q2;
    void* f1 = nullptr;
    void* f2 = nullptr;
    cudaError_t e = cudaGetDriverEntryPoint("cuCtxGetCurrent", &f1, cudaEnableDefault, &q1);
    if (e == cudaSuccess) e = cudaGetDriverEntryPoint("cuCtxGetId", &f2, cudaEnableDefault, &q2);
    if (e != cudaSuccess) return e;
    if (q1 != cudaDriverEntryPointSuccess || q2 != cudaDriverEntryPointSuccess || !f1 || !f2)
      return cudaErrorSymbolNotFound;
    get_current = reinterpret_cast<CtxGetCurrentFn>(f1);
    get_id = reinterpret_cast<CtxGetIdFn>(f2);
  }
  CUcontext ctx = nullptr;
  if (get_current(&ctx) != CUDA_SUCCESS) return cudaErrorDeviceUninitialized;
  *id = 0;
  if (ctx && get_id(ctx, id) != CUDA_SUCCESS) return cudaErrorDeviceUninitialized;
  return cudaSuccess;
}

static cudaError_t static_partial(double** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= 128) return cudaErrorInvalidDevice;
  unsigned long long id = 0;
  if ((e = current_context_id(&id)) != cudaSuccess) return e;
  std::lock_guard<std::mutex> lock(g_partial_mu);
  StaticAddr& a = g_partial_addr[dev];
  if (!a.addr || id == 0 || id != a.ctx_id) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_fcf_static_partial);  // makes the primary context current
    if (e != cudaSuccess) return e;
    if ((e = current_context_id(&id)) != cudaSuccess) return e;
    a.addr = static_cast<double*>(p);
    a.ctx_id = id;
  }
  *out = a.addr;
  return cudaSuccess;
}

static bool on_device(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

}  // namespace mg

using namespace mg;

extern "C" mgrit_status mgrit_fcf_residual_static(const double* c_old, double* c_new, double* r, double* norm2,
                                                  int32_t nx, int32_t m, int32_t n_intervals, int32_t ntaps,
                                                  const int32_t* offsets, const double* coeffs, int32_t precision,
                                                  void* stream) {
  if (n_intervals < 1 || n_intervals > kStaticMaxIntervals) {
    set_error("n_intervals must be in 1.." + std::to_string(kStaticMaxIntervals) +
              " (size of the library's static scratch array)");
    return MGRIT_ERR_INVALID;
  }
  if (nx < 8 || !slab_pair_fits(nx)) {  // two padded FP64 slabs in one CTA's shared memory
    set_error("nx must be in 8.." + std::to_string(kMaxSlabNx));
    return MGRIT_ERR_INVALID;
  }
  if (m < 1 || ntaps < 1 || ntaps > kMaxDevTaps || !offsets || !coeffs || (precision != 0 && precision != 1)) {
    set_error("bad m, taps or precision");
    return MGRIT_ERR_INVALID;
  }
  if (!c_old || !c_new || !r || !norm2 || !on_device(c_old) || !on_device(c_new) || !on_device(r) ||
      !on_device(norm2)) {
    set_error("c_old, c_new, r and norm2 must be device pointers");
    return MGRIT_ERR_INVALID;
  }
  for (int k = 0; k < ntaps; ++k) {
    if (offsets[k] <= -nx || offsets[k] >= nx) {
      set_error("tap offsets must satisfy |offset| < nx");
      return MGRIT_ERR_INVALID;
    }
  }
  DevTaps t;
  if (!make_dev_taps(offsets, coeffs, ntaps, &t)) {
    set_error("bad taps");
    return MGRIT_ERR_INVALID;
  }
  double* partial = nullptr;
  cudaError_t e = static_partial(&partial);
  if (e != cudaSuccess) {
    set_error(std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
    return MGRIT_ERR_CUDA;
  }
  cudaStream_t s = (cudaStream_t)stream;
  // the array keeps the previous call's values: the norm also sums entry 0,
  // which the relaxation never writes, so clear it
  e = cudaMemsetAsync(partial, 0, sizeof(double), s);
  if (e == cudaSuccess) {
    FcfArgs a = {};
    a.u_old = c_old;
    a.cstride = nx;
    a.c_new = c_new;
    a.g = nullptr;
    a.r = r;
    a.partial = partial;
    a.nx = nx;
    a.m = m;
    a.N = n_intervals;
    a.zero_old = 0;
    e = launch_fcf(a, t, precision, nx >= 2048 ? 512 : (nx >= 512 ? 256 : 128), s);
  }
  if (e == cudaSuccess) e = launch_norm(partial, n_intervals, norm2, s);
  if (e != cudaSuccess) {
    set_error(std::string("mgrit_fcf_residual_static: ") + cudaGetErrorString(e));
    return MGRIT_ERR_CUDA;
  }
  return MGRIT_OK;
}
