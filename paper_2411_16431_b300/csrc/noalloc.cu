// Allocation-free conditional marginals.
//
// Some callers cannot let a library call cudaMalloc at run time: a service
// that reserves all of the device's memory for its own pool at start-up and
// must never see an allocation fail mid-request, a real-time loop that cannot
// afford the device-wide synchronisation cudaMalloc and cudaFree may cause,
// or a host process whose memory budget is fixed when it loads the library.
// sgtn_conditionals_noalloc serves them: it computes exactly what
// sgtn_conditionals computes, but every device temporary lives in the static
// array below, reserved once per device when the library's device code is
// loaded, so the call itself allocates no device memory.
#include <string>

#include "../../include/sgtn.h"
#include "handle.h"

// The scratch: file scope, 256-byte aligned, SGTN_NOALLOC_SCRATCH_BYTES bytes
// on every device that loads this library, held until the process exits.
static __device__ __align__(256) unsigned char g_noalloc_scratch[SGTN_NOALLOC_SCRATCH_BYTES];

namespace {

// Device address of the scratch on the current device, looked up on every
// call: in host code the array's name is only a host-side stand-in, and an
// address cached across calls would go stale if the application reset the
// device (cudaDeviceReset) and the module were loaded again.
void* scratch_address() {
  void* p = nullptr;
  cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
  if (e != cudaSuccess || !p)
    throw SgtnError(SGTN_ERR_CUDA, std::string("cudaGetSymbolAddress(scratch): ") + cudaGetErrorString(e));
  return p;
}

}  // namespace

extern "C" int sgtn_conditionals_noalloc(sgtn_h h, int32_t step, int32_t count, const int32_t* configs,
                                         double* out_p) {
  if (!h) return SGTN_ERR_ARG;
  try {
    SGTN_CUDA(cudaSetDevice(h->device));
    void* scratch = scratch_address();
    sgtn::PrecisionScope ps(h, true);
    sgtn::conditionals_arena(h, step, count, configs, out_p, scratch, SGTN_NOALLOC_SCRATCH_BYTES);
    h->err.clear();
    return SGTN_OK;
  } catch (const SgtnError& e) {
    h->err = e.what();
    cudaGetLastError();
    return e.code;
  } catch (const std::exception& e) {
    h->err = e.what();
    return SGTN_ERR_CUDA;
  }
}
