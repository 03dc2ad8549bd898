// recon_run_noalloc: the whole reconstruction with no device allocation at all.
//
// Some callers are not allowed to allocate GPU memory: code that runs inside a host
// application which has already partitioned the device memory among its components
// (a fixed arena handed out by the host, nothing else may call cudaMalloc), real-time
// acquisition loops in which cudaMalloc/cudaFree are forbidden because they can
// synchronise the device and stall the stream that is streaming detector frames, and
// plugins loaded into processes whose allocator owns every byte.  For them this file
// keeps the run's scratch (plan tables, spectra, per-layer intermediates, layer stacks)
// in one static device array that is part of the library image: it exists on every
// device that loads this code, from the first use until the process exits.
//
// The host cannot use the array's name as a device address (in host code it names a
// host-side shadow; a kernel handed that would fault or silently touch the wrong
// memory), so every call looks up the device address with cudaGetSymbolAddress while
// the caller's device is current, and that pointer is what the kernels receive.  The
// lookup allocates nothing and is cheap; doing it on every call (rather than caching it
// per device) keeps the address right after a cudaDeviceReset or a primary-context
// re-creation, which can reload the module at a new address.
#include "recon.h"
#include "recon_internal.h"

namespace {

static __device__ __align__(256) unsigned char g_scratch[RECON_NOALLOC_SCRATCH_BYTES];

}  // namespace

extern "C" int recon_run_noalloc(recon_plan_t plan, const float* images, float* volume, void* stream) {
  void* ptr = nullptr;
  const cudaError_t e = cudaGetSymbolAddress(&ptr, g_scratch);
  if (e != cudaSuccess || !ptr) {
    recon::set_last_error("recon_run_noalloc: cudaGetSymbolAddress of the static scratch failed");
    return RECON_E_CUDA;
  }
  return recon::run_in_scratch(plan, images, volume, static_cast<char*>(ptr), RECON_NOALLOC_SCRATCH_BYTES,
                               (cudaStream_t)stream);
}
