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
// memory), so the device address is looked up once per device with
// cudaGetSymbolAddress while that device is current, and that pointer is what the
// kernels receive.
#include <mutex>

#include "recon.h"
#include "recon_internal.h"

namespace {

static __device__ __align__(256) unsigned char g_scratch[RECON_NOALLOC_SCRATCH_BYTES];

constexpr int kMaxDevices = 256;
std::mutex g_mutex;
void* g_scratch_ptr[kMaxDevices] = {};

}  // namespace

extern "C" int recon_run_noalloc(recon_plan_t plan, const float* images, float* volume, void* stream) {
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    recon::set_last_error("recon_run_noalloc: cudaGetDevice failed or device index out of range");
    return RECON_E_CUDA;
  }
  void* ptr = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_mutex);
    if (!g_scratch_ptr[dev]) {
      void* p = nullptr;
      e = cudaGetSymbolAddress(&p, g_scratch);
      if (e != cudaSuccess || !p) {
        recon::set_last_error("recon_run_noalloc: cudaGetSymbolAddress of the static scratch failed");
        return RECON_E_CUDA;
      }
      g_scratch_ptr[dev] = p;
    }
    ptr = g_scratch_ptr[dev];
  }
  return recon::run_in_scratch(plan, images, volume, static_cast<char*>(ptr), RECON_NOALLOC_SCRATCH_BYTES,
                               (cudaStream_t)stream);
}
