// elsar_sort_noalloc: the whole sort for callers that cannot allocate device
// memory.  Some callers may not call cudaMalloc at all: code running inside a
// plugin or callback whose host runtime forbids device allocation, code whose
// device memory is fully reserved by another allocator, and latency-critical
// code that must never trigger the device-wide synchronisation of cudaFree.
// For them this entry point takes only the input and output records and uses
// a fixed scratch area compiled into the library instead of a caller
// workspace.  The paper has no counterpart; it is an interface convenience.
#include <cstdio>
#include <mutex>

#include "../../include/elsar.h"
#include "common.cuh"

namespace elsar {
void set_last_error(const char* msg);
}

namespace {

// Scratch of every call on this device.  It exists on each GPU that loads
// the library, for the life of the process.
static __device__ __align__(256) uint8_t g_noalloc_scratch[ELSAR_NOALLOC_SCRATCH_BYTES];

constexpr int kMaxDevices = 256;
std::mutex g_mu;
void* g_scratch_ptr[kMaxDevices] = {};

}  // namespace

extern "C" elsar_status elsar_sort_noalloc(const void* d_in, void* d_out, uint64_t n, const elsar_params* p,
                                           elsar_stream_t stream) {
  const size_t need = elsar_workspace_size(n, p);
  if (need == 0) return ELSAR_EINVAL;  // parameters rejected; elsar_last_error() says why
  if (need > (size_t)ELSAR_NOALLOC_SCRATCH_BYTES) {
    char msg[200];
    snprintf(msg, sizeof msg, "elsar_sort_noalloc: %llu records need %zu bytes of scratch; the built-in scratch holds %u",
             (unsigned long long)n, need, (unsigned)ELSAR_NOALLOC_SCRATCH_BYTES);
    elsar::set_last_error(msg);
    return ELSAR_EUNSUPPORTED;
  }
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    elsar::set_last_error("elsar_sort_noalloc: no usable current device");
    return ELSAR_ECUDA;
  }
  void* scratch = nullptr;
  {
    // first call on this device: look up the device address of the scratch
    // array (in host code its name is only a stand-in, not a device address)
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_scratch_ptr[dev]) {
      void* ptr = nullptr;
      e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
      if (e != cudaSuccess || !ptr) {
        elsar::set_last_error("elsar_sort_noalloc: cudaGetSymbolAddress failed for the scratch array");
        return ELSAR_ECUDA;
      }
      g_scratch_ptr[dev] = ptr;
    }
    scratch = g_scratch_ptr[dev];
  }
  // elsar_sort clears, on the stream, every scratch word that must start at zero
  const elsar_status s = elsar_sort(d_in, d_out, n, p, scratch, ELSAR_NOALLOC_SCRATCH_BYTES, stream, nullptr);
  return (s == ELSAR_OK && n) ? elsar_wait(scratch, ELSAR_NOALLOC_SCRATCH_BYTES, stream) : s;
}
