// Discrete energy without any allocation (sophie_energy_noalloc).
//
// Some callers cannot allocate device memory at the point where they need
// the energy: code that records the step loop into a CUDA graph (cudaMalloc
// may not be called while a stream is being captured), or a host under a
// fixed device-memory budget that reserves everything up front. This variant
// of the energy reduction keeps its per-block partial sums in a file-scope
// static device array instead of a buffer allocated at run time.
//
// The array is a host-side stand-in in host code: its device address is
// fetched once per device, with that device current, by cudaGetSymbolAddress.
// The first call on a device does that set-up, so it should come before any
// stream capture. The array holds at most kMaxBlocks partial sums; every call
// overwrites every slot it later reads, and calls that overlap on the GPU
// race on it.
#include <cuda_runtime.h>

#include <mutex>

#include "sophie_internal.h"

namespace sophie {

namespace {

constexpr int kMaxBlocks = 152 * 16;  // one double per reduction block: 19 KiB per device
constexpr int kMaxDevices = 64;

static __device__ __align__(256) double g_energy_partials[kMaxBlocks];

std::mutex g_mu;
double* g_addr[kMaxDevices] = {nullptr};

}  // namespace

int energy_noalloc(const StepArgs& a, const double* eps_tab, double scale, double* W_dev, cudaStream_t s,
                   const char** why) {
  const int nblocks = energy_blocks(a.d);
  if (nblocks > kMaxBlocks) {
    *why = "grid needs more reduction blocks than the static scratch holds";
    return -1;
  }
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    *why = "no current CUDA device (or device id above 63)";
    return -4;
  }
  double* scratch = nullptr;
  {
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_addr[dev]) {
      void* p = nullptr;
      const cudaError_t e = cudaGetSymbolAddress(&p, g_energy_partials);
      if (e != cudaSuccess || !p) {
        *why = cudaGetErrorString(e);
        return -4;
      }
      g_addr[dev] = static_cast<double*>(p);
    }
    scratch = g_addr[dev];
  }
  const cudaError_t e = launch_energy_scaled(a, eps_tab, scratch, nblocks, scale, W_dev, s);
  if (e != cudaSuccess) {
    *why = cudaGetErrorString(e);
    return -4;
  }
  return 0;
}

}  // namespace sophie
