// Discrete energy without any allocation (sophie_energy_noalloc).
//
// Some callers cannot allocate device memory at the point where they need
// the energy: an application that reserves its whole device-memory budget up
// front (a caching allocator that owns the heap, or an embedded host that
// forbids allocation once it runs), where a cudaMalloc would fail or is not
// allowed. This variant of the energy reduction keeps its per-block partial
// sums in a file-scope static device array instead of a buffer allocated at
// run time.
//
// In host code the array's name is a host-side stand-in, not a device
// address: its device address is fetched once per device, with that device
// current, by cudaGetSymbolAddress. The first call on a device does that
// set-up, so it should come before any stream capture. The array holds
// kEnergyMaxBlocks partial sums, the most any grid's reduction uses (the
// block count is capped there and a grid-stride loop covers larger grids),
// so no grid is rejected for its size. Every call overwrites every slot it
// later reads; calls that overlap on the GPU race on the array.
#include <cuda_runtime.h>

#include <mutex>

#include "sophie_internal.h"

namespace sophie {

namespace {

constexpr int kMaxDevices = 64;

// one double per reduction block: 19 KiB per device
static __device__ __align__(256) double g_energy_partials[kEnergyMaxBlocks];

std::mutex g_mu;
double* g_addr[kMaxDevices] = {nullptr};

}  // namespace

int energy_noalloc(const StepArgs& a, const double* eps_tab, double scale, double* W_dev, cudaStream_t s,
                   const char** why) {
  const int nblocks = energy_blocks(a.d);
  if (nblocks > kEnergyMaxBlocks) {  // energy_blocks caps the count: never taken
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
