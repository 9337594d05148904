// Device-side checks used by the self-test and guard entry points.
#include "sophie_internal.h"
#include "tma_util.cuh"

namespace sophie {

namespace {

// One thread waits, with the bounded wait of the step kernels, for phase 0 of
// an mbarrier whose arrival count is never reached (nothing arrives). The
// wait gives up after its limit; the kernel records code 32 in the error word
// and returns normally.
__global__ void wait_timeout_kernel(int* err, unsigned long long* waited_ns) {
  __shared__ __align__(8) unsigned long long bar;
  if (threadIdx.x != 0) return;
  const uint32_t b = smem_u32(&bar);
  mbar_init(b, 1);
  fence_mbar_init();
  const unsigned long long t0 = globaltimer_ns();
  const bool done = mbar_wait(b, 0);
  *waited_ns = globaltimer_ns() - t0;
  if (!done) atomicOr(err, 32);
}

// Count the bytes of [p, p + n) that differ from `pattern`.
__global__ void guard_check_kernel(const unsigned char* p, size_t n, unsigned char pattern,
                                   unsigned long long* bad) {
  unsigned long long local = 0;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    local += p[i] != pattern;
  if (local) atomicAdd(bad, local);
}

}  // namespace

cudaError_t launch_wait_timeout(int* err, unsigned long long* waited_ns, cudaStream_t s) {
  wait_timeout_kernel<<<1, 32, 0, s>>>(err, waited_ns);
  return cudaGetLastError();
}

cudaError_t launch_guard_check(const void* p, size_t n, unsigned char pattern, unsigned long long* bad,
                               cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  guard_check_kernel<<<152 * 2, 256, 0, s>>>(static_cast<const unsigned char*>(p), n, pattern, bad);
  return cudaGetLastError();
}

}  // namespace sophie
