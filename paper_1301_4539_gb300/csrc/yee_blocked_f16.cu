// The temporally blocked step kernel for kF16 field storage (yee_blocked.cuh).
#include "yee_blocked.cuh"

namespace sophie {

cudaError_t launch_blocked_f16(const StepArgs& a, const CUtensorMap& tmF, const CUtensorMap& tmM,
                               const BlockedTiling& t, cudaStream_t s) {
  // six equal scales: the unit-scale form (no scale multiplications)
  return a.fold ? launch_fmt<kF16U>(a, tmF, tmM, t, s) : launch_fmt<kF16>(a, tmF, tmM, t, s);
}

}  // namespace sophie
