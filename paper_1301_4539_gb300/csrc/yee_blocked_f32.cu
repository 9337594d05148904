// The temporally blocked step kernel for kF32 field storage (yee_blocked.cuh).
#include "yee_blocked.cuh"

namespace sophie {

cudaError_t launch_blocked_f32(const StepArgs& a, const CUtensorMap& tmF, const CUtensorMap& tmM,
                               const BlockedTiling& t, cudaStream_t s) {
  return launch_fmt<kF32>(a, tmF, tmM, t, s);
}

}  // namespace sophie
