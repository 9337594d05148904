// The temporally blocked step kernel for kF24 field storage (yee_blocked.cuh).
#include "yee_blocked.cuh"

namespace sophie {

cudaError_t launch_blocked_f24(const StepArgs& a, const CUtensorMap& tmF, const CUtensorMap& tmM,
                               const BlockedTiling& t, cudaStream_t s) {
  return launch_fmt<kF24>(a, tmF, tmM, t, s);
}

}  // namespace sophie
