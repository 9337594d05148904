// The temporally blocked step kernel for kF16HL field storage (yee_blocked.cuh).
#include "yee_blocked.cuh"

namespace sophie {

cudaError_t launch_blocked_f16hl(const StepArgs& a, const CUtensorMap& tmF, const CUtensorMap& tmM,
                               const BlockedTiling& t, cudaStream_t s) {
  // six equal scales: the unit-scale form (no scale multiplications)
  return a.fold ? launch_fmt<kF16HLU>(a, tmF, tmM, t, s) : launch_fmt<kF16HL>(a, tmF, tmM, t, s);
}

}  // namespace sophie
