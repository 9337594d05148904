// The temporally blocked step kernel for kBF16 field storage (yee_blocked.cuh).
#include "yee_blocked.cuh"

namespace sophie {

cudaError_t launch_blocked_bf16(const StepArgs& a, const CUtensorMap& tmF, const CUtensorMap& tmM,
                               const BlockedTiling& t, cudaStream_t s) {
  // six equal scales: the unit-scale form (no scale multiplications)
  return a.fold ? launch_fmt<kBF16U>(a, tmF, tmM, t, s) : launch_fmt<kBF16>(a, tmF, tmM, t, s);
}

}  // namespace sophie
