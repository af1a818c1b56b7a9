// TMA-pipelined step kernel (placeholder until the pipelined kernel lands).
#include "mmod_internal.h"
#include "tma_plan.h"

namespace mmod {

bool make_tma_plan(const mmod_config &, int, float *const *, const float *, CUtensorMap *,
                   CUtensorMap *, CUtensorMap *, TmaPlan *) {
    return false;
}

cudaError_t launch_step_tma(const StepArgs &, const CUtensorMap *, const CUtensorMap *,
                            const CUtensorMap *, const TmaPlan &, cudaStream_t) {
    return cudaErrorNotSupported;
}

}  // namespace mmod
