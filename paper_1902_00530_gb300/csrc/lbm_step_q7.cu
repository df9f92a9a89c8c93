// lbm_step_q7.cu -- the D2Q7 step and observe kernels for every storage type.
#include "lbm_internal.h"
#include "lbm_step_q7.cuh"

namespace lbm {

cudaError_t launch_step_q7(int storage, int model, int vec, bool sample, int noise, const StepArgs &a, int blocks,
                           int warps, cudaStream_t stream)
{
    if (storage == ST_F32) return launch_step_q7_storage<ST_F32>(model, vec, sample, noise, a, blocks, warps, stream);
    if (storage == ST_F16) return launch_step_q7_storage<ST_F16>(model, vec, sample, noise, a, blocks, warps, stream);
    return launch_step_q7_storage<ST_BF16>(model, vec, sample, noise, a, blocks, warps, stream);
}

cudaError_t launch_observe_q7(int storage, int vec, const StepArgs &a, int blocks, int warps, cudaStream_t stream)
{
    if (storage == ST_F32) return launch_observe_q7_storage<ST_F32>(vec, a, blocks, warps, stream);
    if (storage == ST_F16) return launch_observe_q7_storage<ST_F16>(vec, a, blocks, warps, stream);
    return launch_observe_q7_storage<ST_BF16>(vec, a, blocks, warps, stream);
}

}  // namespace lbm
