// lbm_step_f16.cu -- fused step (per-step and persistent launches) and observe kernels
// for f16 population storage.
#include "lbm_internal.h"
#include "lbm_step_staged.cuh"
#include "lbm_step_persistent.cuh"

LBM_INSTANTIATE_STORAGE(lbm::ST_F16, f16)
LBM_INSTANTIATE_PERSISTENT(9, lbm::ST_F16, f16)
