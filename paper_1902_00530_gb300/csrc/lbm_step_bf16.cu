// lbm_step_bf16.cu -- fused step (per-step and persistent launches) and observe kernels
// for bf16 population storage.
#include "lbm_internal.h"
#include "lbm_step_staged.cuh"
#include "lbm_step_persistent.cuh"

LBM_INSTANTIATE_STORAGE(lbm::ST_BF16, bf16)
LBM_INSTANTIATE_PERSISTENT(9, lbm::ST_BF16, bf16)
