// lbm_step_bf16.cu -- fused step and observe kernels for bf16 population storage.
#include "lbm_internal.h"
#include "lbm_step_staged.cuh"

LBM_INSTANTIATE_STORAGE(lbm::ST_BF16, bf16)
