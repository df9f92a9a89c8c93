// lbm_step_f16.cu -- fused step and observe kernels for f16 population storage.
#include "lbm_internal.h"
#include "lbm_step_staged.cuh"

LBM_INSTANTIATE_STORAGE(lbm::ST_F16, f16)
