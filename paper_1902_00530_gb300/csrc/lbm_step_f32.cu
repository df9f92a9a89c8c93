// lbm_step_f32.cu -- fused step and observe kernels for f32 population storage.
#include "lbm_internal.h"
#include "lbm_step_staged.cuh"

LBM_INSTANTIATE_STORAGE(lbm::ST_F32, f32)
