// lbm_step_q7_f32.cu -- D2Q7 step and observe kernels for f32 population storage.
#include "lbm_internal.h"
#include "lbm_step_q7_staged.cuh"

LBM_INSTANTIATE_Q7(lbm::ST_F32, f32)
