// lbm_step_q7_f32.cu -- D2Q7 step (per-step and persistent launches) and observe kernels for
// f32 population storage.
#include "lbm_internal.h"
#include "lbm_step_q7_staged.cuh"

LBM_INSTANTIATE_Q7(lbm::ST_F32, f32)
LBM_INSTANTIATE_PERSISTENT(7, lbm::ST_F32, q7_f32)
