// lbm_step_q7_f16.cu -- D2Q7 step (per-step and persistent launches) and observe kernels for
// f16 population storage.
#include "lbm_internal.h"
#include "lbm_step_q7_staged.cuh"

LBM_INSTANTIATE_Q7(lbm::ST_F16, f16)
LBM_INSTANTIATE_PERSISTENT(7, lbm::ST_F16, q7_f16)
