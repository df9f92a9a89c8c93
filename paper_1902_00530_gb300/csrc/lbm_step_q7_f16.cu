// lbm_step_q7_f16.cu -- D2Q7 step and observe kernels for f16 population storage.
#include "lbm_internal.h"
#include "lbm_step_q7_staged.cuh"

LBM_INSTANTIATE_Q7(lbm::ST_F16, f16)
