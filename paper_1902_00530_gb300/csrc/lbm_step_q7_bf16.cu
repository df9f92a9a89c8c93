// lbm_step_q7_bf16.cu -- D2Q7 step (per-step and persistent launches) and observe kernels for
// bf16 population storage.
#include "lbm_internal.h"
#include "lbm_step_q7_staged.cuh"

LBM_INSTANTIATE_Q7(lbm::ST_BF16, bf16)
LBM_INSTANTIATE_PERSISTENT(7, lbm::ST_BF16, q7_bf16)
