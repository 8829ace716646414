// Fused step kernel instantiations: D3Q27, __nv_bfloat16 storage.
#include "lbm_step_inst.cuh"
LBM_DEFINE_STEP_UNIT(launch_step_q27_bf16, 27, __nv_bfloat16)
