// Fused step kernel instantiations: D3Q19, __nv_bfloat16 storage.
#include "lbm_step_inst.cuh"
LBM_DEFINE_STEP_UNIT(launch_step_q19_bf16, 19, __nv_bfloat16)
