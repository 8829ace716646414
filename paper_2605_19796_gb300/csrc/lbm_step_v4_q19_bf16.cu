// Four-cell step kernel instantiations (variants 14 and 16): D3Q19, __nv_bfloat16 storage.
#include "lbm_step_v4_inst.cuh"
LBM_DEFINE_V4_UNIT(19, __nv_bfloat16)
