// Four-cell step kernel instantiations (variants 14 and 16): D3Q19, __half storage.
#include "lbm_step_v4_inst.cuh"
LBM_DEFINE_V4_UNIT(19, __half)
