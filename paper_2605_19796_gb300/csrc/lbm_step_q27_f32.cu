// Fused step kernel instantiations: D3Q27, float storage.
#include "lbm_step_inst.cuh"
LBM_DEFINE_STEP_UNIT(launch_step_q27_f32, 27, float)
