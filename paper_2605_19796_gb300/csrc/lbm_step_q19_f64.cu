// Fused step kernel instantiations: D3Q19, double storage.
#include "lbm_step_inst.cuh"
LBM_DEFINE_STEP_UNIT(launch_step_q19_f64, 19, double)
