// Four-cell step kernel instantiations for the channel (variants 14 and 16):
// D3Q19, float storage, halfway bounce-back walls in y with a body force, BGK
// and KC-MP.
#include "lbm_step_v4_inst.cuh"

namespace lbmk {

cudaError_t launch_v4_walls_q19(int closure, int ty, bool tma, const StepArgs* a, int nbatch, cudaStream_t s)
{
    constexpr int Q = 19;
    using S = float;
#define LBM_V4W_CASE(CL, TYV, LPRV)                                                                   \
    if (closure == CL && ty == TYV)                                                                   \
        return a ? launch_v4_t<Q, S, CL, LPRV, BC_WALLS_Y>(*a, nbatch, s, tma)                        \
                 : (nbatch < 0 ? prepare_v4_t<Q, S, CL, LPRV, BC_WALLS_Y>() : cudaSuccess);
    LBM_V4W_CASE(CL_KCMP, 8, 32)
    LBM_V4W_CASE(CL_BGK, 8, 32)
    LBM_V4W_CASE(CL_KCMP, 16, 16)
    LBM_V4W_CASE(CL_BGK, 16, 16)
#undef LBM_V4W_CASE
    return cudaErrorNotSupported;
}

}  // namespace lbmk
