// Instantiation helper: each lbm_step_q<Q>_<storage>.cu translation unit
// instantiates the fused step kernel for one lattice and one storage type
// (all closures, both boundary modes, the tile heights the tuner may pick), so
// the units compile in parallel.
#pragma once

#include "lbm_step.cuh"

namespace lbmk {

// a == nullptr: only report whether the combination is instantiated.
template <int Q, typename S>
cudaError_t launch_step_qs(int closure, int bc, int ty, const StepArgs* a, int nbatch, cudaStream_t s)
{
#define LBM_STEP_CASE(CL, BCV, TYV)                                                             \
    if (closure == CL && bc == BCV && ty == TYV)                                                \
        return a ? launch_step_t<Q, S, CL, BCV, TYV>(*a, nbatch, s) : cudaSuccess;
    LBM_STEP_CASE(CL_BGK, BC_PERIODIC, 8)
    LBM_STEP_CASE(CL_KCMP, BC_PERIODIC, 8)
    LBM_STEP_CASE(CL_KCRB_H, BC_PERIODIC, 8)
    LBM_STEP_CASE(CL_KCRB_RAW, BC_PERIODIC, 8)
    LBM_STEP_CASE(CL_BGK, BC_WALLS_Y, 8)
    LBM_STEP_CASE(CL_KCMP, BC_WALLS_Y, 8)
    LBM_STEP_CASE(CL_KCRB_H, BC_WALLS_Y, 8)
    LBM_STEP_CASE(CL_KCRB_RAW, BC_WALLS_Y, 8)
    if constexpr (sizeof(typename StoreTraits<S>::R) == 4) {
        LBM_STEP_CASE(CL_KCMP, BC_PERIODIC, 4)
        LBM_STEP_CASE(CL_KCMP, BC_PERIODIC, 16)
    }
#undef LBM_STEP_CASE
    return cudaErrorNotSupported;
}

}  // namespace lbmk

#define LBM_DEFINE_STEP_UNIT(NAME, Q, S)                                                                   \
    namespace lbmk {                                                                                       \
    cudaError_t NAME(int closure, int bc, int ty, const StepArgs* a, int nbatch, cudaStream_t s)          \
    {                                                                                                      \
        return launch_step_qs<Q, S>(closure, bc, ty, a, nbatch, s);                                        \
    }                                                                                                      \
    }
