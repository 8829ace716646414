// Instantiation helper: each lbm_step_q<Q>_<storage>.cu translation unit
// instantiates the fused step kernel for one lattice and one storage type
// (all closures, both boundary modes, the tile heights the tuner may pick), so
// the units compile in parallel.
#pragma once

#include "lbm_step.cuh"
#include "lbm_step_async.cuh"
#include "lbm_step_tma.cuh"
#include "lbm_step_pf.cuh"
#include "lbm_step_split.cuh"
#include "lbm_step_x2.cuh"

#include <type_traits>

namespace lbmk {

// a == nullptr, nbatch == 0: only report whether the combination is instantiated;
// a == nullptr, nbatch == -1: set the kernel's shared-memory attribute (prepare).
template <int Q, typename S>
cudaError_t launch_step_qs(int closure, int bc, int ty, int variant, const StepArgs* a, int nbatch, cudaStream_t s)
{
    if constexpr (std::is_same_v<S, float>) {
        if (variant == VAR_TMA) {
#define LBM_TMA_CASE(CL, TYV, NSV)                                                                          \
    if (closure == CL && bc == BC_PERIODIC && ty == TYV)                                                \
        return a ? launch_step_tma_t<Q, CL, TYV, NSV>(*a, nbatch, s)                                    \
                 : (nbatch < 0 ? prepare_tma_t<Q, CL, TYV, NSV>() : cudaSuccess);
            LBM_TMA_CASE(CL_BGK, 8, 4)
            LBM_TMA_CASE(CL_KCMP, 8, 4)
            LBM_TMA_CASE(CL_KCRB_H, 8, 4)
            LBM_TMA_CASE(CL_KCRB_RAW, 8, 4)
            LBM_TMA_CASE(CL_KCMP, 4, 3)
#undef LBM_TMA_CASE
            return cudaErrorNotSupported;
        }
        if (variant == VAR_ASYNC) {
#define LBM_ASYNC_CASE(CL, TYV)                                                                          \
    if (closure == CL && bc == BC_PERIODIC && ty == TYV)                                               \
        return a ? launch_step_async_t<Q, CL, TYV>(*a, nbatch, s) : (nbatch < 0 ? prepare_async_t<Q, CL, TYV>() : cudaSuccess);
            LBM_ASYNC_CASE(CL_BGK, 8)
            LBM_ASYNC_CASE(CL_KCMP, 8)
            LBM_ASYNC_CASE(CL_KCRB_H, 8)
            LBM_ASYNC_CASE(CL_KCRB_RAW, 8)
            LBM_ASYNC_CASE(CL_KCMP, 4)
            LBM_ASYNC_CASE(CL_KCMP, 16)
#undef LBM_ASYNC_CASE
            return cudaErrorNotSupported;
        }
    }
    if constexpr (sizeof(typename StoreTraits<S>::R) == 4) {
        if (variant == VAR_REGISTER_OCC3) {
            if (closure == CL_KCMP && bc == BC_PERIODIC && ty == 8)
                return a ? launch_step_t<Q, S, CL_KCMP, BC_PERIODIC, 8, 3>(*a, nbatch, s) : (nbatch < 0 ? prepare_step_t<Q, S, CL_KCMP, BC_PERIODIC, 8, 3>() : cudaSuccess);
            if (closure == CL_BGK && bc == BC_PERIODIC && ty == 8)
                return a ? launch_step_t<Q, S, CL_BGK, BC_PERIODIC, 8, 3>(*a, nbatch, s) : (nbatch < 0 ? prepare_step_t<Q, S, CL_BGK, BC_PERIODIC, 8, 3>() : cudaSuccess);
            return cudaErrorNotSupported;
        }
    }
    if (variant == VAR_PREFETCH) {
#define LBM_PF_CASE(CL, BCV, TYV)                                                               \
    if (closure == CL && bc == BCV && ty == TYV)                                                \
        return a ? launch_pf_t<Q, S, CL, BCV, TYV>(*a, nbatch, s) : (nbatch < 0 ? prepare_pf_t<Q, S, CL, BCV, TYV>() : cudaSuccess);
        LBM_PF_CASE(CL_BGK, BC_PERIODIC, 8)
        LBM_PF_CASE(CL_KCMP, BC_PERIODIC, 8)
        LBM_PF_CASE(CL_KCRB_H, BC_PERIODIC, 8)
        LBM_PF_CASE(CL_KCRB_RAW, BC_PERIODIC, 8)
        LBM_PF_CASE(CL_BGK, BC_WALLS_Y, 8)
        LBM_PF_CASE(CL_KCMP, BC_WALLS_Y, 8)
        if constexpr (sizeof(typename StoreTraits<S>::R) == 4) {
            LBM_PF_CASE(CL_KCMP, BC_PERIODIC, 4)
            LBM_PF_CASE(CL_KCMP, BC_PERIODIC, 16)
        }
#undef LBM_PF_CASE
        return cudaErrorNotSupported;
    }
    if (variant == VAR_SPLIT) {
#define LBM_SB_CASE(CL, BCV, TYV)                                                               \
    if (closure == CL && bc == BCV && ty == TYV)                                                \
        return a ? launch_sb_t<Q, S, CL, BCV, TYV>(*a, nbatch, s) : (nbatch < 0 ? prepare_sb_t<Q, S, CL, BCV, TYV>() : cudaSuccess);
        LBM_SB_CASE(CL_BGK, BC_PERIODIC, 8)
        LBM_SB_CASE(CL_KCMP, BC_PERIODIC, 8)
        LBM_SB_CASE(CL_KCRB_H, BC_PERIODIC, 8)
        LBM_SB_CASE(CL_KCRB_RAW, BC_PERIODIC, 8)
        LBM_SB_CASE(CL_BGK, BC_WALLS_Y, 8)
        LBM_SB_CASE(CL_KCMP, BC_WALLS_Y, 8)
        if constexpr (sizeof(typename StoreTraits<S>::R) == 4) {
            LBM_SB_CASE(CL_KCMP, BC_PERIODIC, 4)
            LBM_SB_CASE(CL_KCMP, BC_PERIODIC, 16)
        }
#undef LBM_SB_CASE
        return cudaErrorNotSupported;
    }
    if (variant == VAR_PAIR) {
        if constexpr (sizeof(typename StoreTraits<S>::R) == 4) {
#define LBM_X2_CASE(CL, BCV, TYV)                                                               \
    if (closure == CL && bc == BCV && ty == TYV)                                                \
        return a ? launch_x2_t<Q, S, CL, BCV, TYV>(*a, nbatch, s) : (nbatch < 0 ? prepare_x2_t<Q, S, CL, BCV, TYV>() : cudaSuccess);
            LBM_X2_CASE(CL_BGK, BC_PERIODIC, 8)
            LBM_X2_CASE(CL_KCMP, BC_PERIODIC, 8)
            LBM_X2_CASE(CL_KCRB_H, BC_PERIODIC, 8)
            LBM_X2_CASE(CL_KCRB_RAW, BC_PERIODIC, 8)
            LBM_X2_CASE(CL_BGK, BC_WALLS_Y, 8)
            LBM_X2_CASE(CL_KCMP, BC_WALLS_Y, 8)
            LBM_X2_CASE(CL_KCMP, BC_PERIODIC, 4)
#undef LBM_X2_CASE
        }
        return cudaErrorNotSupported;
    }
    if (variant == VAR_PAIR_REPULL) {
        if constexpr (sizeof(typename StoreTraits<S>::R) == 4) {
#define LBM_X2R_CASE(CL, BCV, TYV)                                                              \
    if (closure == CL && bc == BCV && ty == TYV)                                                \
        return a ? launch_x2_t<Q, S, CL, BCV, TYV, true>(*a, nbatch, s) : (nbatch < 0 ? prepare_x2_t<Q, S, CL, BCV, TYV, true>() : cudaSuccess);
            LBM_X2R_CASE(CL_BGK, BC_PERIODIC, 8)
            LBM_X2R_CASE(CL_KCMP, BC_PERIODIC, 8)
            LBM_X2R_CASE(CL_KCRB_H, BC_PERIODIC, 8)
            LBM_X2R_CASE(CL_KCRB_RAW, BC_PERIODIC, 8)
#undef LBM_X2R_CASE
        }
        return cudaErrorNotSupported;
    }
    if (variant == VAR_REPULL || variant == VAR_REPULL_OCC4) {
#define LBM_RP_CASE(CL, BCV, TYV)                                                                        \
    if (closure == CL && bc == BCV && ty == TYV) {                                                       \
        if (variant == VAR_REPULL)                                                                       \
            return a ? launch_step_t<Q, S, CL, BCV, TYV, 3, true>(*a, nbatch, s)                         \
                     : (nbatch < 0 ? prepare_step_t<Q, S, CL, BCV, TYV, 3, true>() : cudaSuccess);       \
        return a ? launch_step_t<Q, S, CL, BCV, TYV, 4, true>(*a, nbatch, s)                             \
                 : (nbatch < 0 ? prepare_step_t<Q, S, CL, BCV, TYV, 4, true>() : cudaSuccess);           \
    }
        if constexpr (sizeof(typename StoreTraits<S>::R) == 4) {
            LBM_RP_CASE(CL_BGK, BC_PERIODIC, 8)
            LBM_RP_CASE(CL_KCMP, BC_PERIODIC, 8)
            LBM_RP_CASE(CL_KCRB_H, BC_PERIODIC, 8)
            LBM_RP_CASE(CL_KCRB_RAW, BC_PERIODIC, 8)
            LBM_RP_CASE(CL_KCMP, BC_WALLS_Y, 8)
        }
#undef LBM_RP_CASE
        return cudaErrorNotSupported;
    }
    if (variant != VAR_REGISTER) return cudaErrorNotSupported;
#define LBM_STEP_CASE(CL, BCV, TYV)                                                             \
    if (closure == CL && bc == BCV && ty == TYV)                                                \
        return a ? launch_step_t<Q, S, CL, BCV, TYV>(*a, nbatch, s) : (nbatch < 0 ? prepare_step_t<Q, S, CL, BCV, TYV>() : cudaSuccess);
    LBM_STEP_CASE(CL_BGK, BC_PERIODIC, 8)
    LBM_STEP_CASE(CL_KCMP, BC_PERIODIC, 8)
    LBM_STEP_CASE(CL_KCRB_H, BC_PERIODIC, 8)
    LBM_STEP_CASE(CL_KCRB_RAW, BC_PERIODIC, 8)
    LBM_STEP_CASE(CL_BGK, BC_WALLS_Y, 8)
    LBM_STEP_CASE(CL_KCMP, BC_WALLS_Y, 8)
    LBM_STEP_CASE(CL_KCRB_H, BC_WALLS_Y, 8)
    LBM_STEP_CASE(CL_KCRB_RAW, BC_WALLS_Y, 8)
    if constexpr (Q == 27) {
        LBM_STEP_CASE(CL_KCRR, BC_PERIODIC, 8)
    }
    if constexpr (sizeof(typename StoreTraits<S>::R) == 4) {
        LBM_STEP_CASE(CL_KCMP, BC_PERIODIC, 4)
        LBM_STEP_CASE(CL_KCMP, BC_PERIODIC, 16)
        LBM_STEP_CASE(CL_LEARNED, BC_PERIODIC, 8)
    }
#undef LBM_STEP_CASE
    return cudaErrorNotSupported;
}

}  // namespace lbmk

#define LBM_DEFINE_STEP_UNIT(NAME, Q, S)                                                                   \
    namespace lbmk {                                                                                       \
    cudaError_t NAME(int closure, int bc, int ty, int variant, const StepArgs* a, int nbatch, cudaStream_t s) \
    {                                                                                                      \
        return launch_step_qs<Q, S>(closure, bc, ty, variant, a, nbatch, s);                               \
    }                                                                                                      \
    }
