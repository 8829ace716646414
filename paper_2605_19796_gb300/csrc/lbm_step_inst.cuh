// Instantiation helper: each lbm_step_q<Q>_<storage>.cu translation unit
// instantiates the fused step kernels for one lattice and one storage type
// (all closures, both boundary modes, the tile heights the tuner may pick), so
// the units compile in parallel.
//
// Variants: 1 register pull (step_kernel, every closure and storage), 8 split
// arrive/wait barrier (step_kernel_sb), 12 variant 8 with L2 prefetches, 13
// variant 8 with the own pulls copied to the
// stash by cp.async one plane ahead (32- and 64-bit storage), 14 four cells per
// thread with vector access and a tensor-memory stash (step_kernel_v4; periodic
// D3Q27, 32- and 16-bit storage; BGK, KC-MP, KC-RB and the learned closure),
// 15 the learned closure with the network on the tcgen05 tensor cores
// (step_kernel_tc, 32 x 4 tiles), 16 variant 14 with the interior of the
// staged rows copied by TMA.
#pragma once

#include "lbm_step.cuh"
#include "lbm_step_split.cuh"
#include "lbm_step_tc.cuh"

#include <type_traits>

namespace lbmk {

// four-cell kernels of lattice Q with storage S (variants 14 and 16), defined
// in lbm_step_v4_*.cu (FP32, FP16 and BF16 storage of either lattice); same
// conventions as launch_step_qs
template <int Q, typename S>
cudaError_t launch_v4_qs(int closure, int bc, int ty, bool tma, const StepArgs* a, int nbatch, cudaStream_t s);

// a == nullptr, nbatch == 0: only report whether the combination is instantiated;
// a == nullptr, nbatch == -1: set the kernel's shared-memory attribute (prepare).
template <int Q, typename S>
cudaError_t launch_step_qs(int closure, int bc, int ty, int variant, const StepArgs* a, int nbatch, cudaStream_t s)
{
    constexpr bool R32 = sizeof(typename StoreTraits<S>::R) == 4;
    if (variant == VAR_VEC4 || variant == VAR_VEC4_TMA) {
        // the four-cell kernels live in their own translation units (lbm_step_v4_*.cu)
        if constexpr (Q == 27 && R32) return launch_v4_qs<27, S>(closure, bc, ty, variant == VAR_VEC4_TMA, a, nbatch, s);
        if constexpr (Q == 19 && R32) return launch_v4_qs<19, S>(closure, bc, ty, variant == VAR_VEC4_TMA, a, nbatch, s);
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
        if constexpr (Q == 27) {
            LBM_SB_CASE(CL_KCRR, BC_PERIODIC, 8)
        }
        if constexpr (R32) {
            LBM_SB_CASE(CL_KCMP, BC_PERIODIC, 4)
            LBM_SB_CASE(CL_KCMP, BC_PERIODIC, 16)
            LBM_SB_CASE(CL_LEARNED, BC_PERIODIC, 8)
            LBM_SB_CASE(CL_LEARNED, BC_PERIODIC, 4)
        }
#undef LBM_SB_CASE
        return cudaErrorNotSupported;
    }
    if (variant == VAR_SPLIT_PF) {
#define LBM_SBP_CASE(CL, BCV, TYV)                                                              \
    if (closure == CL && bc == BCV && ty == TYV)                                                \
        return a ? launch_sb_t<Q, S, CL, BCV, TYV, true>(*a, nbatch, s) : (nbatch < 0 ? prepare_sb_t<Q, S, CL, BCV, TYV, true>() : cudaSuccess);
        LBM_SBP_CASE(CL_BGK, BC_PERIODIC, 8)
        LBM_SBP_CASE(CL_KCMP, BC_PERIODIC, 8)
        LBM_SBP_CASE(CL_KCRB_H, BC_PERIODIC, 8)
        LBM_SBP_CASE(CL_KCRB_RAW, BC_PERIODIC, 8)
        LBM_SBP_CASE(CL_BGK, BC_WALLS_Y, 8)
        LBM_SBP_CASE(CL_KCMP, BC_WALLS_Y, 8)
        if constexpr (Q == 27) {
            LBM_SBP_CASE(CL_KCRR, BC_PERIODIC, 8)
        }
        if constexpr (R32) {
            LBM_SBP_CASE(CL_LEARNED, BC_PERIODIC, 8)
            LBM_SBP_CASE(CL_LEARNED, BC_PERIODIC, 4)
        }
#undef LBM_SBP_CASE
        return cudaErrorNotSupported;
    }
    if (variant == VAR_ASYNC) {
        if constexpr (sizeof(S) == sizeof(typename StoreTraits<S>::R)) {
#define LBM_AS_CASE(CL, BCV, TYV)                                                               \
    if (closure == CL && bc == BCV && ty == TYV)                                                \
        return a ? launch_sb_t<Q, S, CL, BCV, TYV, false, true>(*a, nbatch, s)                  \
                 : (nbatch < 0 ? prepare_sb_t<Q, S, CL, BCV, TYV, false, true>() : cudaSuccess);
            LBM_AS_CASE(CL_BGK, BC_PERIODIC, 8)
            LBM_AS_CASE(CL_KCMP, BC_PERIODIC, 8)
            LBM_AS_CASE(CL_KCRB_H, BC_PERIODIC, 8)
            LBM_AS_CASE(CL_KCRB_RAW, BC_PERIODIC, 8)
            LBM_AS_CASE(CL_BGK, BC_WALLS_Y, 8)
            LBM_AS_CASE(CL_KCMP, BC_WALLS_Y, 8)
            if constexpr (Q == 27) {
                LBM_AS_CASE(CL_KCRR, BC_PERIODIC, 8)
            }
#undef LBM_AS_CASE
        }
        return cudaErrorNotSupported;
    }
    if (variant == VAR_TCNET) {
        // the learned closure's register pull on 32 x 4 tiles with the network
        // on the tcgen05 tensor cores (one 128-row GEMM per layer and CTA)
        if constexpr (R32) {
            if (closure == CL_LEARNED && bc == BC_PERIODIC && ty == 4)
                return a ? launch_tc_t<Q, S>(*a, nbatch, s) : (nbatch < 0 ? prepare_tc_t<Q, S>() : cudaSuccess);
        }
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
    if constexpr (R32) {
        LBM_STEP_CASE(CL_KCMP, BC_PERIODIC, 4)
        LBM_STEP_CASE(CL_KCMP, BC_PERIODIC, 16)
        LBM_STEP_CASE(CL_LEARNED, BC_PERIODIC, 8)
        LBM_STEP_CASE(CL_LEARNED, BC_PERIODIC, 4)
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
