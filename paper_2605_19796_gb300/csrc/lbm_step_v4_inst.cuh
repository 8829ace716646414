// Instantiation helper of the four-cell step kernels (variants 14 and 16,
// step_kernel_v4): each lbm_step_v4_*.cu translation unit instantiates them
// for one lattice and storage type, apart from the other variants, so that the
// units compile in parallel.
#pragma once

#include <type_traits>

#include "lbm_step_v4.cuh"

namespace lbmk {

// the channel (bounce-back walls in y, body force), FP32 storage, BGK and KC-MP;
// defined in lbm_step_v4_walls.cu (D3Q27) and lbm_step_v4_q19_walls.cu (D3Q19)
cudaError_t launch_v4_walls_q27(int closure, int ty, bool tma, const StepArgs* a, int nbatch, cudaStream_t s);
cudaError_t launch_v4_walls_q19(int closure, int ty, bool tma, const StepArgs* a, int nbatch, cudaStream_t s);

template <int Q, typename S>
cudaError_t launch_v4_qs(int closure, int bc, int ty, bool tma, const StepArgs* a, int nbatch, cudaStream_t s)
{
    // tile_y 8: 128 x 8 tiles (one row per warp); 16: 64 x 16 tiles (two rows per
    // warp); tma (variant 16) stages the rows' interior by TMA (analytic closures)
    if (tma && closure == CL_LEARNED) return cudaErrorNotSupported;
    if (bc == BC_WALLS_Y) {
        if constexpr (std::is_same<S, float>::value)
            return Q == 27 ? launch_v4_walls_q27(closure, ty, tma, a, nbatch, s)
                           : launch_v4_walls_q19(closure, ty, tma, a, nbatch, s);
        return cudaErrorNotSupported;
    }
#define LBM_V4_CASE(CL, TYV, LPRV)                                                                     \
    if (closure == CL && bc == BC_PERIODIC && ty == TYV)                                               \
        return a ? launch_v4_t<Q, S, CL, LPRV>(*a, nbatch, s, tma) : (nbatch < 0 ? prepare_v4_t<Q, S, CL, LPRV>() : cudaSuccess);
    LBM_V4_CASE(CL_BGK, 8, 32)
    LBM_V4_CASE(CL_KCMP, 8, 32)
    LBM_V4_CASE(CL_KCRB_H, 8, 32)
    LBM_V4_CASE(CL_KCRB_RAW, 8, 32)
    LBM_V4_CASE(CL_BGK, 16, 16)
    LBM_V4_CASE(CL_KCMP, 16, 16)
    LBM_V4_CASE(CL_KCRB_H, 16, 16)
    LBM_V4_CASE(CL_KCRB_RAW, 16, 16)
    if constexpr (Q == 27) {  // KC-RR is defined on D3Q27
        LBM_V4_CASE(CL_KCRR, 8, 32)
        LBM_V4_CASE(CL_KCRR, 16, 16)
    }
    // the learned closure (D3Q27): its network block and exchanges fit beside
    // the FP32 staging area of 64 x 16 tiles only
    if constexpr (Q == 27) {
        LBM_V4_CASE(CL_LEARNED, 16, 16)
        if constexpr (sizeof(S) == 2) {
            LBM_V4_CASE(CL_LEARNED, 8, 32)
        }
    }
#undef LBM_V4_CASE
    return cudaErrorNotSupported;
}

}  // namespace lbmk

#define LBM_DEFINE_V4_UNIT(Q, S) \
    namespace lbmk {            \
    template cudaError_t launch_v4_qs<Q, S>(int, int, int, bool, const StepArgs*, int, cudaStream_t); \
    }
