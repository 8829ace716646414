// Run-time dispatch of the fused step kernel over lattice x storage.
#include "lbm_internal.h"

namespace lbmk {

cudaError_t launch_step_q19_f64(int, int, int, int, const StepArgs*, int, cudaStream_t);
cudaError_t launch_step_q19_f32(int, int, int, int, const StepArgs*, int, cudaStream_t);
cudaError_t launch_step_q19_f16(int, int, int, int, const StepArgs*, int, cudaStream_t);
cudaError_t launch_step_q19_bf16(int, int, int, int, const StepArgs*, int, cudaStream_t);
cudaError_t launch_step_q27_f64(int, int, int, int, const StepArgs*, int, cudaStream_t);
cudaError_t launch_step_q27_f32(int, int, int, int, const StepArgs*, int, cudaStream_t);
cudaError_t launch_step_q27_f16(int, int, int, int, const StepArgs*, int, cudaStream_t);
cudaError_t launch_step_q27_bf16(int, int, int, int, const StepArgs*, int, cudaStream_t);

namespace {
using Fn = cudaError_t (*)(int, int, int, int, const StepArgs*, int, cudaStream_t);
Fn pick(int q, int storage)
{
    if (q == 19) {
        switch (storage) {
        case ST_F64: return launch_step_q19_f64;
        case ST_F32: return launch_step_q19_f32;
        case ST_F16S: return launch_step_q19_f16;
        case ST_BF16S: return launch_step_q19_bf16;
        }
    } else if (q == 27) {
        switch (storage) {
        case ST_F64: return launch_step_q27_f64;
        case ST_F32: return launch_step_q27_f32;
        case ST_F16S: return launch_step_q27_f16;
        case ST_BF16S: return launch_step_q27_bf16;
        }
    }
    return nullptr;
}
}  // namespace

cudaError_t launch_step(int q, int storage, int closure, int bc, int tile_y, int variant, const StepArgs& a,
                        int nbatch, cudaStream_t s)
{
    Fn f = pick(q, storage);
    if (!f) return cudaErrorNotSupported;
    return f(closure, bc, tile_y, variant, &a, nbatch, s);
}

bool step_supported(int q, int storage, int closure, int bc, int tile_y, int variant)
{
    Fn f = pick(q, storage);
    return f && f(closure, bc, tile_y, variant, nullptr, 0, nullptr) == cudaSuccess;
}

bool vec4_shape_ok(int nx) { return nx % 8 == 0; }
bool vec4_tma_shape_ok(int nx, int tile_y) { return nx % (tile_y == 16 ? 64 : 128) == 0; }

cudaError_t prepare_step(int q, int storage, int closure, int bc, int tile_y, int variant)
{
    Fn f = pick(q, storage);
    if (!f) return cudaErrorNotSupported;
    // nbatch = -1 with no arguments selects the prepare mode of the launchers
    return f(closure, bc, tile_y, variant, nullptr, -1, nullptr);
}

}  // namespace lbmk
