// Tensor maps of the population buffers for the TMA step kernel.
#include <cuda.h>
#include <cuda_runtime.h>

#include "lbm_internal.h"

namespace lbmk {

bool tma_shape_ok(int nx, int ny, int tile_y) { return nx % 32 == 0 && ny % tile_y == 0; }

cudaError_t encode_population_map(void* map_out, const void* buf, int nx, int ny, int nz, int q, int nbatch, int tile_y)
{
    using EncodeFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
    static EncodeFn encode = nullptr;
    if (!encode) {
        void* fn = nullptr;
        cudaDriverEntryPointQueryResult qr;
        cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &qr);
        if (e != cudaSuccess) return e;
        if (qr != cudaDriverEntryPointSuccess || !fn) return cudaErrorNotSupported;
        encode = reinterpret_cast<EncodeFn>(fn);
    }
    const cuuint64_t dims[4] = {(cuuint64_t)nx, (cuuint64_t)ny, (cuuint64_t)nz, (cuuint64_t)q * (cuuint64_t)nbatch};
    const cuuint64_t strides[3] = {(cuuint64_t)nx * 4, (cuuint64_t)nx * ny * 4, (cuuint64_t)nx * ny * nz * 4};
    const cuuint32_t box[4] = {40u, (cuuint32_t)(tile_y + 2), 1u, 1u};
    const cuuint32_t estr[4] = {1u, 1u, 1u, 1u};
    CUresult r = encode(static_cast<CUtensorMap*>(map_out), CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, const_cast<void*>(buf),
                        dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                        CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

}  // namespace lbmk
