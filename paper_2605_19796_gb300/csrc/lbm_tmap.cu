// Tensor maps (TMA descriptors) of the population buffers for the four-cell
// step kernel's staged pulls: a buffer seen as a 4D array (x, y, z, population
// of box), the box of one copy TX x rows x 1 x 1 (rows = the staged rows of a
// tile, or 1 for the rows of tiles whose staged rows wrap around y).
#include <cuda.h>
#include <cuda_runtime.h>

#include "../../include/lbm.h"
#include "lbm_internal.h"

namespace lbmk {

cudaError_t encode_v4_map(void* map_out, const void* buf, int storage, int nx, int ny, int nz, int q, int nbatch,
                          int box_x, int box_rows)
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
    CUtensorMapDataType dt;
    cuuint64_t es;
    switch (storage) {
    case LBM_FP32: dt = CU_TENSOR_MAP_DATA_TYPE_FLOAT32; es = 4; break;
    case LBM_FP16_SHIFTED: dt = CU_TENSOR_MAP_DATA_TYPE_FLOAT16; es = 2; break;
    case LBM_BF16_SHIFTED: dt = CU_TENSOR_MAP_DATA_TYPE_BFLOAT16; es = 2; break;
    default: return cudaErrorInvalidValue;
    }
    const cuuint64_t dims[4] = {(cuuint64_t)nx, (cuuint64_t)ny, (cuuint64_t)nz, (cuuint64_t)q * (cuuint64_t)nbatch};
    const cuuint64_t strides[3] = {(cuuint64_t)nx * es, (cuuint64_t)nx * ny * es, (cuuint64_t)nx * ny * nz * es};
    const cuuint32_t box[4] = {(cuuint32_t)box_x, (cuuint32_t)box_rows, 1u, 1u};
    const cuuint32_t estr[4] = {1u, 1u, 1u, 1u};
    CUresult r = encode(static_cast<CUtensorMap*>(map_out), dt, 4, const_cast<void*>(buf), dims, strides, box, estr,
                        CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                        CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

}  // namespace lbmk
