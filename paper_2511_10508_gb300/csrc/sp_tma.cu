// sp_tma.cu -- host side of the tensor-map (TMA) plane loads: the tensor maps
// of a 3D field for the plane-ring kernel's boxes (cuTensorMapEncodeTiled,
// resolved from the driver at first use).
#include <mutex>

#include "sp_internal.h"

namespace sp {

typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                  const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static EncodeTiledFn encoder() {
    static std::once_flag once;
    static EncodeTiledFn fn = nullptr;
    std::call_once(once, [] {
        void *f = nullptr;
        cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) !=
                cudaSuccess ||
            q != cudaDriverEntryPointSuccess) {
            cudaGetLastError();
            f = nullptr;
        }
        fn = reinterpret_cast<EncodeTiledFn>(f);
    });
    return fn;
}

bool tma_available() { return encoder() != nullptr; }

cudaError_t encode_plane_maps(TmaMaps *maps, bool bf16, const void *f0, const void *f1, int nx, int ny, int nz,
                              int box_x, int box_y) {
    EncodeTiledFn enc = encoder();
    if (!enc) return cudaErrorNotSupported;
    const size_t es = bf16 ? 2 : 4;
    const cuuint64_t dims[3] = {(cuuint64_t)nx, (cuuint64_t)ny, (cuuint64_t)nz};
    const cuuint64_t strides[2] = {(cuuint64_t)nx * es, (cuuint64_t)nx * (cuuint64_t)ny * es};
    const cuuint32_t box[3] = {(cuuint32_t)box_x, (cuuint32_t)box_y, 1};
    const cuuint32_t estr[3] = {1, 1, 1};
    const void *src[2] = {f0, f1};
    for (int f = 0; f < 2; ++f) {
        const CUresult r = enc(&maps->m[f], bf16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32,
                               3, const_cast<void *>(src[f]), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                               CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_NONE,
                               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        if (r != CUDA_SUCCESS) return cudaErrorInvalidValue;
    }
    return cudaSuccess;
}

}  // namespace sp
