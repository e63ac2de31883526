// Host side of the TMA plane staging: the tensor maps of the stage input's fields, encoded by
// the driver's cuTensorMapEncodeTiled (fetched through the runtime's driver entry point, so the
// library links only the CUDA runtime).
#include <cudaTypedefs.h>
#include <stdint.h>

#include "tma.cuh"

namespace hydro {

namespace {

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
    static const PFN_cuTensorMapEncodeTiled_v12000 fn = [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                             &q) != cudaSuccess ||
            q != cudaDriverEntryPointSuccess)
            p = nullptr;
        return reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    }();
    return fn;
}

}  // namespace

cudaError_t encode_plane_maps(TmaMaps *out, const void *const planes[5], const int n[3],
                              int box_w, int box_h) {
    const PFN_cuTensorMapEncodeTiled_v12000 fn = encode_fn();
    if (!fn) return cudaErrorNotSupported;
    if (n[0] < 1 || n[1] < 1 || n[2] < 1 || n[0] % 4 != 0 || box_w < 1 || box_w > 256 ||
        box_h < 1 || box_h > 256 || (box_w * 4) % 16 != 0)
        return cudaErrorInvalidValue;
    const cuuint64_t dims[3] = {(cuuint64_t)n[0], (cuuint64_t)n[1], (cuuint64_t)n[2]};
    const cuuint64_t strides[2] = {(cuuint64_t)n[0] * 4u, (cuuint64_t)n[0] * (cuuint64_t)n[1] * 4u};
    const cuuint32_t box[3] = {(cuuint32_t)box_w, (cuuint32_t)box_h, 1u};
    const cuuint32_t estride[3] = {1u, 1u, 1u};
    for (int k = 0; k < 5; ++k) {
        if (!planes[k] || reinterpret_cast<uintptr_t>(planes[k]) % 16 != 0) return cudaErrorInvalidValue;
        const CUresult r = fn(&out->map[k], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3,
                              const_cast<void *>(planes[k]), dims, strides, box, estride,
                              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                              CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        if (r != CUDA_SUCCESS) return cudaErrorInvalidValue;
    }
    return cudaSuccess;
}

}  // namespace hydro
