// tma_map.cu -- tensor maps (TMA descriptors) for the input planes of the
// 3D star temporal-blocking kernel.
//
// cuTensorMapEncodeTiled is a driver-API function; it is looked up through
// the runtime's driver entry-point query, so the library links only the
// static CUDA runtime.  Encoding is pure host work (no device call).
#include <cuda.h>
#include <cuda_runtime.h>

#include <cstring>
#include <mutex>

#include "kernels.hpp"

namespace so2dr {

namespace {
using EncodeTiledFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                   const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                   CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn() {
    static std::once_flag once;
    static EncodeTiledFn fn = nullptr;
    std::call_once(once, [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiledFn>(p);
        else
            cudaGetLastError();
    });
    return fn;
}
}  // namespace

cudaError_t encode_plane_map(CUtensorMap* map, int esize, const void* base, int64_t nx, int64_t ny, int64_t cap,
                             int box_x, int box_rows) {
    std::memset(map, 0, sizeof(*map));
    EncodeTiledFn fn = encode_fn();
    if (!fn) return cudaErrorNotSupported;
    const CUtensorMapDataType dt = esize == 4 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32
                                              : CU_TENSOR_MAP_DATA_TYPE_UINT16;  // raw 16-bit storage
    // dims innermost first: columns, rows, plane slots; strides in bytes
    const cuuint64_t dims[3] = {(cuuint64_t)nx, (cuuint64_t)ny, (cuuint64_t)cap};
    const cuuint64_t strides[2] = {(cuuint64_t)(nx * esize), (cuuint64_t)(nx * ny * esize)};
    const cuuint32_t box[3] = {(cuuint32_t)box_x, (cuuint32_t)box_rows, 1};
    const cuuint32_t estr[3] = {1, 1, 1};
    CUresult r = fn(map, dt, 3, const_cast<void*>(base), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                    CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

}  // namespace so2dr
