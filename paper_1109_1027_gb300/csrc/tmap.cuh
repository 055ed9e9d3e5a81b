// tmap.cuh -- host-side construction of TMA tensor maps (cuTensorMapEncodeTiled,
// reached through the runtime's driver entry point, so the library does not
// link libcuda) for row boxes over complex and real 2D grids.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <mutex>

namespace nlse {

using EncodeTiled = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                 const cuuint64_t*, const cuuint32_t*, const cuuint32_t*,
                                 CUtensorMapInterleave, CUtensorMapSwizzle, CUtensorMapL2promotion,
                                 CUtensorMapFloatOOBfill);

inline EncodeTiled encoder() {
    static EncodeTiled fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess && q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiled>(p);
    });
    return fn;
}

inline bool encode(CUtensorMap* m, CUtensorMapDataType type, int rank, const void* base, const cuuint64_t* dims,
            const cuuint64_t* strides, const cuuint32_t* box) {
    EncodeTiled fn = encoder();
    if (!fn || !base) return false;
    const cuuint32_t ones[3] = {1, 1, 1};
    return fn(m, type, (cuuint32_t)rank, const_cast<void*>(base), dims, strides, box, ones,
              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// Row boxes `width` points wide over an nx x ny complex grid.
template <typename R>
inline bool complex_map(CUtensorMap* m, const void* base, int nx, int ny, int width) {
    if constexpr (sizeof(R) == 4) {
        cuuint64_t dims[2] = {(cuuint64_t)nx, (cuuint64_t)ny};
        cuuint64_t strides[1] = {(cuuint64_t)nx * 8};
        cuuint32_t box[2] = {(cuuint32_t)width, 1};
        return encode(m, CU_TENSOR_MAP_DATA_TYPE_UINT64, 2, base, dims, strides, box);
    } else {
        cuuint64_t dims[3] = {2, (cuuint64_t)nx, (cuuint64_t)ny};
        cuuint64_t strides[2] = {16, (cuuint64_t)nx * 16};
        cuuint32_t box[3] = {2, (cuuint32_t)width, 1};
        return encode(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 3, base, dims, strides, box);
    }
}

template <typename R>
inline bool real_map(CUtensorMap* m, const void* base, int nx, int ny, int width) {
    cuuint64_t dims[2] = {(cuuint64_t)nx, (cuuint64_t)ny};
    cuuint64_t strides[1] = {(cuuint64_t)nx * sizeof(R)};
    cuuint32_t box[2] = {(cuuint32_t)width, 1};
    return encode(m, sizeof(R) == 4 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 2, base,
                  dims, strides, box);
}

}  // namespace nlse
