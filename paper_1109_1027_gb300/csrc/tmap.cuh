// tmap.cuh -- host-side construction of TMA tensor maps (cuTensorMapEncodeTiled,
// reached through the runtime's driver entry point, so the library does not
// link libcuda) for row boxes over complex and real 2D grids.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <cstring>
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

// One tensor map, encoded by the driver on first use and then served from a
// small per-thread cache: a map holds nothing but its arguments (address,
// geometry, box), so a cached map is valid for as long as they are the same,
// and launches outside a captured graph do not re-encode theirs.
struct MapKey {
    const void* base;
    int type, rank;
    cuuint64_t dims[3], strides[2];
    cuuint32_t box[3];
};

inline bool encode(CUtensorMap* m, CUtensorMapDataType type, int rank, const void* base, const cuuint64_t* dims,
            const cuuint64_t* strides, const cuuint32_t* box) {
    EncodeTiled fn = encoder();
    if (!fn || !base || rank < 1 || rank > 3) return false;
    MapKey k;
    std::memset(&k, 0, sizeof k);
    k.base = base;
    k.type = (int)type;
    k.rank = rank;
    for (int i = 0; i < rank; ++i) {
        k.dims[i] = dims[i];
        k.box[i] = box[i];
        if (i + 1 < rank) k.strides[i] = strides[i];
    }
    constexpr int kCache = 64;
    struct Slot { MapKey k; CUtensorMap m; bool used; };
    thread_local Slot cache[kCache];
    thread_local int next = 0;
    for (const Slot& s : cache)
        if (s.used && std::memcmp(&s.k, &k, sizeof k) == 0) {
            *m = s.m;
            return true;
        }
    const cuuint32_t ones[3] = {1, 1, 1};
    if (fn(m, type, (cuuint32_t)rank, const_cast<void*>(base), dims, strides, box, ones,
           CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
           CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
        return false;
    Slot& s = cache[next];
    next = (next + 1) % kCache;
    s.k = k;
    s.m = *m;
    s.used = true;
    return true;
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
