// stage3d_tma_z128.cu -- the TMA-fed FP32 3D stage kernels with 128 z planes per CTA.
#include "stage3d_tma.cuh"

namespace nlse {

cudaError_t launch_stage_3d_tma_planes128(const StageLaunch& L, cudaStream_t st) {
    return tma3d::launch_planes<128>(L, st);
}

}  // namespace nlse
