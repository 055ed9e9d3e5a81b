// stage2d_tma_r8.cu -- the TMA-fed 2D stage kernels with 8 rows per CTA.
#include "stage2d_tma.cuh"

namespace nlse {

cudaError_t launch_stage_2d_tma_rows8(const StageLaunch& L, cudaStream_t st) {
    return tma2d::launch_rows<8>(L, st);
}

}  // namespace nlse
