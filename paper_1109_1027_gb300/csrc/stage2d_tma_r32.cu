// stage2d_tma_r32.cu -- the TMA-fed 2D stage kernels with 32 rows per CTA.
#include "stage2d_tma.cuh"

namespace nlse {

cudaError_t launch_stage_2d_tma_rows32(const StageLaunch& L, cudaStream_t st) {
    return tma2d::launch_rows<32>(L, st);
}

}  // namespace nlse
