// adjoint2d_tma_r32.cu -- the TMA-fed 2D adjoint stage kernels with 32 rows per CTA.
#include "adjoint2d_tma.cuh"

namespace nlse {

cudaError_t launch_adjoint_2d_tma_rows32(const AdjLaunch& A, cudaStream_t st) {
    return adjtma::launch_rows<32>(A, st);
}

}  // namespace nlse
