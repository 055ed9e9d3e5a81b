// adjoint2d_tma_r8.cu -- the TMA-fed 2D adjoint stage kernels with 8 rows per CTA.
#include "adjoint2d_tma.cuh"

namespace nlse {

cudaError_t launch_adjoint_2d_tma_rows8(const AdjLaunch& A, cudaStream_t st) {
    return adjtma::launch_rows<8>(A, st);
}

}  // namespace nlse
