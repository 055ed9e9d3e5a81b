// adjoint2d_tma_r16.cu -- the TMA-fed 2D adjoint stage kernels with 16 rows per CTA.
#include "adjoint2d_tma.cuh"

namespace nlse {

cudaError_t launch_adjoint_2d_tma_rows16(const AdjLaunch& A, cudaStream_t st) {
    return adjtma::launch_rows<16>(A, st);
}

}  // namespace nlse
