// selftest.cu -- a self-test of the library's failure path for bounded waits
// (no counterpart in the paper).  Every mbarrier wait of the TMA-fed kernels
// gives up after a time limit, sets the timeout bit of the context's status
// and lets the kernel return, so that a copy that never lands cannot hang the
// GPU.  This kernel runs that path on purpose: it waits, with the kernels'
// own bounded wait, on an mbarrier that nothing will complete, so the wait
// runs out, the bit is set and the kernel returns.  No copy is issued, no
// memory is touched outside the kernel's own shared barrier and the status
// word, and nothing traps.
#include "nlse.h"
#include "nlse_internal.h"
#include "tma.cuh"

namespace nlse {
namespace {

__global__ void bounded_wait_probe(int* flag, uint64_t limit_ns) {
    __shared__ alignas(8) uint64_t bar;
    const uint32_t b = smem_u32(&bar);
    if (threadIdx.x == 0) {
        mbar_init(b, 1);                  // one arrival expected; none will come
        mbar_init_fence();
    }
    __syncthreads();
    const bool landed = mbar_wait(b, 0, limit_ns);
    if (!landed && threadIdx.x == 0) atomicOr(flag, kStatusTimeout);
}

}  // namespace

cudaError_t launch_bounded_wait_probe(int* flag, double limit_ms, cudaStream_t st) {
    bounded_wait_probe<<<1, 32, 0, st>>>(flag, (uint64_t)(limit_ms * 1e6));
    return cudaGetLastError();
}

}  // namespace nlse
