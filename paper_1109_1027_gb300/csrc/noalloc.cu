// noalloc.cu -- nlse_invariants_noalloc: mass, energy and the time-step bound
// without a context and without any device allocation.
//
// Some callers cannot allocate device memory themselves: code that runs
// inside a host framework which owns all device memory through its own pool
// or a fixed budget and forbids allocations outside it, and latency-critical
// paths that cannot afford the implicit device synchronisation a cudaMalloc /
// cudaFree may bring.  They cannot create an nlse_ctx (which allocates its
// work space), so this entry point runs the same two reduction kernels as
// nlse_invariants with their scratch -- one row of partial sums per block and
// the reduced row -- in a file-scope __device__ array instead.
//
// The array is loaded with the library and occupies kScratchBytes on every
// GPU that loads it until the process exits.  In host code the name g_scratch
// only stands for the symbol; its device address is looked up once per device
// with cudaGetSymbolAddress (on the first call on that device, with the
// device current) and cached.  Every call shares the array and it keeps the
// previous call's contents; nothing needs clearing because each call writes
// every row it reads before reading it.  Calls whose work overlaps on the GPU
// (different streams, no ordering) race on the array.
#include <cmath>
#include <cstdio>
#include <mutex>

#include "nlse.h"
#include "nlse_internal.h"
#include "stability.cuh"

namespace {

constexpr int kPointsPerBlock = 4096;     // one partial row per 4096 grid points
constexpr int kMaxRows = 16384;
constexpr int64_t kMaxPoints = (int64_t)kPointsPerBlock * kMaxRows;    // 67,108,864
constexpr int kScratchDoubles = (kMaxRows + 1) * nlse::kPartialWidth;
constexpr size_t kScratchBytes = sizeof(double) * kScratchDoubles;
static_assert(kScratchBytes == 786480, "the documented size of the static scratch");

static __device__ __align__(256) double g_scratch[kScratchDoubles];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
double* g_scratch_addr[kMaxDevices] = {};

// Device address of g_scratch on the current device (looked up once per device).
cudaError_t scratch_address(int dev, double** out) {
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_scratch_addr[dev]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_scratch);
        if (e != cudaSuccess) return e;
        g_scratch_addr[dev] = static_cast<double*>(p);
    }
    *out = g_scratch_addr[dev];
    return cudaSuccess;
}

int check_params(const nlse_params* p, int64_t* npts) {
    if (!p) return nlse::report_error(NLSE_EINVAL, "params is NULL");
    if (p->dim < 1 || p->dim > 3) return nlse::report_error(NLSE_EINVAL, "dim must be 1, 2 or 3");
    int64_t n = 1;
    for (int ax = 0; ax < p->dim; ++ax) {
        if (p->n[ax] < 3) return nlse::report_error(NLSE_EINVAL, "need at least 3 points per axis");
        if (p->n[ax] > kMaxPoints) break;
        n *= p->n[ax];
        if (n > kMaxPoints) break;
    }
    if (n > kMaxPoints)
        return nlse::report_error(NLSE_EINVAL,
                                  "grid exceeds the 67,108,864 points that the static scratch of "
                                  "nlse_invariants_noalloc covers; use nlse_invariants");
    if (!(std::isfinite(p->h) && p->h > 0)) return nlse::report_error(NLSE_EINVAL, "h must be positive and finite");
    if (!(std::isfinite(p->a) && p->a > 0)) return nlse::report_error(NLSE_EINVAL, "a must be positive and finite");
    if (!std::isfinite(p->s)) return nlse::report_error(NLSE_EINVAL, "s must be finite");
    if (p->bc < NLSE_BC_DIRICHLET || p->bc > NLSE_BC_LAPZERO) return nlse::report_error(NLSE_EINVAL, "unknown bc");
    if (p->prec != NLSE_FP32 && p->prec != NLSE_FP64) return nlse::report_error(NLSE_EINVAL, "unknown prec");
    if (p->lap != NLSE_LAP_2SHOC && p->lap != NLSE_LAP_CD && p->lap != NLSE_LAP_2SHOC_MS)
        return nlse::report_error(NLSE_EINVAL, "unknown lap");
    if (p->flags & NLSE_FLAG_STACK)
        return nlse::report_error(NLSE_EUNSUPPORTED, "stacked grids: use nlse_invariants");
    *npts = n;
    return NLSE_OK;
}

int cuda_error(cudaError_t e, const char* what) {
    char buf[256];
    snprintf(buf, sizeof buf, "%s: %s", what, cudaGetErrorString(e));
    return nlse::report_error(NLSE_ECUDA, buf);
}

}  // namespace

extern "C" int nlse_invariants_noalloc(const nlse_params* p, const void* psi_dev, const void* V_dev,
                                       double* mass, double* energy, double* dt_max, void* stream) {
    nlse::report_error(NLSE_OK, "");
    int64_t npts = 0;
    int rc = check_params(p, &npts);
    if (rc) return rc;
    if (!psi_dev || !V_dev) return nlse::report_error(NLSE_EINVAL, "NULL device pointer");
    if (((uintptr_t)psi_dev | (uintptr_t)V_dev) % 16)
        return nlse::report_error(NLSE_EINVAL, "device pointers must be 16-byte aligned");

    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_error(e, "cudaGetDevice");
    if (dev < 0 || dev >= kMaxDevices) return nlse::report_error(NLSE_EINVAL, "device index out of range");
    double* scratch = nullptr;
    e = scratch_address(dev, &scratch);
    if (e != cudaSuccess) return cuda_error(e, "looking up the static scratch");

    nlse::InvLaunch L;
    L.dim = p->dim;
    for (int ax = 0; ax < 3; ++ax) L.n[ax] = ax < p->dim ? p->n[ax] : 1;
    L.prec = p->prec; L.lap = p->lap; L.bc = p->bc;
    L.h = p->h; L.a = p->a; L.s = p->s;
    L.psi = psi_dev;
    L.lo = nullptr;
    L.V = V_dev;
    L.energy = energy != nullptr;
    const int nrows = (int)((npts + kPointsPerBlock - 1) / kPointsPerBlock);
    double* result = scratch + (size_t)kMaxRows * nlse::kPartialWidth;
    cudaStream_t st = (cudaStream_t)stream;
    e = nlse::launch_invariants(L, scratch, nrows, result, st);
    if (e != cudaSuccess) return cuda_error(e, "invariants launch");
    double r[nlse::kPartialWidth];
    e = cudaMemcpyAsync(r, result, sizeof r, cudaMemcpyDeviceToHost, st);
    if (e != cudaSuccess) return cuda_error(e, "invariants copy");
    e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_error(e, "invariants synchronise");

    const double h = p->h, hd = std::pow(h, (double)p->dim);
    if (mass) *mass = hd * r[0];
    if (energy) *energy = hd * r[1];
    if (dt_max) *dt_max = nlse::dt_bound(p->dim, h, p->a, r[2], r[3], r[4]);
    if (r[5] != 0.0 || !std::isfinite(r[0]))
        return nlse::report_error(NLSE_ENONFINITE, "state holds non-finite values");
    return NLSE_OK;
}
