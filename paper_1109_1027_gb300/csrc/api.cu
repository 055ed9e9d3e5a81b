// api.cu -- the C ABI of libnlse (include/nlse.h): parameter validation,
// context and work-space ownership, the RK4 stage schedule, CUDA-graph replay
// of the time loop and the host side of the invariants.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <vector>
#include <algorithm>
#include <new>
#include <string>

#include <nvtx3/nvToolsExt.h>

#include "nlse.h"
#include "nlse_internal.h"
#include "stability.cuh"

using nlse::StageLaunch;

namespace {

thread_local char g_err[512] = "";

int fail(int code, const char* fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof g_err, fmt, ap);
    va_end(ap);
    return code;
}

int cuda_fail(cudaError_t e, const char* what) {
    return fail(e == cudaErrorMemoryAllocation ? NLSE_ENOMEM : NLSE_ECUDA, "%s: %s", what,
                cudaGetErrorString(e));
}

// NVTX range over the rest of the enclosing scope (seen by profilers; a
// no-op without one).
struct Range {
    explicit Range(const char* name) { nvtxRangePushA(name); }
    ~Range() { nvtxRangePop(); }
    Range(const Range&) = delete;
    Range& operator=(const Range&) = delete;
};

#define NLSE_CUDA(call, what)                                  \
    do {                                                       \
        cudaError_t e_ = (call);                               \
        if (e_ != cudaSuccess) return cuda_fail(e_, what);     \
    } while (0)

// nlse_run replays CUDA graphs of 2^j RK4 steps, j = 0 .. kGraphLevels - 1,
// captured on first use for the state pointer: n steps are n / 32 replays of
// the 32-step graph and one replay of each graph whose bit is set in n % 32.
constexpr int kGraphLevels = 6;
constexpr int64_t kGraphSteps = (int64_t)1 << (kGraphLevels - 1);
constexpr int kNoInstance = 0x7f7f7f7f;       // StatusBlock::inst when no instance was refused

}  // namespace

struct nlse_ctx {
    nlse_params p;
    const void* V;
    int device;
    int64_t npts;
    size_t cbytes;            // bytes of one complex field
    void* Y[2];               // stage inputs (ping-pong)
    void* acc;                // accumulated RK4 increment
    void* lo;                 // FP32 compensated low part (FP32 only)
    void* plain[4];           // unfused schedule: D, K, Y, acc
    int* flag;                // status bits (the first member of status)
    nlse::StatusBlock* status;  // device status block (nlse_check reads and clears it)
    // nlse_run's entry check (check.cu): one entry per instance, its rows of
    // partial extremes and each instance's bound.
    nlse::CheckEntry* check_tab;
    int* check_row_entry;     // per row of partials, its entry
    int check_count, check_nrows;
    double* check_partials;
    double* check_bounds;
    double* partials;         // reduction scratch, nblocks x kPartialWidth
    int nblocks;
    double* epartials;        // 2D Dirichlet: rows of the tiled energy pass (etiles)
    int* emap;                // batch: per energy tile its instance
    int etiles;
    double* red_out;          // reduced values on the device
    double* host_out;         // pinned copy of red_out
    const void* state_psi;    // psi whose compensated part lo currently holds
    cudaGraphExec_t graphs[kGraphLevels];   // graphs[j]: 2^j steps on graph_psi
    const void* graph_psi;
    // Batched instances (nlse_create_batch): count > 0.
    int count;
    nlse::BatchPlan* batch;
    nlse_params* bparams;     // per-instance parameters
    int64_t* boff;            // per-instance element offsets
    int* brow;                // per-instance first row of partials (count + 1 entries)
    const void* maps_psi;     // Psi buffer the batch tensor maps currently point at
    // Adjoint work space (nlse_adjoint), allocated on first use, and the
    // forward pass it holds (nlse_adjoint_forward) for a reverse sweep.
    void* adj_buf;
    size_t adj_bytes;
    bool adj_ready;           // a forward pass awaits its reverse sweep
    int64_t adj_nsteps, adj_ckpt;
    // Device copy of a host state (nlse_run_host), allocated on first use.
    void* host_state;
    // Batch: per-instance table of the one-launch invariants (device).
    nlse::InvBatchEntry* inv_table;
    // Pipelined host runs of a batch (nlse_run_host): chunks of consecutive
    // instances whose copy in, steps and copy out overlap on three streams.
    int hp_chunks;
    std::vector<int> hp_first;          // first instance of each chunk (+ the count)
    std::vector<int> check_row0;        // entry check: first row of each entry (+ the total)
    cudaStream_t hp_stream[3];          // copy in, steps, copy out
    cudaEvent_t hp_start, hp_done;
    std::vector<cudaEvent_t> hp_ev;     // per chunk: copied in, stepped
    nlse::StatusBlock* hp_status;       // per chunk (device): a chunk's refusal stops that chunk only
    // Instances of a stack (NLSE_FLAG_STACK), else 1.
    int stack;
    // Tiling choices (nlse_set_tiling); 0 = the default.
    int tile_rows, tile_planes;
    int resident;             // 1D time loop: 0 default, -1 tiled kernels, else largest cluster
    int fuse2;                // 2D FP32: two stages per launch (NLSE_TILE_2D_FUSE)
    int adj_rows;             // adjoint: rows per CTA of the TMA walk; -1 the tile kernel; 0 default
};

namespace {

int validate(const nlse_params* p) {
    if (!p) return fail(NLSE_EINVAL, "params is NULL");
    if (p->dim < 1 || p->dim > 3) return fail(NLSE_EINVAL, "dim must be 1, 2 or 3 (got %d)", p->dim);
    for (int ax = 0; ax < p->dim; ++ax) {
        if (p->n[ax] < 3) return fail(NLSE_EINVAL, "n[%d] = %lld: need at least 3 points", ax, (long long)p->n[ax]);
        if (p->n[ax] > (int64_t)1 << 30) return fail(NLSE_EINVAL, "n[%d] too large", ax);
    }
    int64_t npts = 1;
    for (int ax = 0; ax < p->dim; ++ax) npts *= p->n[ax];
    if (p->flags & NLSE_FLAG_STACK) {
        if (p->dim != 2) return fail(NLSE_EINVAL, "NLSE_FLAG_STACK needs dim = 2");
        if (p->n[2] < 1 || p->n[2] > (1 << 20)) return fail(NLSE_EINVAL, "stack of %lld instances", (long long)p->n[2]);
        if (p->n[1] * p->n[2] > ((int64_t)1 << 30)) return fail(NLSE_EINVAL, "stack too tall");
        npts *= p->n[2];
    }
    if (npts > ((int64_t)1 << 34)) return fail(NLSE_EINVAL, "grid too large (%lld points)", (long long)npts);
    if (!(std::isfinite(p->h) && p->h > 0)) return fail(NLSE_EINVAL, "h must be positive and finite");
    if (!(std::isfinite(p->dt) && p->dt > 0)) return fail(NLSE_EINVAL, "dt must be positive and finite");
    if (!(std::isfinite(p->a) && p->a > 0)) return fail(NLSE_EINVAL, "a must be positive and finite (Eq. NLSE)");
    if (!std::isfinite(p->s)) return fail(NLSE_EINVAL, "s must be finite");
    if (p->bc < NLSE_BC_DIRICHLET || p->bc > NLSE_BC_LAPZERO) return fail(NLSE_EINVAL, "unknown bc %d", p->bc);
    if (p->prec != NLSE_FP32 && p->prec != NLSE_FP64) return fail(NLSE_EINVAL, "unknown prec %d", p->prec);
    if (p->lap != NLSE_LAP_2SHOC && p->lap != NLSE_LAP_CD && p->lap != NLSE_LAP_2SHOC_MS)
        return fail(NLSE_EINVAL, "unknown lap %d", p->lap);
    if (p->bc != NLSE_BC_DIRICHLET && p->lap == NLSE_LAP_2SHOC_MS && p->dim > 1)
        return fail(NLSE_EUNSUPPORTED, "the multi-storage 2SHOC is built for Dirichlet boundaries only");
    if ((p->flags & NLSE_FLAG_STACK) && (p->bc != NLSE_BC_DIRICHLET || (p->flags & NLSE_FLAG_PLAIN_SCHEDULE)))
        return fail(NLSE_EUNSUPPORTED, "stacks run Dirichlet boundaries on the fused schedule only");
    if ((p->flags & NLSE_FLAG_PLAIN_SCHEDULE) && p->lap == NLSE_LAP_2SHOC_MS && p->dim > 1)
        return fail(NLSE_EUNSUPPORTED, "the unfused schedule has the single-storage 2SHOC and CD only");
    return NLSE_OK;
}

StageLaunch base_launch(const nlse_ctx* c) {
    StageLaunch L;
    std::memset(&L, 0, sizeof L);
    L.dim = c->p.dim;
    for (int ax = 0; ax < 3; ++ax) L.n[ax] = ax < c->p.dim ? c->p.n[ax] : 1;
    if (c->stack > 1) {                          // a stack is one tall grid with a boundary every n[1] rows
        L.n[1] = c->p.n[1] * c->stack;
        L.rows1 = c->p.n[1];
    }
    L.prec = c->p.prec;
    L.lap = c->p.lap;
    L.bc = c->p.bc;
    L.h = c->p.h; L.a = c->p.a; L.s = c->p.s; L.dt = c->p.dt;
    L.V = c->V;
    L.flag = c->flag;
    L.tile_rows = c->tile_rows ? c->tile_rows : 16;
    L.tile_planes = c->tile_planes ? c->tile_planes : 32;
    L.keep_v = nlse::keep_v_in_l2((size_t)(c->npts / c->stack) * (c->p.prec == NLSE_FP32 ? 4 : 8)) ? 1 : 0;
    return L;
}

// Drops the captured time-loop graphs (their launches bake in the tiling and
// the state pointer).
void drop_graph(nlse_ctx* c) {
    for (auto& g : c->graphs) {
        if (g) cudaGraphExecDestroy(g);
        g = nullptr;
    }
    c->graph_psi = nullptr;
}

cudaError_t launch_stage(const StageLaunch& L, cudaStream_t st) {
    switch (L.dim) {
        case 1: return nlse::launch_stage_1d(L, st);
        case 2: return nlse::launch_stage_2d(L, st);
        default: return nlse::launch_stage_3d(L, st);
    }
}

// Whether the unfused kernels (plain.cu) run this context's steps: on
// request, or for MSD boundaries in 2D and 3D, which only they implement.
bool unfused(const nlse_params& p) {
    return (p.flags & NLSE_FLAG_PLAIN_SCHEDULE) || (p.bc == NLSE_BC_MSD && p.dim > 1) ||
           p.bc == NLSE_BC_PERIODIC || p.bc == NLSE_BC_LAPZERO;
}

nlse::PlainLaunch plain_launch(const nlse_ctx* c, const void* psi) {
    nlse::PlainLaunch L;
    L.dim = c->p.dim;
    for (int ax = 0; ax < 3; ++ax) L.n[ax] = ax < c->p.dim ? c->p.n[ax] : 1;
    L.prec = c->p.prec; L.lap = c->p.lap; L.bc = c->p.bc;
    L.h = c->p.h; L.a = c->p.a; L.s = c->p.s; L.dt = c->p.dt;
    L.psi = const_cast<void*>(psi); L.lo = c->lo; L.V = c->V;
    L.D = c->plain[0]; L.K = c->plain[1]; L.Y = c->plain[2]; L.acc = c->plain[3];
    L.flag = c->flag;
    return L;
}

// One step of the unfused schedule (plain.cu).
int enqueue_plain_step(nlse_ctx* c, void* psi, cudaStream_t st) {
    cudaError_t e = nlse::launch_plain_step(plain_launch(c, psi), st);
    if (e != cudaSuccess) return cuda_fail(e, "unfused RK4 step launch");
    return NLSE_OK;
}

// The four fused stages of one RK4 step (Eq. RK4) on psi, in place.
int enqueue_step(nlse_ctx* c, void* psi, cudaStream_t st) {
    if (unfused(c->p)) return enqueue_plain_step(c, psi, st);
    StageLaunch L = base_launch(c);
    L.psi = psi;
    L.psi_out = psi;
    L.acc = c->acc;
    L.lo = c->lo;
    const void* in[5] = {nullptr, psi, c->Y[0], c->Y[1], c->Y[0]};
    void* out[5] = {nullptr, c->Y[0], c->Y[1], c->Y[0], nullptr};
    static const char* const names[5] = {"", "RK4 stage 1", "RK4 stage 2", "RK4 stage 3", "RK4 stage 4"};
    for (int s = 1; s <= 4; ++s) {
        Range range(names[s]);
        L.stage = s;
        L.yin = in[s];
        L.yout = out[s];
        cudaError_t e = c->batch ? nlse::batch2d_launch(c->batch, L, st) : launch_stage(L, st);
        if (e != cudaSuccess) return cuda_fail(e, "RK4 stage launch");
    }
    return NLSE_OK;
}

// Whether this context's steps run as two stage pairs (NLSE_TILE_2D_FUSE).
// The caller's state must be 16-byte aligned, which the entry points check.
bool fused_steps(const nlse_ctx* c) {
    if (!c->fuse2 || c->batch || unfused(c->p)) return false;
    StageLaunch L = base_launch(c);
    L.psi = L.yin = c->Y[0];
    L.psi_out = c->Y[0];
    L.acc = c->acc;
    L.lo = c->lo;
    L.yout = c->Y[1];
    return nlse::rk4_2d_fused_eligible(L);
}

// One RK4 step as two stage pairs, Psi^n read from psi_in and Psi^{n+1}
// written to psi_out, another buffer: the second pair reads Psi^n on rows
// next to its block, which the neighbouring CTAs are overwriting meanwhile.
// Stages 1+2 write Y_2 into Y[1]; stages 3+4 read it.
int enqueue_fused_step(nlse_ctx* c, const void* psi_in, void* psi_out, cudaStream_t st) {
    StageLaunch L = base_launch(c);
    L.psi = psi_in;
    L.psi_out = psi_out;
    L.acc = c->acc;
    L.lo = c->lo;
    L.stage = 1;
    L.yin = psi_in;
    L.yout = c->Y[1];
    cudaError_t e = nlse::launch_rk4_2d_fused(L, 0, st);
    if (e == cudaSuccess) {
        L.stage = 3;
        L.yin = c->Y[1];
        L.yout = nullptr;
        e = nlse::launch_rk4_2d_fused(L, 1, st);
    }
    if (e != cudaSuccess) return cuda_fail(e, "fused RK4 stage-pair launch");
    return NLSE_OK;
}

// n RK4 steps on psi in place.  Fused steps alternate between psi and the
// context's Y[0] (free on that path).
int enqueue_steps(nlse_ctx* c, void* psi, int64_t n, cudaStream_t st) {
    if (!fused_steps(c)) {
        for (int64_t i = 0; i < n; ++i) {
            int rc = enqueue_step(c, psi, st);
            if (rc) return rc;
        }
        return NLSE_OK;
    }
    const int64_t nfused = n - n % 2;
    for (int64_t i = 0; i < nfused; ++i) {
        const bool even = i % 2 == 0;
        int rc = enqueue_fused_step(c, even ? psi : c->Y[0], even ? c->Y[0] : psi, st);
        if (rc) return rc;
    }
    // An odd count ends, with the state back in psi, on one step of four
    // single-stage launches in place (the same bits as a fused step).
    if (n % 2) return enqueue_step(c, psi, st);
    return NLSE_OK;
}

// Points the batch's tensor maps at psi (re-encoding and uploading the
// descriptor table on the stream) when they point elsewhere.
int bind_maps(nlse_ctx* c, const void* psi, cudaStream_t st) {
    if (!c->batch || c->maps_psi == psi) return NLSE_OK;
    cudaError_t e = nlse::batch2d_bind(c->batch, psi, st);
    if (e != cudaSuccess) {
        c->maps_psi = nullptr;
        return cuda_fail(e, "encoding the batch tensor maps");
    }
    c->maps_psi = psi;
    return NLSE_OK;
}

// Largest cluster for the resident 1D loop (0: tiled kernels; default 16,
// the fastest in both precisions for 1024 to 4096 points).
int resident_cluster(const nlse_ctx* c) {
    if (c->resident < 0) return 0;
    return c->resident > 0 ? c->resident : 16;
}

// Whether this context's steps run as one resident launch (small 1D grids).
bool resident_1d(const nlse_ctx* c) {
    return !c->batch && c->p.dim == 1 && resident_cluster(c) > 0 && !unfused(c->p) &&
           nlse::rk4_1d_resident_fits(c->p.n[0]);
}

int enqueue_resident(nlse_ctx* c, void* psi, int64_t nsteps, cudaStream_t st) {
    nlse::ResidentLaunch R;
    R.prec = c->p.prec; R.lap = c->p.lap; R.bc = c->p.bc;
    R.max_cluster = resident_cluster(c);
    R.n = c->p.n[0];
    R.h = c->p.h; R.a = c->p.a; R.s = c->p.s; R.dt = c->p.dt;
    R.psi = psi; R.lo = c->lo; R.V = c->V;
    R.nsteps = nsteps;
    R.flag = c->flag;
    cudaError_t e = nlse::launch_rk4_1d_resident(R, st);
    if (e != cudaSuccess) return cuda_fail(e, "1D resident RK4 launch");
    return NLSE_OK;
}

// Zeroes the compensated part when the state pointer changes.
int bind_state(nlse_ctx* c, const void* psi, cudaStream_t st) {
    int rc = bind_maps(c, psi, st);
    if (rc) return rc;
    if (c->state_psi == psi) return NLSE_OK;
    if (c->lo) NLSE_CUDA(cudaMemsetAsync(c->lo, 0, c->cbytes, st), "zeroing the compensated part");
    c->state_psi = psi;
    return NLSE_OK;
}

int invariants_batch_impl(nlse_ctx* c, const void* psi, double* mass, double* energy, double* dt_max,
                          cudaStream_t st);

int invariants_impl(nlse_ctx* c, const void* psi, double* mass, double* energy, double* dt_max,
                    cudaStream_t st) {
    if (c->batch) return fail(NLSE_EINVAL, "a batch context takes nlse_invariants_batch");
    nlse::InvLaunch L;
    L.dim = c->p.dim;
    for (int ax = 0; ax < 3; ++ax) L.n[ax] = ax < c->p.dim ? c->p.n[ax] : 1;
    if (c->stack > 1) {
        L.n[1] = c->p.n[1] * c->stack;
        L.rows1 = c->p.n[1];
    }
    L.prec = c->p.prec; L.lap = c->p.lap; L.bc = c->p.bc;
    L.h = c->p.h; L.a = c->p.a; L.s = c->p.s;
    L.psi = psi;
    L.lo = (c->lo && psi == c->state_psi) ? c->lo : nullptr;
    L.V = c->V;
    L.energy = energy != nullptr;
    L.epartials = c->epartials;
    NLSE_CUDA(nlse::launch_invariants(L, c->partials, c->nblocks, c->red_out, st), "invariants launch");
    NLSE_CUDA(cudaMemcpyAsync(c->host_out, c->red_out, sizeof(double) * nlse::kPartialWidth,
                              cudaMemcpyDeviceToHost, st), "invariants copy");
    NLSE_CUDA(cudaStreamSynchronize(st), "invariants synchronise");
    const double* r = c->host_out;
    const double h = c->p.h, hd = std::pow(h, (double)c->p.dim);
    if (mass) *mass = hd * r[0];
    if (energy) *energy = hd * r[1];
    if (dt_max) *dt_max = nlse::dt_bound(c->p.dim, h, c->p.a, r[2], r[3], r[4]);
    if (r[5] != 0.0 || !std::isfinite(r[0]))
        return fail(NLSE_ENONFINITE, "state holds %g non-finite values", r[5]);
    return NLSE_OK;
}

// Per-instance invariants of a batch: one launch over every instance's rows
// of partials, one launch reducing each instance's rows into its result row,
// one copy, one sync.
int invariants_batch_impl(nlse_ctx* c, const void* psi, double* mass, double* energy, double* dt_max,
                          cudaStream_t st) {
    nlse::InvBatchLaunch B;
    B.table = c->inv_table;
    B.count = c->count;
    B.nrows = c->nblocks;
    B.prec = c->p.prec; B.bc = c->p.bc; B.lap = c->p.lap;
    B.psi = psi;
    B.lo = (c->lo && psi == c->state_psi) ? c->lo : nullptr;
    B.V = c->V;
    B.energy = energy != nullptr;
    B.partials = c->partials;
    B.out = c->red_out;
    B.emap = c->emap;
    B.etiles = c->etiles;
    B.epartials = c->epartials;
    NLSE_CUDA(nlse::launch_invariants_batch(B, st), "invariants launch");
    NLSE_CUDA(cudaMemcpyAsync(c->host_out, c->red_out, sizeof(double) * nlse::kPartialWidth * c->count,
                              cudaMemcpyDeviceToHost, st), "invariants copy");
    NLSE_CUDA(cudaStreamSynchronize(st), "invariants synchronise");
    int bad = -1;
    for (int i = 0; i < c->count; ++i) {
        const double* r = c->host_out + (size_t)i * nlse::kPartialWidth;
        const nlse_params& q = c->bparams[i];
        const double h2 = q.h * q.h;
        if (mass) mass[i] = h2 * r[0];
        if (energy) energy[i] = h2 * r[1];
        if (dt_max) dt_max[i] = nlse::dt_bound(2, q.h, q.a, r[2], r[3], r[4]);
        if ((r[5] != 0.0 || !std::isfinite(r[0])) && bad < 0) bad = i;
    }
    if (bad >= 0) return fail(NLSE_ENONFINITE, "instance %d holds non-finite values", bad);
    return NLSE_OK;
}

// nlse_run's entry check, enqueued on the stream (no host synchronisation):
// the bound of Eq. (kdfull) of every instance against its dt; a refusal is
// left in the status block, where it stops the stage-4 kernels from writing
// the state and where nlse_check finds it.  MSD contexts need the boundary
// term B of Table t:bc2 and take the full invariants reduction; the other
// boundary rules have B = 0 and take the extremes pass of check.cu.
int enqueue_entry_check(nlse_ctx* c, const void* psi, cudaStream_t st) {
    Range range("entry check (Eq. kdfull)");
    const void* lo = (c->lo && psi == c->state_psi) ? c->lo : nullptr;
    if (c->p.bc == NLSE_BC_MSD) {
        nlse::InvLaunch L;
        L.dim = c->p.dim;
        for (int ax = 0; ax < 3; ++ax) L.n[ax] = ax < c->p.dim ? c->p.n[ax] : 1;
        L.prec = c->p.prec; L.lap = c->p.lap; L.bc = c->p.bc;
        L.h = c->p.h; L.a = c->p.a; L.s = c->p.s;
        L.psi = psi; L.lo = lo; L.V = c->V;
        L.energy = false;
        NLSE_CUDA(nlse::launch_invariants(L, c->partials, c->nblocks, c->red_out, st), "entry check launch");
        NLSE_CUDA(nlse::launch_invariants_gate(c->red_out, c->p.dim, c->p.h, c->p.a, c->p.dt, c->check_bounds,
                                               c->status, st), "entry check launch");
        return NLSE_OK;
    }
    nlse::CheckLaunch C;
    C.table = c->check_tab;
    C.row_entry = c->check_row_entry;
    C.count = c->check_count;
    C.nrows = c->check_nrows;
    C.prec = c->p.prec;
    C.psi = psi; C.lo = lo; C.V = c->V;
    C.partials = c->check_partials;
    C.bounds = c->check_bounds;
    C.status = c->status;
    NLSE_CUDA(nlse::launch_entry_check(C, st), "entry check launch");
    return NLSE_OK;
}

// Builds the entry check's per-instance table (one entry per instance of a
// batch or of a stack, one for a single grid) and its scratch.
int setup_entry_check(nlse_ctx* c) {
    const int count = c->count ? c->count : c->stack;
    std::vector<nlse::CheckEntry> tab(count);
    int rows = 0;
    for (int i = 0; i < count; ++i) {
        nlse::CheckEntry& e = tab[i];
        const nlse_params& q = c->count ? c->bparams[i] : c->p;
        int64_t npts = c->count ? q.n[0] * q.n[1] : c->npts / c->stack;
        e.psi_off = c->count ? c->boff[i] : (int64_t)i * npts;
        e.v_off = c->count ? c->boff[i] : 0;           // a stack's instances share V
        e.npts = npts;
        e.h = q.h; e.a = q.a; e.s = q.s; e.dt = q.dt;
        e.h2a = q.h * q.h / q.a;
        e.dim = q.dim;
        e.row0 = rows;
        rows += nlse::check_rows(npts);
        e.row1 = rows;
    }
    c->check_count = count;
    c->check_row0.resize(count + 1);
    for (int i = 0; i < count; ++i) c->check_row0[i] = tab[i].row0;
    c->check_row0[count] = rows;
    c->check_nrows = rows;
    NLSE_CUDA(cudaMalloc((void**)&c->check_tab, sizeof(nlse::CheckEntry) * count), "allocating the check table");
    NLSE_CUDA(cudaMemcpy(c->check_tab, tab.data(), sizeof(nlse::CheckEntry) * count, cudaMemcpyHostToDevice),
              "uploading the check table");
    NLSE_CUDA(cudaMalloc((void**)&c->check_partials, sizeof(double) * 3 * rows), "allocating check partials");
    std::vector<int> row_entry(rows);
    for (int i = 0; i < count; ++i)
        for (int r = tab[i].row0; r < tab[i].row1; ++r) row_entry[r] = i;
    NLSE_CUDA(cudaMalloc((void**)&c->check_row_entry, sizeof(int) * rows), "allocating the check row map");
    NLSE_CUDA(cudaMemcpy(c->check_row_entry, row_entry.data(), sizeof(int) * rows, cudaMemcpyHostToDevice),
              "uploading the check row map");
    NLSE_CUDA(cudaMalloc((void**)&c->check_bounds, sizeof(double) * count), "allocating check bounds");
    NLSE_CUDA(cudaMalloc((void**)&c->status, sizeof(nlse::StatusBlock)), "allocating the status block");
    c->flag = &c->status->bits;
    NLSE_CUDA(cudaMemset(&c->status->bits, 0, sizeof(int)), "zeroing the status");
    NLSE_CUDA(cudaMemset(&c->status->inst, 0x7f, 2 * sizeof(int)), "zeroing the status");
    return NLSE_OK;
}

// Status of the device block s (read by the caller after a synchronisation),
// cleared on the stream when it holds anything: NLSE_ETIMEOUT, then the entry
// check's refusals, then a non-finite value written by a step.
int report_status(nlse_ctx* c, const nlse::StatusBlock& s, cudaStream_t st) {
    if (!s.bits) return NLSE_OK;
    double bound = 0.0;
    if ((s.bits & nlse::kStatusUnstable) && s.inst >= 0 && s.inst < c->check_count)
        NLSE_CUDA(cudaMemcpyAsync(&bound, c->check_bounds + s.inst, sizeof(double), cudaMemcpyDeviceToHost, st),
                  "bound copy");
    NLSE_CUDA(cudaMemsetAsync(&c->status->bits, 0, sizeof(int), st), "status reset");
    NLSE_CUDA(cudaMemsetAsync(&c->status->inst, 0x7f, 2 * sizeof(int), st), "status reset");
    NLSE_CUDA(cudaStreamSynchronize(st), "status synchronise");
    if (s.bits & nlse::kStatusBounds)
        return fail(NLSE_EBOUNDS, "bounds-check build: an index outside its array at site %d (file %d, line %d); "
                    "the access was skipped", s.site, s.site / 100000, s.site % 100000);
    if (s.bits & nlse::kStatusTimeout)
        return fail(NLSE_ETIMEOUT, "a bounded device-side wait gave up (a data transfer never completed)");
    const int inst = s.inst == kNoInstance ? 0 : s.inst;
    const char* what = c->count ? "instance" : (c->stack > 1 ? "stacked instance" : "grid");
    if (s.bits & nlse::kStatusUnstable) {
        const double dt = c->count ? c->bparams[inst].dt : c->p.dt;
        return fail(NLSE_EUNSTABLE, "entry check of nlse_run (%s %d): dt = %.17g exceeds the bound %.17g of Eq. (kdfull); "
                    "the steps were not taken", what, inst, dt, bound);
    }
    if (s.bits & nlse::kStatusEntryNonFinite)
        return fail(NLSE_ENONFINITE, "entry check of nlse_run (%s %d): the state holds non-finite values; the steps "
                    "were not taken", what, inst);
    return fail(NLSE_ENONFINITE, "a non-finite value appeared in the state");
}

// Sets up the pipelined host run of a batch: up to 16 chunks of consecutive
// instances of about equal points, their work lists, streams, events and
// per-chunk status blocks.
int setup_host_pipe(nlse_ctx* c) {
    const int n = std::min(16, c->count);
    std::vector<int> first(1, 0);
    // Chunk targets: the first and the last chunk a quarter of the others, so
    // that the pipeline fills and drains sooner.
    std::vector<double> cum(n + 1, 0.0);
    for (int k = 0; k < n; ++k) cum[k + 1] = cum[k] + ((k == 0 || k == n - 1) && n > 2 ? 0.25 : 1.0);
    int64_t done = 0;
    for (int i = 0; i < c->count; ++i) {
        done += c->bparams[i].n[0] * c->bparams[i].n[1];
        const int k = (int)first.size();
        if (k < n && (double)done >= cum[k] / cum[n] * (double)c->npts && i + 1 < c->count) first.push_back(i + 1);
    }
    first.push_back(c->count);
    const int nch = (int)first.size() - 1;
    NLSE_CUDA(nlse::batch2d_set_chunks(c->batch, first), "building the chunk work lists");
    for (cudaStream_t& sp : c->hp_stream) NLSE_CUDA(cudaStreamCreateWithFlags(&sp, cudaStreamNonBlocking), "stream");
    NLSE_CUDA(cudaEventCreateWithFlags(&c->hp_start, cudaEventDisableTiming), "event");
    NLSE_CUDA(cudaEventCreateWithFlags(&c->hp_done, cudaEventDisableTiming), "event");
    c->hp_ev.assign(2 * nch, nullptr);
    for (cudaEvent_t& ev : c->hp_ev) NLSE_CUDA(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming), "event");
    NLSE_CUDA(cudaMalloc((void**)&c->hp_status, sizeof(nlse::StatusBlock) * nch), "allocating chunk status");
    c->hp_first = first;
    c->hp_chunks = nch;
    return NLSE_OK;
}

// The four fused stages of n RK4 steps on the instances of chunk k only,
// with that chunk's status word (its refusal stops only its stage 4).
int enqueue_chunk_steps(nlse_ctx* c, void* psi, int k, int64_t n, int* flag, cudaStream_t st) {
    StageLaunch L = base_launch(c);
    L.psi = psi;
    L.psi_out = psi;
    L.acc = c->acc;
    L.lo = c->lo;
    L.flag = flag;
    const void* in[5] = {nullptr, psi, c->Y[0], c->Y[1], c->Y[0]};
    void* out[5] = {nullptr, c->Y[0], c->Y[1], c->Y[0], nullptr};
    for (int64_t i = 0; i < n; ++i)
        for (int s = 1; s <= 4; ++s) {
            L.stage = s;
            L.yin = in[s];
            L.yout = out[s];
            cudaError_t e = nlse::batch2d_launch_chunk(c->batch, L, k, st);
            if (e != cudaSuccess) return cuda_fail(e, "RK4 stage launch");
        }
    return NLSE_OK;
}

// nlse_run_host of a batch: per chunk, the copy in (stream 0), the entry check
// and the steps (stream 1) and the copy out (stream 2), so that the copies of
// one chunk overlap the steps of its neighbours.  The caller's stream orders
// the whole and is synchronised at the end.
int run_host_pipelined(nlse_ctx* c, void* psi_host, int64_t nsteps, cudaStream_t st) {
    Range range("pipelined host run");
    if (!c->hp_chunks) {
        int rc = setup_host_pipe(c);
        if (rc) return rc;
    }
    int rc = bind_maps(c, c->host_state, st);
    if (rc) return rc;
    c->state_psi = c->host_state;                 // its compensated part is zeroed per chunk below
    const int nch = c->hp_chunks;
    const size_t eb = c->p.prec == NLSE_FP32 ? 8 : 16;
    cudaStream_t sin = c->hp_stream[0], scomp = c->hp_stream[1], sout = c->hp_stream[2];
    NLSE_CUDA(cudaMemsetAsync(c->hp_status, 0, sizeof(nlse::StatusBlock) * nch, st), "chunk status reset");
    NLSE_CUDA(cudaMemset2DAsync(&c->hp_status[0].inst, sizeof(nlse::StatusBlock), 0x7f, 2 * sizeof(int), nch, st),
              "chunk status reset");
    NLSE_CUDA(cudaEventRecord(c->hp_start, st), "event");
    for (cudaStream_t sp : c->hp_stream) NLSE_CUDA(cudaStreamWaitEvent(sp, c->hp_start, 0), "stream wait");
    char* dev = static_cast<char*>(c->host_state);
    char* host = static_cast<char*>(psi_host);
    for (int k = 0; k < nch; ++k) {
        const int64_t o0 = c->boff[c->hp_first[k]];
        const int64_t o1 = c->hp_first[k + 1] < c->count ? c->boff[c->hp_first[k + 1]] : c->npts;
        NLSE_CUDA(cudaMemcpyAsync(dev + o0 * eb, host + o0 * eb, (o1 - o0) * eb, cudaMemcpyHostToDevice, sin),
                  "state copy in");
        NLSE_CUDA(cudaEventRecord(c->hp_ev[2 * k], sin), "event");
    }
    for (int k = 0; k < nch; ++k) {
        const int i0 = c->hp_first[k], i1 = c->hp_first[k + 1];
        const int64_t o0 = c->boff[i0], o1 = i1 < c->count ? c->boff[i1] : c->npts;
        NLSE_CUDA(cudaStreamWaitEvent(scomp, c->hp_ev[2 * k], 0), "stream wait");
        if (c->lo)
            NLSE_CUDA(cudaMemsetAsync(static_cast<char*>(c->lo) + o0 * eb, 0, (o1 - o0) * eb, scomp),
                      "zeroing the compensated part");
        if (nsteps > 0 && !(c->p.flags & NLSE_FLAG_NO_STABILITY_CHECK)) {
            nlse::CheckLaunch C;
            C.table = c->check_tab;
            C.row_entry = c->check_row_entry;
            C.inst_base = i0;
            C.count = i1 - i0;
            C.row_base = c->check_row0[i0];
            C.nrows = c->check_row0[i1] - c->check_row0[i0];
            C.prec = c->p.prec;
            C.psi = c->host_state; C.lo = c->lo; C.V = c->V;
            C.partials = c->check_partials;
            C.bounds = c->check_bounds;
            C.status = &c->hp_status[k];
            NLSE_CUDA(nlse::launch_entry_check(C, scomp), "entry check launch");
        }
        if ((rc = enqueue_chunk_steps(c, c->host_state, k, nsteps, &c->hp_status[k].bits, scomp))) return rc;
        NLSE_CUDA(cudaEventRecord(c->hp_ev[2 * k + 1], scomp), "event");
    }
    for (int k = 0; k < nch; ++k) {
        const int64_t o0 = c->boff[c->hp_first[k]];
        const int64_t o1 = c->hp_first[k + 1] < c->count ? c->boff[c->hp_first[k + 1]] : c->npts;
        NLSE_CUDA(cudaStreamWaitEvent(sout, c->hp_ev[2 * k + 1], 0), "stream wait");
        NLSE_CUDA(cudaMemcpyAsync(host + o0 * eb, dev + o0 * eb, (o1 - o0) * eb, cudaMemcpyDeviceToHost, sout),
                  "state copy out");
    }
    NLSE_CUDA(cudaEventRecord(c->hp_done, sout), "event");
    NLSE_CUDA(cudaStreamWaitEvent(st, c->hp_done, 0), "stream wait");
    // The chunks' status blocks and the context's, merged.
    std::vector<nlse::StatusBlock> hs(nch + 1);
    NLSE_CUDA(cudaMemcpyAsync(hs.data(), c->hp_status, sizeof(nlse::StatusBlock) * nch, cudaMemcpyDeviceToHost, st),
              "status copy");
    NLSE_CUDA(cudaMemcpyAsync(&hs[nch], c->status, sizeof(nlse::StatusBlock), cudaMemcpyDeviceToHost, st),
              "status copy");
    NLSE_CUDA(cudaStreamSynchronize(st), "synchronise");
    nlse::StatusBlock m = hs[nch];
    for (int k = 0; k < nch; ++k) {
        m.bits |= hs[k].bits;
        m.inst = std::min(m.inst, hs[k].inst);
        m.site = std::min(m.site, hs[k].site);
    }
    return report_status(c, m, st);
}

// Captures n RK4 steps on psi (n = 2^j) into c->graphs[j].
int capture_steps(nlse_ctx* c, void* psi, int j) {
    cudaStream_t cs;
    NLSE_CUDA(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking), "capture stream");
    cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeRelaxed);
    if (e != cudaSuccess) {
        cudaStreamDestroy(cs);
        return cuda_fail(e, "begin capture");
    }
    int rc = enqueue_steps(c, psi, (int64_t)1 << j, cs);
    cudaGraph_t g = nullptr;
    e = cudaStreamEndCapture(cs, &g);
    cudaStreamDestroy(cs);
    if (rc) {
        if (g) cudaGraphDestroy(g);
        return rc;
    }
    if (e != cudaSuccess) return cuda_fail(e, "end capture");
    e = cudaGraphInstantiate(&c->graphs[j], g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) {
        c->graphs[j] = nullptr;
        return cuda_fail(e, "graph instantiate");
    }
    return NLSE_OK;
}

// n RK4 steps on psi as replays of the cached graphs (see kGraphLevels).
// Every level is captured together on the first run for a state pointer, so
// that no later step count pays for a capture.
int run_graphs(nlse_ctx* c, void* psi, int64_t n, cudaStream_t st) {
    if (c->graph_psi != psi || !c->graphs[0]) {
        drop_graph(c);
        for (int j = 0; j < kGraphLevels; ++j) {
            int rc = capture_steps(c, psi, j);
            if (rc) {
                drop_graph(c);
                return rc;
            }
        }
        c->graph_psi = psi;
    }
    for (int64_t i = 0; i < n / kGraphSteps; ++i)
        NLSE_CUDA(cudaGraphLaunch(c->graphs[kGraphLevels - 1], st), "graph launch");
    for (int j = kGraphLevels - 2; j >= 0; --j)
        if ((n >> j) & 1) NLSE_CUDA(cudaGraphLaunch(c->graphs[j], st), "graph launch");
    return NLSE_OK;
}

void release(nlse_ctx* c) {
    if (!c) return;
    for (cudaStream_t& sp : c->hp_stream)
        if (sp) cudaStreamDestroy(sp);
    for (cudaEvent_t ev : c->hp_ev)
        if (ev) cudaEventDestroy(ev);
    if (c->hp_start) cudaEventDestroy(c->hp_start);
    if (c->hp_done) cudaEventDestroy(c->hp_done);
    cudaFree(c->hp_status);
    cudaFree(c->adj_buf);
    cudaFree(c->host_state);
    cudaFree(c->inv_table);
    for (auto& g : c->graphs)
        if (g) cudaGraphExecDestroy(g);
    cudaFree(c->check_tab);
    cudaFree(c->check_row_entry);
    cudaFree(c->check_partials);
    cudaFree(c->check_bounds);
    nlse::batch2d_destroy(c->batch);
    delete[] c->bparams;
    delete[] c->boff;
    delete[] c->brow;
    cudaFree(c->Y[0]);
    cudaFree(c->Y[1]);
    cudaFree(c->acc);
    cudaFree(c->lo);
    for (int i = 0; i < 4; ++i) cudaFree(c->plain[i]);
    cudaFree(c->status);
    cudaFree(c->partials);
    cudaFree(c->epartials);
    cudaFree(c->emap);
    cudaFree(c->red_out);
    cudaFreeHost(c->host_out);
    delete c;
}

}  // namespace

namespace nlse {
int report_error(int code, const char* msg) { return fail(code, "%s", msg); }
}  // namespace nlse

extern "C" {

const char* nlse_last_error(void) { return g_err; }

int nlse_create(const nlse_params* p, const void* V_dev, nlse_ctx** out) {
    g_err[0] = 0;
    if (!out) return fail(NLSE_EINVAL, "out is NULL");
    *out = nullptr;
    int rc = validate(p);
    if (rc) return rc;
    if (!V_dev) return fail(NLSE_EINVAL, "V_dev is NULL");
    if ((uintptr_t)V_dev % 16) return fail(NLSE_EINVAL, "V_dev must be 16-byte aligned");

    nlse_ctx* c = new (std::nothrow) nlse_ctx();
    if (!c) return fail(NLSE_ENOMEM, "host allocation failed");
    c->p = *p;
    c->V = V_dev;
    c->stack = (p->flags & NLSE_FLAG_STACK) ? (int)p->n[2] : 1;
    c->npts = c->stack;
    for (int ax = 0; ax < p->dim; ++ax) c->npts *= p->n[ax];
    c->cbytes = (size_t)c->npts * (p->prec == NLSE_FP32 ? 8 : 16);

    cudaError_t e;
    int nsm = 0;
#define TRY(call, what) do { e = (call); if (e != cudaSuccess) { rc = cuda_fail(e, what); release(c); return rc; } } while (0)
    TRY(cudaGetDevice(&c->device), "cudaGetDevice");
    TRY(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, c->device), "device query");
    if (unfused(*p)) {
        for (int i = 0; i < 4; ++i) TRY(cudaMalloc(&c->plain[i], c->cbytes), "allocating RK4 work array");
    } else {
        TRY(cudaMalloc(&c->Y[0], c->cbytes), "allocating stage buffer");
        TRY(cudaMalloc(&c->Y[1], c->cbytes), "allocating stage buffer");
        TRY(cudaMalloc(&c->acc, c->cbytes), "allocating accumulator");
    }
    if (p->prec == NLSE_FP32 && !(p->flags & NLSE_FLAG_PLAIN_SCHEDULE)) {
        TRY(cudaMalloc(&c->lo, c->cbytes), "allocating compensated part");
        TRY(cudaMemset(c->lo, 0, c->cbytes), "zeroing compensated part");
    }
    {
        nlse::InvLaunch L;
        L.dim = p->dim;
        for (int ax = 0; ax < 3; ++ax) L.n[ax] = ax < p->dim ? p->n[ax] : 1;
        c->nblocks = nlse::inv_num_blocks(L, nsm);
    }
    TRY(cudaMalloc((void**)&c->partials, sizeof(double) * nlse::kPartialWidth * c->nblocks), "allocating partials");
    if ((p->dim == 2 || p->dim == 3) && p->bc == NLSE_BC_DIRICHLET) {
        c->etiles = p->dim == 2 ? nlse::energy2d_tiles(p->n[0], p->n[1] * c->stack)
                                : nlse::energy3d_tiles(p->n[0], p->n[1], p->n[2]);
        TRY(cudaMalloc((void**)&c->epartials, sizeof(double) * c->etiles), "allocating energy partials");
    }
    TRY(cudaMalloc((void**)&c->red_out, sizeof(double) * nlse::kPartialWidth), "allocating result");
    TRY(cudaMallocHost((void**)&c->host_out, sizeof(double) * nlse::kPartialWidth), "allocating pinned result");
#undef TRY
    if ((rc = setup_entry_check(c))) {
        release(c);
        return rc;
    }
    *out = c;
    return NLSE_OK;
}

void nlse_destroy(nlse_ctx* c) {
    if (!c) return;
    cudaDeviceSynchronize();
    release(c);
}

int nlse_create_batch(int count, const nlse_params* p, const void* V_dev, nlse_ctx** out) {
    g_err[0] = 0;
    if (!out) return fail(NLSE_EINVAL, "out is NULL");
    *out = nullptr;
    if (count < 1 || !p) return fail(NLSE_EINVAL, "need count >= 1 and a params array");
    if (!V_dev || (uintptr_t)V_dev % 16) return fail(NLSE_EINVAL, "V_dev must be a 16-byte aligned device pointer");
    int64_t total = 0;
    for (int i = 0; i < count; ++i) {
        int rc = validate(&p[i]);
        if (rc) return fail(rc, "instance %d: %s", i, std::string(g_err).c_str());
        if (p[i].prec != p[0].prec || p[i].lap != p[0].lap || p[i].bc != p[0].bc || p[i].flags != p[0].flags)
            return fail(NLSE_EINVAL, "instance %d: prec, lap, bc and flags must match instance 0", i);
        if (p[i].flags & (NLSE_FLAG_PLAIN_SCHEDULE | NLSE_FLAG_STACK))
            return fail(NLSE_EUNSUPPORTED, "batches run the fused schedule on unstacked grids only");
        if (!nlse::batch2d_instance_ok(p[i]))
            return fail(NLSE_EUNSUPPORTED, "instance %d: batches need 2D Dirichlet grids with n[0] a multiple of "
                        "%d", i, p[0].prec == NLSE_FP32 ? 4 : 2);
        total += p[i].n[0] * p[i].n[1];
    }
    nlse_ctx* c = new (std::nothrow) nlse_ctx();
    if (!c) return fail(NLSE_ENOMEM, "host allocation failed");
    c->p = p[0];
    c->V = V_dev;
    c->stack = 1;
    c->count = count;
    c->npts = total;
    c->cbytes = (size_t)total * (p[0].prec == NLSE_FP32 ? 8 : 16);
    c->bparams = new (std::nothrow) nlse_params[count];
    c->boff = new (std::nothrow) int64_t[count];
    c->brow = new (std::nothrow) int[count + 1];
    if (!c->bparams || !c->boff || !c->brow) { release(c); return fail(NLSE_ENOMEM, "host allocation failed"); }
    cudaError_t e;
    int rc, nsm = 0;
#define TRY(call, what) do { e = (call); if (e != cudaSuccess) { rc = cuda_fail(e, what); release(c); return rc; } } while (0)
    TRY(cudaGetDevice(&c->device), "cudaGetDevice");
    TRY(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, c->device), "device query");
    int64_t off = 0;
    c->brow[0] = 0;
    for (int i = 0; i < count; ++i) {
        c->bparams[i] = p[i];
        c->boff[i] = off;
        off += p[i].n[0] * p[i].n[1];
        nlse::InvLaunch L;
        L.dim = 2; L.n[0] = p[i].n[0]; L.n[1] = p[i].n[1]; L.n[2] = 1;
        c->brow[i + 1] = c->brow[i] + nlse::inv_num_blocks(L, nsm);
    }
    TRY(cudaMalloc(&c->Y[0], c->cbytes), "allocating stage buffer");
    TRY(cudaMalloc(&c->Y[1], c->cbytes), "allocating stage buffer");
    TRY(cudaMalloc(&c->acc, c->cbytes), "allocating accumulator");
    if (p[0].prec == NLSE_FP32) {
        TRY(cudaMalloc(&c->lo, c->cbytes), "allocating compensated part");
        TRY(cudaMemset(c->lo, 0, c->cbytes), "zeroing compensated part");
    }
    c->nblocks = c->brow[count];
    TRY(cudaMalloc((void**)&c->partials, sizeof(double) * nlse::kPartialWidth * c->nblocks), "allocating partials");
    TRY(cudaMalloc((void**)&c->red_out, sizeof(double) * nlse::kPartialWidth * count), "allocating results");
    TRY(cudaMallocHost((void**)&c->host_out, sizeof(double) * nlse::kPartialWidth * count),
        "allocating pinned results");
    {
        std::vector<nlse::InvBatchEntry> tab(count);
        std::vector<int> emap;
        for (int i = 0; i < count; ++i) {
            tab[i].off = c->boff[i];
            tab[i].nx = (int)p[i].n[0];
            tab[i].ny = (int)p[i].n[1];
            tab[i].h = p[i].h; tab[i].a = p[i].a; tab[i].s = p[i].s;
            tab[i].row0 = c->brow[i];
            tab[i].row1 = c->brow[i + 1];
            tab[i].erow0 = (int)emap.size();
            if (p[0].bc == NLSE_BC_DIRICHLET) emap.resize(emap.size() + nlse::energy2d_tiles(p[i].n[0], p[i].n[1]), i);
            tab[i].erow1 = (int)emap.size();
        }
        if (!emap.empty()) {
            c->etiles = (int)emap.size();
            TRY(cudaMalloc((void**)&c->epartials, sizeof(double) * c->etiles), "allocating energy partials");
            TRY(cudaMalloc((void**)&c->emap, sizeof(int) * c->etiles), "allocating the energy tile map");
            TRY(cudaMemcpy(c->emap, emap.data(), sizeof(int) * c->etiles, cudaMemcpyHostToDevice),
                "uploading the energy tile map");
        }
        TRY(cudaMalloc((void**)&c->inv_table, sizeof(nlse::InvBatchEntry) * count), "allocating the instance table");
        TRY(cudaMemcpy(c->inv_table, tab.data(), sizeof(nlse::InvBatchEntry) * count, cudaMemcpyHostToDevice),
            "uploading the instance table");
    }
    TRY(nlse::batch2d_create(count, p, V_dev, c->Y[0], c->Y[1], c->acc, c->lo, &c->batch), "building the batch plan");
#undef TRY
    if ((rc = setup_entry_check(c))) {
        release(c);
        return rc;
    }
    *out = c;
    return NLSE_OK;
}

}  // extern "C"

namespace {

// Layout of the adjoint work space for nsteps steps with a checkpoint every
// ckpt steps: state S, checkpoints (state + compensated part), the four stage
// inputs (Psi_n, Y2, Y3, Y4) of every step of one segment, two cotangents,
// two adjoint states (the first holds dL/dPsi_T after the forward pass), the
// dL/dV contributions of reversed stages 4, 3, 2, in FP32 the double-float
// running dL/dV, for a stack the per-instance dL/dV, loss partials and the
// loss.
struct AdjLayout {
    int64_t nseg, seglen;
    int nb;
    size_t ck_bytes, need;
    char *S, *ck, *seg, *W, *WN, *LA, *LB, *G, *GA;
    double *part, *lossd, *gvs;
};

AdjLayout adj_layout(nlse_ctx* c, int64_t nsteps, int64_t ckpt_every) {
    AdjLayout A;
    const size_t cb = c->cbytes;
    A.nseg = (nsteps + ckpt_every - 1) / ckpt_every;
    A.seglen = nsteps < ckpt_every ? nsteps : ckpt_every;
    A.nb = nlse::loss_num_blocks(c->npts);
    A.ck_bytes = (size_t)A.nseg * cb * (c->lo ? 2 : 1);
    const size_t gv_bytes = c->stack > 1 ? sizeof(double) * (size_t)c->npts : 0;
    const size_t g_bytes = 3 * (cb / 2);          // three real arrays
    const size_t ga_bytes = c->p.prec == NLSE_FP32 ? 8 * (size_t)c->npts : 0;
    A.need = cb + A.ck_bytes + 4 * (size_t)A.seglen * cb + 4 * cb + g_bytes + ga_bytes + gv_bytes +
             sizeof(double) * (A.nb + 1);
    char* base = static_cast<char*>(c->adj_buf);
    A.S = base;
    A.ck = A.S + cb;
    A.seg = A.ck + A.ck_bytes;
    A.W = A.seg + 4 * (size_t)A.seglen * cb;
    A.WN = A.W + cb;
    A.LA = A.WN + cb;
    A.LB = A.LA + cb;
    A.G = A.LB + cb;
    // The running and per-instance dL/dV before the loss scalars, so that they
    // stay as aligned as the arrays before them (the TMA walk of the reversed
    // stages reads the running dL/dV by rows).
    A.GA = ga_bytes ? A.G + g_bytes : nullptr;
    A.gvs = c->stack > 1 ? reinterpret_cast<double*>(A.G + g_bytes + ga_bytes) : nullptr;
    A.part = reinterpret_cast<double*>(A.G + g_bytes + ga_bytes + gv_bytes);
    A.lossd = A.part + A.nb;
    return A;
}

int adjoint_check_args(nlse_ctx* c, int64_t nsteps, int64_t ckpt_every) {
    if (c->batch || c->p.dim != 2 || c->p.bc != NLSE_BC_DIRICHLET || (c->p.flags & NLSE_FLAG_PLAIN_SCHEDULE))
        return fail(NLSE_EUNSUPPORTED, "the adjoint is implemented for single 2D Dirichlet grids (fused schedule)");
    if (nsteps < 0 || ckpt_every < 1) return fail(NLSE_EINVAL, "need nsteps >= 0 and ckpt_every >= 1");
    return NLSE_OK;
}

// The forward pass with checkpoints, dL/dPsi_T = 2 (Psi_T - target) into LA
// and the loss on the device; no synchronisation.
int adjoint_forward(nlse_ctx* c, const void* psi0, const void* target, int64_t nsteps, int64_t ckpt_every,
                    cudaStream_t st) {
    c->adj_ready = false;
    AdjLayout A = adj_layout(c, nsteps, ckpt_every);
    if (A.need > c->adj_bytes) {
        cudaFree(c->adj_buf);
        c->adj_buf = nullptr;
        c->adj_bytes = 0;
        NLSE_CUDA(cudaMalloc(&c->adj_buf, A.need), "allocating adjoint work space");
        c->adj_bytes = A.need;
        A = adj_layout(c, nsteps, ckpt_every);
    }
    const size_t cb = c->cbytes;
    const bool has_lo = c->lo != nullptr;
    auto ckp = [&](int64_t i) { return A.ck + (size_t)i * cb * (has_lo ? 2 : 1); };
    // S is the state; the context's compensated part belongs to S for the
    // duration of the pass.
    NLSE_CUDA(cudaMemcpyAsync(A.S, psi0, cb, cudaMemcpyDeviceToDevice, st), "copying psi0");
    if (has_lo) NLSE_CUDA(cudaMemsetAsync(c->lo, 0, cb, st), "zeroing the compensated part");
    c->state_psi = nullptr;
    for (int64_t g = 0; g < A.nseg; ++g) {
        NLSE_CUDA(cudaMemcpyAsync(ckp(g), A.S, cb, cudaMemcpyDeviceToDevice, st), "checkpoint");
        if (has_lo) NLSE_CUDA(cudaMemcpyAsync(ckp(g) + cb, c->lo, cb, cudaMemcpyDeviceToDevice, st), "checkpoint");
        const int64_t steps = std::min<int64_t>(ckpt_every, nsteps - g * ckpt_every);
        int rc = enqueue_steps(c, A.S, steps, st);
        if (rc) return rc;
    }
    NLSE_CUDA(nlse::launch_loss(c->p.prec, A.S, target, A.LA, c->npts, A.part, A.nb, A.lossd, st), "loss launch");
    c->adj_nsteps = nsteps;
    c->adj_ckpt = ckpt_every;
    c->adj_ready = true;
    return NLSE_OK;
}

// The reverse sweep of the held forward pass, segment by segment from the
// last, with dL/dPsi_T scaled by dloss; no synchronisation.
int adjoint_backward(nlse_ctx* c, double dloss, void* dpsi0, void* dV, cudaStream_t st) {
    const int64_t nsteps = c->adj_nsteps, ckpt_every = c->adj_ckpt;
    AdjLayout A = adj_layout(c, nsteps, ckpt_every);
    c->adj_ready = false;                        // the sweep consumes dL/dPsi_T
    const size_t cb = c->cbytes;
    const bool has_lo = c->lo != nullptr;
    auto ckp = [&](int64_t i) { return A.ck + (size_t)i * cb * (has_lo ? 2 : 1); };
    auto yin = [&](int64_t m, int j) { return A.seg + ((size_t)m * 4 + (size_t)(j - 1)) * cb; };  // Y_j of step m
    double* gvs = c->stack > 1 ? A.gvs : static_cast<double*>(dV);
    const int64_t vpts = c->npts / c->stack;
    if (dloss != 1.0)
        NLSE_CUDA(nlse::launch_scale(c->p.prec, A.LA, dloss, c->npts, st), "scaling the loss cotangent");
    char* lamp = A.LA;
    char* lam = A.LB;
    StageLaunch F = base_launch(c);
    F.acc = c->acc;
    F.lo = c->lo;
    nlse::AdjLaunch J;
    J.prec = c->p.prec; J.lap = c->p.lap;
    J.nx = c->p.n[0]; J.ny = c->p.n[1] * c->stack;
    J.rows1 = c->p.n[1];
    J.h = c->p.h; J.a = c->p.a; J.s = c->p.s;
    J.V = c->V;
    // The running dL/dV: FP64 in place, or in FP32 the double-float work array
    // converted at the end.
    J.gV = A.GA ? static_cast<void*>(A.GA) : static_cast<void*>(gvs);
    J.flag = &c->status->bits;
    J.walk_rows = c->adj_rows < 0 ? 0 : (c->adj_rows ? c->adj_rows : 8);
    char* G[3] = {A.G, A.G + cb / 2, A.G + cb};   // contributions of reversed stages 4, 3, 2
    for (int i = 0; i < 3; ++i) J.g_in[i] = G[i];
    NLSE_CUDA(cudaMemsetAsync(J.gV, 0, sizeof(double) * c->npts, st), "zeroing dV");
    const double k = c->p.dt;
    for (int64_t g = A.nseg - 1; g >= 0; --g) {
        const int64_t steps = std::min<int64_t>(ckpt_every, nsteps - g * ckpt_every);
        // Recompute the segment from its checkpoint with the fused stage
        // kernels, keeping every stage input: stage j of step m reads
        // Y_j(m) and writes Y_{j+1}(m); stage 4 writes Psi_{m+1} = Y_1(m+1).
        // Same arithmetic, and so the same bits, as the forward pass.
        NLSE_CUDA(cudaMemcpyAsync(yin(0, 1), ckp(g), cb, cudaMemcpyDeviceToDevice, st), "restore");
        if (has_lo) NLSE_CUDA(cudaMemcpyAsync(c->lo, ckp(g) + cb, cb, cudaMemcpyDeviceToDevice, st), "restore");
        for (int64_t m = 0; m < steps; ++m) {
            for (int sg = 1; sg <= 4; ++sg) {
                if (sg == 4 && m + 1 == steps) break;     // the segment's last state is not needed
                F.stage = sg;
                F.psi = yin(m, 1);
                F.psi_out = sg == 4 ? yin(m + 1, 1) : nullptr;
                F.yin = yin(m, sg);
                F.yout = sg < 4 ? yin(m, sg + 1) : nullptr;
                cudaError_t e = launch_stage(F, st);
                if (e != cudaSuccess) return cuda_fail(e, "segment recompute");
            }
        }
        for (int64_t m = steps - 1; m >= 0; --m) {
            const void* Ys[5] = {nullptr, yin(m, 1), yin(m, 2), yin(m, 3), yin(m, 4)};
            // Stages 4 .. 1 reversed.
            const void* w[5] = {nullptr, A.W, A.WN, A.W, lamp};
            const double sw[5] = {0, 1, 1, 1, k / 6.0};
            void* wn[5] = {nullptr, nullptr, A.W, A.WN, A.W};
            const double cw[5] = {0, 0, k / 6.0, k / 3.0, k / 3.0};
            const double cy[5] = {0, 0, k / 2.0, k / 2.0, k};
            for (int j = 4; j >= 1; --j) {
                J.j = j;
                J.w = w[j]; J.scale_w = sw[j]; J.Y = Ys[j];
                J.lamp = lamp; J.lam = lam; J.w_next = wn[j];
                J.cw = cw[j]; J.cy = cy[j];
                J.g_out = j > 1 ? G[4 - j] : nullptr;
                cudaError_t e = nlse::launch_adjoint_stage_2d(J, st);
                if (e != cudaSuccess) return cuda_fail(e, "adjoint stage launch");
            }
            std::swap(lamp, lam);
        }
    }
    NLSE_CUDA(cudaMemcpyAsync(dpsi0, lamp, cb, cudaMemcpyDeviceToDevice, st), "gradient copy");
    if (A.GA) NLSE_CUDA(nlse::launch_gv_double(A.GA, gvs, c->npts, st), "dV to FP64");
    if (c->stack > 1)
        NLSE_CUDA(nlse::launch_stack_sum(gvs, c->stack, vpts, static_cast<double*>(dV), st), "summing dV over the stack");
    return NLSE_OK;
}

// Synchronises; reads the loss (when asked) and the status.  A refusal of an
// earlier nlse_run that nobody read kept the stage-4 kernels from stepping:
// then the forward pass did not run, and the refusal is returned; so is a
// bounded wait of the adjoint walk that gave up, or (bounds-check build) an
// index outside its array.
int adjoint_finish(nlse_ctx* c, double* loss, cudaStream_t st) {
    double h_loss = 0.0;
    nlse::StatusBlock* hs = reinterpret_cast<nlse::StatusBlock*>(c->host_out);
    if (loss) {
        AdjLayout A = adj_layout(c, c->adj_nsteps, c->adj_ckpt);
        NLSE_CUDA(cudaMemcpyAsync(&h_loss, A.lossd, sizeof(double), cudaMemcpyDeviceToHost, st), "loss copy");
    }
    NLSE_CUDA(cudaMemcpyAsync(hs, c->status, sizeof(nlse::StatusBlock), cudaMemcpyDeviceToHost, st), "status copy");
    NLSE_CUDA(cudaStreamSynchronize(st), "adjoint synchronise");
    c->state_psi = nullptr;          // the compensated part no longer belongs to any caller state
    const nlse::StatusBlock sb = *hs;
    if (sb.bits & (nlse::kStatusRefused | nlse::kStatusTimeout | nlse::kStatusBounds)) {
        c->adj_ready = false;
        return report_status(c, sb, st);
    }
    if (loss) *loss = h_loss;
    return NLSE_OK;
}

}  // namespace

extern "C" {

int nlse_adjoint(nlse_ctx* c, const void* psi0, const void* target, int64_t nsteps, int64_t ckpt_every,
                 void* dpsi0, void* dV, double* loss, void* stream) {
    g_err[0] = 0;
    Range range("nlse_adjoint");
    if (!c || !psi0 || !target || !dpsi0 || !dV) return fail(NLSE_EINVAL, "NULL argument");
    int rc = adjoint_check_args(c, nsteps, ckpt_every);
    if (rc) return rc;
    if (((uintptr_t)psi0 | (uintptr_t)target | (uintptr_t)dpsi0 | (uintptr_t)dV) % 16)
        return fail(NLSE_EINVAL, "pointers must be 16-byte aligned");
    cudaStream_t st = (cudaStream_t)stream;
    if ((rc = adjoint_forward(c, psi0, target, nsteps, ckpt_every, st))) return rc;
    if ((rc = adjoint_backward(c, 1.0, dpsi0, dV, st))) return rc;
    return adjoint_finish(c, loss, st);
}

int nlse_adjoint_forward(nlse_ctx* c, const void* psi0, const void* target, int64_t nsteps, int64_t ckpt_every,
                         double* loss, void* stream) {
    g_err[0] = 0;
    Range range("nlse_adjoint_forward");
    if (!c || !psi0 || !target) return fail(NLSE_EINVAL, "NULL argument");
    int rc = adjoint_check_args(c, nsteps, ckpt_every);
    if (rc) return rc;
    if (((uintptr_t)psi0 | (uintptr_t)target) % 16) return fail(NLSE_EINVAL, "pointers must be 16-byte aligned");
    cudaStream_t st = (cudaStream_t)stream;
    if ((rc = adjoint_forward(c, psi0, target, nsteps, ckpt_every, st))) return rc;
    return adjoint_finish(c, loss, st);
}

int nlse_adjoint_backward(nlse_ctx* c, double dloss, void* dpsi0, void* dV, void* stream) {
    g_err[0] = 0;
    Range range("nlse_adjoint_backward");
    if (!c || !dpsi0 || !dV) return fail(NLSE_EINVAL, "NULL argument");
    if (!c->adj_ready)
        return fail(NLSE_EINVAL, "no forward pass to reverse: call nlse_adjoint_forward first (each forward pass "
                    "admits one reverse sweep)");
    if (!std::isfinite(dloss)) return fail(NLSE_EINVAL, "dloss must be finite");
    if (((uintptr_t)dpsi0 | (uintptr_t)dV) % 16) return fail(NLSE_EINVAL, "pointers must be 16-byte aligned");
    cudaStream_t st = (cudaStream_t)stream;
    int rc = adjoint_backward(c, dloss, dpsi0, dV, st);
    if (rc) return rc;
    return adjoint_finish(c, nullptr, st);
}

int nlse_invariants_batch(nlse_ctx* c, const void* psi, double* mass, double* energy, double* dt_max,
                          void* stream) {
    g_err[0] = 0;
    if (!c || !psi) return fail(NLSE_EINVAL, "NULL argument");
    if (!c->batch) return fail(NLSE_EINVAL, "not a batch context: use nlse_invariants");
    return invariants_batch_impl(c, psi, mass, energy, dt_max, (cudaStream_t)stream);
}

int nlse_batch_count(const nlse_ctx* c) { return c ? c->count : 0; }

int nlse_set_tiling(nlse_ctx* c, int key, int value) {
    g_err[0] = 0;
    if (!c) return fail(NLSE_EINVAL, "NULL context");
    switch (key) {
        case NLSE_TILE_ROWS:
            if (value != 8 && value != 16 && value != 32) return fail(NLSE_EINVAL, "rows per CTA: 8, 16 or 32");
            c->tile_rows = value;
            break;
        case NLSE_TILE_PLANES:
            if (value != 32 && value != 64 && value != 128) return fail(NLSE_EINVAL, "planes per CTA: 32, 64 or 128");
            c->tile_planes = value;
            break;
        case NLSE_TILE_1D_RESIDENT:
            if (value < 0 || value > nlse::rk4_1d_max_cluster() || (value & (value - 1)))
                return fail(NLSE_EINVAL, "1D resident loop: 0 or a power of two up to %d", nlse::rk4_1d_max_cluster());
            c->resident = value ? value : -1;
            break;
        case NLSE_TILE_2D_FUSE:
            if (value != 0 && value != 1) return fail(NLSE_EINVAL, "two stages per launch: 0 or 1");
            c->fuse2 = value;
            break;
        case NLSE_TILE_ADJ_ROWS:
            if (value != 0 && value != 8 && value != 16 && value != 32)
                return fail(NLSE_EINVAL, "adjoint rows per CTA: 0, 8, 16 or 32");
            c->adj_rows = value ? value : -1;
            break;
        case NLSE_TILE_BATCH_NARROW: {
            if (!c->batch) return fail(NLSE_EINVAL, "not a batch context");
            if (value < 0) return fail(NLSE_EINVAL, "the narrow-tile width bound must be >= 0");
            cudaError_t e = nlse::batch2d_retile(c->batch, value);
            if (e != cudaSuccess) return cuda_fail(e, "rebuilding the batch tiles");
            c->maps_psi = nullptr;                       // re-encode the maps for the new box widths
            break;
        }
        default:
            return fail(NLSE_EINVAL, "unknown tiling key %d", key);
    }
    drop_graph(c);
    return NLSE_OK;
}

int nlse_get_tiling(const nlse_ctx* c, int key, int* value) {
    g_err[0] = 0;
    if (!c || !value) return fail(NLSE_EINVAL, "NULL argument");
    switch (key) {
        case NLSE_TILE_ROWS: *value = c->tile_rows ? c->tile_rows : 16; return NLSE_OK;
        case NLSE_TILE_PLANES: *value = c->tile_planes ? c->tile_planes : 32; return NLSE_OK;
        case NLSE_TILE_BATCH_NARROW:
            if (!c->batch) return fail(NLSE_EINVAL, "not a batch context");
            *value = nlse::batch2d_narrow(c->batch);
            return NLSE_OK;
        case NLSE_TILE_1D_RESIDENT: *value = resident_cluster(c); return NLSE_OK;
        case NLSE_TILE_2D_FUSE: *value = c->fuse2; return NLSE_OK;
        case NLSE_TILE_ADJ_ROWS: *value = c->adj_rows < 0 ? 0 : (c->adj_rows ? c->adj_rows : 8); return NLSE_OK;
    }
    return fail(NLSE_EINVAL, "unknown tiling key %d", key);
}

int nlse_lap2shoc(nlse_ctx* c, const void* psi, void* lap, void* stream) {
    g_err[0] = 0;
    Range range("nlse_lap2shoc");
    if (!c || !psi || !lap) return fail(NLSE_EINVAL, "NULL argument");
    if (((uintptr_t)psi | (uintptr_t)lap) % 16) return fail(NLSE_EINVAL, "pointers must be 16-byte aligned");
    const char *a0 = (const char*)psi, *b0 = (const char*)lap;
    if (a0 < b0 + c->cbytes && b0 < a0 + c->cbytes) return fail(NLSE_EINVAL, "psi and lap overlap");
    if (unfused(c->p) && c->p.bc != NLSE_BC_DIRICHLET) {
        cudaError_t e = nlse::launch_plain_laplacian(plain_launch(c, psi), lap, (cudaStream_t)stream);
        if (e != cudaSuccess) return cuda_fail(e, "Laplacian launch");
        return NLSE_OK;
    }
    StageLaunch L = base_launch(c);
    L.stage = 0;
    L.yin = psi;
    L.lap_out = lap;
    if (c->batch) {
        int rc = bind_maps(c, psi, (cudaStream_t)stream);
        if (rc) return rc;
    }
    cudaError_t e = c->batch ? nlse::batch2d_launch(c->batch, L, (cudaStream_t)stream)
                             : launch_stage(L, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "Laplacian launch");
    return NLSE_OK;
}

int nlse_rk4_step(nlse_ctx* c, void* psi, void* stream) {
    g_err[0] = 0;
    Range range("nlse_rk4_step");
    if (!c || !psi) return fail(NLSE_EINVAL, "NULL argument");
    if ((uintptr_t)psi % 16) return fail(NLSE_EINVAL, "psi must be 16-byte aligned");
    cudaStream_t st = (cudaStream_t)stream;
    int rc = bind_state(c, psi, st);
    if (rc) return rc;
    if (resident_1d(c)) return enqueue_resident(c, psi, 1, st);
    return enqueue_steps(c, psi, 1, st);
}

int nlse_run(nlse_ctx* c, void* psi, int64_t nsteps, void* stream) {
    g_err[0] = 0;
    Range range("nlse_run");
    if (!c || !psi) return fail(NLSE_EINVAL, "NULL argument");
    if (nsteps < 0) return fail(NLSE_EINVAL, "nsteps must be >= 0");
    if ((uintptr_t)psi % 16) return fail(NLSE_EINVAL, "psi must be 16-byte aligned");
    cudaStream_t st = (cudaStream_t)stream;
    int rc = bind_state(c, psi, st);
    if (rc) return rc;
    if (nsteps == 0) return NLSE_OK;
    if (!(c->p.flags & NLSE_FLAG_NO_STABILITY_CHECK) && (rc = enqueue_entry_check(c, psi, st))) return rc;
    if (resident_1d(c)) return enqueue_resident(c, psi, nsteps, st);
    // Inside a caller's stream capture the steps are enqueued as they are
    // (they become part of the caller's graph); otherwise cached graphs.
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    NLSE_CUDA(cudaStreamIsCapturing(st, &cap), "stream capture query");
    if (cap != cudaStreamCaptureStatusNone) return enqueue_steps(c, psi, nsteps, st);
    return run_graphs(c, psi, nsteps, st);
}

int nlse_run_host(nlse_ctx* c, void* psi_host, int64_t nsteps, void* stream) {
    g_err[0] = 0;
    Range range("nlse_run_host");
    if (!c || !psi_host) return fail(NLSE_EINVAL, "NULL argument");
    if (nsteps < 0) return fail(NLSE_EINVAL, "nsteps must be >= 0");
    cudaStream_t st = (cudaStream_t)stream;
    if (!c->host_state) NLSE_CUDA(cudaMalloc(&c->host_state, c->cbytes), "allocating the device state");
    if (c->batch && c->count > 1) return run_host_pipelined(c, psi_host, nsteps, st);
    NLSE_CUDA(cudaMemcpyAsync(c->host_state, psi_host, c->cbytes, cudaMemcpyHostToDevice, st), "state copy in");
    if (c->state_psi == c->host_state) c->state_psi = nullptr;    // a new state: no compensated part yet
    int rc = nlse_run(c, c->host_state, nsteps, stream);
    if (rc) return rc;
    nlse::StatusBlock* hs = reinterpret_cast<nlse::StatusBlock*>(c->host_out);
    NLSE_CUDA(cudaMemcpyAsync(hs, c->status, sizeof(nlse::StatusBlock), cudaMemcpyDeviceToHost, st), "status copy");
    NLSE_CUDA(cudaMemcpyAsync(psi_host, c->host_state, c->cbytes, cudaMemcpyDeviceToHost, st), "state copy out");
    NLSE_CUDA(cudaStreamSynchronize(st), "synchronise");
    const nlse::StatusBlock s = *hs;
    return report_status(c, s, st);
}

int nlse_invariants(nlse_ctx* c, const void* psi, double* mass, double* energy, double* dt_max,
                    void* stream) {
    g_err[0] = 0;
    Range range("nlse_invariants");
    if (!c || !psi) return fail(NLSE_EINVAL, "NULL argument");
    return invariants_impl(c, psi, mass, energy, dt_max, (cudaStream_t)stream);
}

int nlse_reset_compensation(nlse_ctx* c, void* stream) {
    g_err[0] = 0;
    if (!c) return fail(NLSE_EINVAL, "NULL argument");
    if (c->lo) NLSE_CUDA(cudaMemsetAsync(c->lo, 0, c->cbytes, (cudaStream_t)stream), "zeroing the compensated part");
    return NLSE_OK;
}

int nlse_selftest_timeout(nlse_ctx* c, double limit_ms, void* stream) {
    g_err[0] = 0;
    if (!c) return fail(NLSE_EINVAL, "NULL context");
    if (!(limit_ms > 0 && limit_ms <= 1000)) return fail(NLSE_EINVAL, "limit_ms must be in (0, 1000]");
    NLSE_CUDA(nlse::launch_bounded_wait_probe(c->flag, limit_ms, (cudaStream_t)stream), "probe launch");
    return NLSE_OK;
}

int nlse_check(nlse_ctx* c, void* stream) {
    g_err[0] = 0;
    Range range("nlse_check");
    if (!c) return fail(NLSE_EINVAL, "NULL argument");
    cudaStream_t st = (cudaStream_t)stream;
    nlse::StatusBlock* hs = reinterpret_cast<nlse::StatusBlock*>(c->host_out);
    NLSE_CUDA(cudaMemcpyAsync(hs, c->status, sizeof(nlse::StatusBlock), cudaMemcpyDeviceToHost, st), "status copy");
    NLSE_CUDA(cudaStreamSynchronize(st), "status synchronise");
    const nlse::StatusBlock s = *hs;
    return report_status(c, s, st);
}

}  // extern "C"
