// nlse_internal.h -- host-side interface between the C ABI (api.cu) and the
// per-dimension kernel files (stage1d.cu, stage2d.cu, stage3d.cu,
// invariants.cu).  No CUDA device code here.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "nlse.h"

namespace nlse {

// The context's status block.  bits collects what the device reports to
// nlse_check; the stage-4 kernels (the only ones that write the state) leave
// the state unchanged while a refusal bit of nlse_run's entry check is set.
constexpr int kStatusNonFinite = 1;        // an RK4 step wrote a NaN or Inf
constexpr int kStatusTimeout = 2;          // a bounded device-side wait gave up
constexpr int kStatusUnstable = 4;         // entry check: dt above the bound of Eq. (kdfull)
constexpr int kStatusEntryNonFinite = 8;   // entry check: the state held a NaN or Inf
constexpr int kStatusRefused = kStatusUnstable | kStatusEntryNonFinite;
constexpr int kStatusBounds = 16;          // bounds-check build: an index outside its array
struct StatusBlock {
    int bits;
    int inst;               // smallest instance the entry check refused (0x7f7f7f7f: none)
    int site;               // bounds-check build: smallest failing site, file * 100000 + line
                            // (0x7f7f7f7f: none)
    int pad;
};

// One launch of a fused RK4 stage (stage 1..4) or of the standalone
// Laplacian (stage 0).  Pointers are device pointers; their element types
// follow prec (complex64 / float or complex128 / double).
struct StageLaunch {
    int dim;
    int64_t n[3];
    int prec, lap, bc;
    double h, a, s, dt;
    int stage;              // 0: Laplacian only; 1..4: RK4 stage of Eq. (RK4)
    const void* yin;        // stage input Psi_s (read with a 2-point halo)
    const void* psi;        // Psi^n (stages 2..4)
    void* psi_out;          // stage 4: Psi^{n+1} (may equal psi)
    void* lo;               // FP32 compensated low part (stage 4), else nullptr
    void* acc;              // accumulated RK4 increment
    void* yout;             // next stage input
    void* lap_out;          // stage 0 output
    const void* V;
    int* flag;              // status bits of the context's StatusBlock (kStatus*)
    int tile_rows;          // 2D TMA kernel: rows per CTA (8, 16, 32)
    int tile_planes;        // 3D TMA kernel: z planes per CTA (32, 64, 128)
    int keep_v;             // TMA kernels: load V with an L2 evict-last hint (V small enough
                            // to stay in L2 across the four stages of a step)
    int64_t rows1;          // 2D: rows of one instance of a stack (n[1] when not stacked);
                            // instance i holds rows i*rows1 .. (i+1)*rows1-1, all share V
};

// Whether V of the given size should be kept resident in L2 (a quarter of it).
bool keep_v_in_l2(size_t v_bytes);

cudaError_t launch_stage_1d(const StageLaunch& L, cudaStream_t st);
cudaError_t launch_stage_2d(const StageLaunch& L, cudaStream_t st);
// The TMA-fed y-streaming 2D kernel (stage2d_tma.cuh) and when it applies;
// one entry per compiled rows-per-CTA variant.
bool stage_2d_tma_eligible(const StageLaunch& L);
// Temporal blocking (stage2d_fused.cu): two RK4 stages per launch, pair 0 =
// stages 1+2 (yin unused: reads psi; writes acc and yout = Y_2), pair 1 =
// stages 3+4 (reads yin = Y_2, psi, acc, lo; writes psi_out and lo).  FP32 2D
// Dirichlet grids on the TMA path, 2SHOC or CD; the same bits as the
// single-stage launches.
bool rk4_2d_fused_eligible(const StageLaunch& L);
cudaError_t launch_rk4_2d_fused(const StageLaunch& L, int pair, cudaStream_t st);
cudaError_t launch_stage_2d_tma(const StageLaunch& L, cudaStream_t st);
cudaError_t launch_stage_2d_tma_rows8(const StageLaunch& L, cudaStream_t st);
cudaError_t launch_stage_2d_tma_rows16(const StageLaunch& L, cudaStream_t st);
cudaError_t launch_stage_2d_tma_rows32(const StageLaunch& L, cudaStream_t st);
cudaError_t launch_stage_3d(const StageLaunch& L, cudaStream_t st);
// The TMA-fed z-streaming FP32 3D kernel (stage3d_tma.cuh) and when it
// applies; one entry per compiled planes-per-CTA variant.
bool stage_3d_tma_eligible(const StageLaunch& L);
cudaError_t launch_stage_3d_tma(const StageLaunch& L, cudaStream_t st);
cudaError_t launch_stage_3d_tma_planes32(const StageLaunch& L, cudaStream_t st);
cudaError_t launch_stage_3d_tma_planes64(const StageLaunch& L, cudaStream_t st);
cudaError_t launch_stage_3d_tma_planes128(const StageLaunch& L, cudaStream_t st);

// One unfused RK4 step (plain.cu): the step-1 field D, the stage slope K,
// the stage input Y and the increment acc are full device arrays.
struct PlainLaunch {
    int dim;
    int64_t n[3];
    int prec, lap, bc;
    double h, a, s, dt;
    void* psi;
    void* lo;               // FP32 compensated part, or nullptr
    const void* V;
    void *D, *K, *Y, *acc;
    int* flag;
};

cudaError_t launch_plain_step(const PlainLaunch& L, cudaStream_t st);
// The Laplacian (boundary points: D_b) through the same unfused kernels.
cudaError_t launch_plain_laplacian(const PlainLaunch& L, void* lap_out, cudaStream_t st);

// Whole RK4 time loops of a small 1D grid in one thread-block cluster
// (rk4_1d_resident.cu).
struct ResidentLaunch {
    int prec, lap, bc;
    int max_cluster;        // largest number of CTAs to spread the grid over (1..16)
    int64_t n;
    double h, a, s, dt;
    void* psi;              // state, in place
    void* lo;               // FP32 compensated part, or nullptr
    const void* V;
    int64_t nsteps;
    int* flag;
};
bool rk4_1d_resident_fits(int64_t n);
int rk4_1d_max_cluster();
cudaError_t launch_rk4_1d_resident(const ResidentLaunch& L, cudaStream_t st);

// Batched uneven 2D instances (batch2d.cu).  The plan owns the per-instance
// tensor-map descriptors and the tile work lists.
struct BatchPlan;
bool batch2d_instance_ok(const nlse_params& p);
cudaError_t batch2d_create(int count, const nlse_params* p, const void* V, void* Y0, void* Y1, void* acc,
                           void* lo, BatchPlan** out);
cudaError_t batch2d_bind(BatchPlan* b, const void* psi, cudaStream_t st);
cudaError_t batch2d_retile(BatchPlan* b, int narrow);   // synchronises the device
int batch2d_narrow(const BatchPlan* b);
cudaError_t batch2d_launch(BatchPlan* b, const StageLaunch& L, cudaStream_t st);
// Chunks of consecutive instances for a pipelined host run: first[k] is the
// first instance of chunk k, first.back() the instance count.  Their work
// lists follow the tile groups (rebuilt with them).
cudaError_t batch2d_set_chunks(BatchPlan* b, const std::vector<int>& first);
int batch2d_chunks(const BatchPlan* b);
// One RK4 stage (or the Laplacian) of chunk k's instances only.
cudaError_t batch2d_launch_chunk(BatchPlan* b, const StageLaunch& L, int k, cudaStream_t st);
void batch2d_destroy(BatchPlan* b);

// Adjoint of one RK4 stage on a 2D grid (adjoint2d.cu).
struct AdjLaunch {
    int prec, lap, j;       // j = 4, 3, 2, 1: the stage being reversed
    int64_t nx, ny;
    double h, a, s;
    const void* w;          // cotangent of K_j (times scale_w)
    double scale_w;
    const void* Y;          // stage input Y_j
    const void* V;
    const void* lamp;       // dL/dPsi_{n+1}
    void* lam;              // dL/dPsi_n being accumulated
    void* w_next;           // cotangent of K_{j-1} = cw lam' + cy Ybar_j
    void* g_out;            // stages 4..2: this stage's dL/dV contribution (R), one per point
    const void* g_in[3];    // stage 1: the contributions of stages 4, 3, 2
    void* gV;               // stage 1: the running dL/dV, 8 bytes a point: FP64, or in FP32 runs a
                            // double-float (float hi, lo) that launch_gv_double converts
    double cw, cy;
    int64_t rows1;          // rows per stacked instance (ny when not stacked); V has rows1 rows
    int* flag;              // status bits (the TMA walk's timeout bit)
    int walk_rows;          // 8, 16, 32: the TMA row walk with that many rows per CTA; 0: the tile kernel
};
cudaError_t launch_adjoint_stage_2d(const AdjLaunch& L, cudaStream_t st);
// out[p] = hi + lo in FP64 for the n double-float pairs at acc.
cudaError_t launch_gv_double(const void* acc, double* out, int64_t n, cudaStream_t st);
// Whether the TMA row walk can run the stage (16-byte aligned rows and arrays).
bool adjoint_2d_tma_eligible(const AdjLaunch& L);
cudaError_t launch_adjoint_2d_tma_rows8(const AdjLaunch& L, cudaStream_t st);
cudaError_t launch_adjoint_2d_tma_rows16(const AdjLaunch& L, cudaStream_t st);
cudaError_t launch_adjoint_2d_tma_rows32(const AdjLaunch& L, cudaStream_t st);
// dst[q] = sum over i of src[i n + q], i = 0 .. count-1 in order (stacked dL/dV).
cudaError_t launch_stack_sum(const double* src, int count, int64_t n, double* dst, cudaStream_t st);
// z *= f over n complex values (the cotangent of the loss, nlse_adjoint_backward).
cudaError_t launch_scale(int prec, void* z, double f, int64_t n, cudaStream_t st);
int loss_num_blocks(int64_t n);
cudaError_t launch_loss(int prec, const void* psi, const void* target, void* lam, int64_t n, double* partials,
                        int nblocks, double* out, cudaStream_t st);

// FP64 reductions for nlse_invariants.  Each of the nblocks blocks of the
// partial kernel writes kPartialWidth doubles to partials; the final kernel
// reduces them in a fixed order into out[0..kPartialWidth).
constexpr int kPartialWidth = 6;   // mass, energy, min L, max L, max |B|, non-finite count
constexpr int kInvThreads = 256;

struct InvLaunch {
    int dim;
    int64_t n[3];
    int prec, lap, bc;
    double h, a, s;
    const void* psi;        // state (hi part in FP32)
    const void* lo;         // FP32 compensated part or nullptr
    const void* V;
    bool energy = true;     // false: skip the energy sum (mass, extremes and count only)
    int64_t rows1 = 0;      // 2D stack: rows per instance (0: not stacked)
    double* epartials = nullptr;   // 2D / 3D Dirichlet: rows for the tiled energy pass
};

int inv_num_blocks(const InvLaunch& L, int num_sms);
// Tiles (blocks) of the tiled energy pass over an nx x ny grid / an nx x ny x nz grid.
int energy2d_tiles(int64_t nx, int64_t ny);
int energy3d_tiles(int64_t nx, int64_t ny, int64_t nz);

// Invariants of every instance of a batch in one launch (plus one for the
// per-instance reduction), with the partial rows a launch per instance gives.
struct InvBatchEntry {
    int64_t off;            // first element of the instance in the flat buffers
    int nx, ny;
    double h, a, s;
    int row0, row1;         // its rows of partials
    int erow0, erow1;       // its tiles of the tiled energy pass
};
struct InvBatchLaunch {
    const InvBatchEntry* table;   // device, count entries, row0 ascending
    int count, nrows;
    int prec, bc, lap;
    const void* psi;
    const void* lo;         // FP32 compensated part or nullptr
    const void* V;
    bool energy;
    double* partials;       // nrows x kPartialWidth
    double* out;            // count x kPartialWidth
    const int* emap = nullptr;     // Dirichlet: per energy tile its instance (nullptr: no tiled pass)
    int etiles = 0;
    double* epartials = nullptr;   // etiles
};
cudaError_t launch_invariants_batch(const InvBatchLaunch& B, cudaStream_t st);

// nlse_run's entry check on the device (check.cu): one entry per instance
// (a single grid: one; a stack: one per stacked instance; a batch: one per
// instance), each with its own points, dt and coefficients.
struct CheckEntry {
    int64_t psi_off;        // first element of the instance in Psi (and lo)
    int64_t v_off;          // first element of its V
    int64_t npts;
    double h, a, s, dt;
    double h2a;             // h^2 / a
    int dim;
    int row0, row1;         // its rows of partials
};
constexpr int64_t kPointsPerCheckRow = 16384;
constexpr int kMaxCheckRowsPerEntry = 2048;
// Rows of partials (blocks of the check) for an instance of npts points.
int check_rows(int64_t npts);
struct CheckLaunch {
    const CheckEntry* table;    // device, all entries, row0 ascending
    const int* row_entry;       // device, per row: the entry it belongs to
    int count, nrows, prec;     // checks entries inst_base .. inst_base + count - 1, whose rows
    int inst_base = 0;          // are row_base .. row_base + nrows - 1
    int row_base = 0;
    const void* psi;
    const void* lo;             // FP32 compensated part or nullptr
    const void* V;
    double* partials;           // nrows x 3
    double* bounds;             // count: each instance's bound of Eq. (kdfull)
    StatusBlock* status;
};
// Enqueues the check: partial extremes, then per instance the bound and the
// refusal bits.  No host synchronisation.
cudaError_t launch_entry_check(const CheckLaunch& C, cudaStream_t st);
// The same verdict from the reduced row (kPartialWidth doubles, on the
// device) of launch_invariants without energy: for MSD contexts, whose bound
// needs the boundary term.
cudaError_t launch_invariants_gate(const double* reduced, int dim, double h, double a, double dt, double* bound_out,
                                   StatusBlock* status, cudaStream_t st);

// The failure path of the bounded waits, run on purpose (selftest.cu): one
// warp waits on an mbarrier nothing completes, gives up after limit_ms and
// sets kStatusTimeout in *flag.
cudaError_t launch_bounded_wait_probe(int* flag, double limit_ms, cudaStream_t st);

// Records msg as the calling thread's nlse_last_error() and returns code.
int report_error(int code, const char* msg);
cudaError_t launch_invariants(const InvLaunch& L, double* partials, int nblocks, double* out,
                              cudaStream_t st);

}  // namespace nlse
