// batch2d.cu -- many independent 2D NLSE instances of uneven sizes and
// parameters (own n, h, dt, a, s and V) advanced together: one launch per RK4
// stage covers every instance.
//
// Layout: every field (Psi, V and the work arrays) is one flat device buffer;
// instance i occupies n_x(i) * n_y(i) points from element offset off(i) = the
// sum of the earlier instances' sizes, row-major with x fastest.
//
// Each CTA takes one tile of the work list -- (instance, x0, y0) -- and runs
// the same TMA-fed streaming walk as the single-grid kernel
// (stage2d_tile.cuh) on that instance, with the instance's tensor maps and
// coefficients read from a descriptor table in device memory.  Instances are
// grouped by tile width (64 or 256 columns) so that narrow grids do not leave
// most of a CTA idle; each group is one launch per stage.  The tile list
// orders the instances from largest to smallest, which keeps the tail of each
// launch short.
#include <algorithm>
#include <cstring>
#include <new>
#include <type_traits>
#include <vector>

#include "nlse_internal.h"
#include "stage2d_tile.cuh"
#include "tmap.cuh"

namespace nlse {
namespace {

constexpr int TYB = 32;                       // rows per tile

// One instance's tensor maps and scalars (device-resident; CUtensorMap's own
// alignment keeps every map 64-byte aligned, as TMA descriptors in global
// memory must be).
struct BatchDesc {
    CUtensorMap in[3][2];                     // stage input Psi / Y0 / Y1: wide box + 4-point box
    CUtensorMap V, psi, acc, lo;              // output-row boxes
    int64_t off;
    int nx, ny, nt;                           // nt: threads per CTA of the instance's group
    double inv_h2, inv_6h2, a, s, inv_a;
    double c_acc[5], c_y[5];                  // stage weights from this instance's dt
};

template <typename R, int LP, int STAGE, int NT>
__global__ void __launch_bounds__(NT)
stage2d_batch_kernel(const BatchDesc* __restrict__ descs, const int4* __restrict__ tiles, StageIO<R> io,
                     const int dir) {
    // Stages that walk their rows upwards also take the tiles in reverse order:
    // the batch spans many waves of CTAs, and each stage then starts on the
    // tiles the previous stage wrote last, which are still in L2.
    const int4 tl = tiles[dir > 0 ? blockIdx.x : gridDim.x - 1 - blockIdx.x];
    const BatchDesc& d = descs[tl.x];
    // This instance's slice of every flat buffer (unused buffers stay null).
    auto at = [&](auto* ptr) { return ptr ? ptr + d.off : ptr; };
    io.yin = at(io.yin); io.psi = at(io.psi); io.psi_out = at(io.psi_out); io.acc = at(io.acc);
    io.yout = at(io.yout); io.V = at(io.V); io.lo = at(io.lo); io.lap = at(io.lap);
    io.rows1 = d.ny;
    io.c_acc = (R)d.c_acc[STAGE];
    io.c_y = (R)d.c_y[STAGE];
    Coef<R> c;
    c.inv_h2 = (R)d.inv_h2; c.inv_6h2 = (R)d.inv_6h2; c.a = (R)d.a; c.s = (R)d.s; c.inv_a = (R)d.inv_a;
    // Stage input: Psi for the Laplacian and stage 1, Y0 for stages 2 and 4, Y1 for stage 3.
    constexpr int sel = STAGE <= 1 ? 0 : (STAGE == 3 ? 2 : 1);
    tile2d::stage2d_tile<R, LP, STAGE, NT, TYB>(&d.in[sel][0], &d.in[sel][1], &d.V, &d.psi, &d.acc, &d.lo, io, c,
                                                d.nx, d.ny, tl.y, tl.z, dir);
}

template <typename R, int LP, int STAGE, int NT>
cudaError_t launch_group(const BatchDesc* descs, const int4* tiles, int ntiles, const StageIO<R>& io, int dir,
                         cudaStream_t st) {
    auto kern = stage2d_batch_kernel<R, LP, STAGE, NT>;
    const int smem = tile2d::Lay<R, NT, STAGE>::TOTAL;
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (e != cudaSuccess) return e;
    }
    kern<<<ntiles, NT, smem, st>>>(descs, tiles, io, dir);
    return cudaGetLastError();
}

template <typename R, int LP, int NT>
cudaError_t launch_stage_nt(int stage, const BatchDesc* descs, const int4* tiles, int ntiles,
                            const StageIO<R>& io, int dir, cudaStream_t st) {
    switch (stage) {
        case 0: return launch_group<R, LP, 0, NT>(descs, tiles, ntiles, io, dir, st);
        case 1: return launch_group<R, LP, 1, NT>(descs, tiles, ntiles, io, dir, st);
        case 2: return launch_group<R, LP, 2, NT>(descs, tiles, ntiles, io, dir, st);
        case 3: return launch_group<R, LP, 3, NT>(descs, tiles, ntiles, io, dir, st);
        case 4: return launch_group<R, LP, 4, NT>(descs, tiles, ntiles, io, dir, st);
    }
    return cudaErrorInvalidValue;
}

template <typename R>
cudaError_t launch_stage_r(int stage, int lap, int nt, const BatchDesc* descs, const int4* tiles, int ntiles,
                           const StageIO<R>& io, int dir, cudaStream_t st) {
    auto by_lap = [&](auto nt_c) -> cudaError_t {
        constexpr int NTC = decltype(nt_c)::value;
        switch (lap) {
            case 0: return launch_stage_nt<R, 0, NTC>(stage, descs, tiles, ntiles, io, dir, st);
            case 1: return launch_stage_nt<R, 1, NTC>(stage, descs, tiles, ntiles, io, dir, st);
            case 2: return launch_stage_nt<R, 2, NTC>(stage, descs, tiles, ntiles, io, dir, st);
        }
        return cudaErrorInvalidValue;
    };
    return nt == 32 ? by_lap(std::integral_constant<int, 32>()) : by_lap(std::integral_constant<int, 128>());
}

template <typename R>
bool encode_instance(BatchDesc& d, const void* const bases[6], int64_t off, int nx, int ny, int nt) {
    const size_t cb = sizeof(cplx<R>);
    auto cplx_at = [&](int k) { return static_cast<const char*>(bases[k]) + off * cb; };
    const int txc = 2 * nt;
    // bases: 0 psi (stage input 1 / Laplacian input), 1 Y0, 2 Y1, 3 acc, 4 lo, 5 V
    for (int s = 0; s < 3; ++s) {
        if (!complex_map<R>(&d.in[s][0], cplx_at(s), nx, ny, txc)) return false;
        if (!complex_map<R>(&d.in[s][1], cplx_at(s), nx, ny, 4)) return false;
    }
    if (!complex_map<R>(&d.psi, cplx_at(0), nx, ny, txc)) return false;
    if (!complex_map<R>(&d.acc, cplx_at(3), nx, ny, txc)) return false;
    if (bases[4]) {
        if (!complex_map<R>(&d.lo, cplx_at(4), nx, ny, txc)) return false;
    } else {
        d.lo = d.acc;
    }
    const char* v = static_cast<const char*>(bases[5]) + off * sizeof(R);
    return real_map<R>(&d.V, v, nx, ny, txc);
}

}  // namespace

struct BatchPlan {
    int count = 0, prec = 0, lap = 0;
    BatchDesc* host = nullptr;                // pinned copy of the table
    BatchDesc* dev = nullptr;
    int4* tiles = nullptr;                    // device work lists, group 0 then group 1
    int ntiles[2] = {0, 0};
    int nt[2] = {32, 128};
    int narrow = 64;
    const void* bases[6] = {};                // psi, Y0, Y1, acc, lo, V
    // Work lists of consecutive instance ranges (chunks) for a pipelined host
    // run: chunk k covers instances [chunk_first[k], chunk_first[k+1]).
    std::vector<int> chunk_first;
    int4* chunk_tiles = nullptr;              // per chunk: group 0 then group 1
    std::vector<int> chunk_off;               // first tile of chunk k's group g: chunk_off[2k + g]
    std::vector<int> chunk_n;                 // tiles of chunk k's group g: chunk_n[2k + g]
};

bool batch2d_instance_ok(const nlse_params& p) {
    return p.dim == 2 && p.bc == 0 && p.n[0] % (p.prec == 0 ? 4 : 2) == 0 && p.n[0] <= (1 << 30);
}

int64_t batch2d_points(const nlse_params& p) { return p.n[0] * p.n[1]; }

cudaError_t build_chunk_tiles(BatchPlan* b);

// Tile lists: instances with n[0] <= narrow get 64-column tiles (one warp),
// the rest 256-column tiles; largest instances first.
cudaError_t build_tiles(BatchPlan* b, int narrow) {
    std::vector<int> order(b->count);
    for (int i = 0; i < b->count; ++i) {
        order[i] = i;
        b->host[i].nt = b->host[i].nx <= narrow ? 32 : 128;
    }
    std::stable_sort(order.begin(), order.end(), [&](int x, int y) {
        return (int64_t)b->host[x].nx * b->host[x].ny > (int64_t)b->host[y].nx * b->host[y].ny;
    });
    std::vector<int4> lists[2];
    for (int i : order) {
        const BatchDesc& d = b->host[i];
        const int g = d.nt == 32 ? 0 : 1;
        const int txc = 2 * d.nt;
        for (int y0 = 0; y0 < d.ny; y0 += TYB)
            for (int x0 = 0; x0 < d.nx; x0 += txc) lists[g].push_back(make_int4(i, x0, y0, 0));
    }
    const size_t total = lists[0].size() + lists[1].size();
    cudaFree(b->tiles);
    b->tiles = nullptr;
    cudaError_t e = cudaMalloc((void**)&b->tiles, sizeof(int4) * (total ? total : 1));
    if (e != cudaSuccess) return e;
    for (int g = 0; g < 2; ++g) b->ntiles[g] = (int)lists[g].size();
    if (!lists[0].empty())
        e = cudaMemcpy(b->tiles, lists[0].data(), sizeof(int4) * lists[0].size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess && !lists[1].empty())
        e = cudaMemcpy(b->tiles + lists[0].size(), lists[1].data(), sizeof(int4) * lists[1].size(),
                       cudaMemcpyHostToDevice);
    b->narrow = narrow;
    if (e == cudaSuccess && !b->chunk_first.empty()) e = build_chunk_tiles(b);
    return e;
}

// The work lists of every chunk, built like the full lists (largest instance
// of the chunk first) from the current tile groups.
cudaError_t build_chunk_tiles(BatchPlan* b) {
    const int nch = (int)b->chunk_first.size() - 1;
    std::vector<int4> all;
    b->chunk_off.assign(2 * nch, 0);
    b->chunk_n.assign(2 * nch, 0);
    for (int k = 0; k < nch; ++k) {
        std::vector<int> order;
        for (int i = b->chunk_first[k]; i < b->chunk_first[k + 1]; ++i) order.push_back(i);
        std::stable_sort(order.begin(), order.end(), [&](int x, int y) {
            return (int64_t)b->host[x].nx * b->host[x].ny > (int64_t)b->host[y].nx * b->host[y].ny;
        });
        for (int g = 0; g < 2; ++g) {
            b->chunk_off[2 * k + g] = (int)all.size();
            for (int i : order) {
                const BatchDesc& d = b->host[i];
                if ((d.nt == 32 ? 0 : 1) != g) continue;
                const int txc = 2 * d.nt;
                for (int y0 = 0; y0 < d.ny; y0 += TYB)
                    for (int x0 = 0; x0 < d.nx; x0 += txc) all.push_back(make_int4(i, x0, y0, 0));
            }
            b->chunk_n[2 * k + g] = (int)all.size() - b->chunk_off[2 * k + g];
        }
    }
    cudaFree(b->chunk_tiles);
    b->chunk_tiles = nullptr;
    cudaError_t e = cudaMalloc((void**)&b->chunk_tiles, sizeof(int4) * (all.empty() ? 1 : all.size()));
    if (e != cudaSuccess) return e;
    if (!all.empty()) e = cudaMemcpy(b->chunk_tiles, all.data(), sizeof(int4) * all.size(), cudaMemcpyHostToDevice);
    return e;
}

cudaError_t batch2d_retile(BatchPlan* b, int narrow) {
    cudaError_t e = cudaDeviceSynchronize();          // no launch may still read the old lists
    if (e != cudaSuccess) return e;
    return build_tiles(b, narrow);                     // the maps are re-encoded at the next bind
}

int batch2d_narrow(const BatchPlan* b) { return b->narrow; }

cudaError_t batch2d_set_chunks(BatchPlan* b, const std::vector<int>& first) {
    b->chunk_first = first;
    return build_chunk_tiles(b);
}

int batch2d_chunks(const BatchPlan* b) { return b->chunk_first.empty() ? 0 : (int)b->chunk_first.size() - 1; }

cudaError_t batch2d_create(int count, const nlse_params* p, const void* V, void* Y0, void* Y1, void* acc,
                           void* lo, BatchPlan** out) {
    *out = nullptr;
    if (!encoder()) return cudaErrorNotSupported;       // no TMA descriptor encoder in this driver
    BatchPlan* b = new (std::nothrow) BatchPlan();
    if (!b) return cudaErrorMemoryAllocation;
    b->count = count;
    b->prec = p[0].prec;
    b->lap = p[0].lap;
    b->bases[1] = Y0; b->bases[2] = Y1; b->bases[3] = acc; b->bases[4] = lo; b->bases[5] = V;
    cudaError_t e = cudaMallocHost((void**)&b->host, sizeof(BatchDesc) * count);
    if (e == cudaSuccess) e = cudaMalloc((void**)&b->dev, sizeof(BatchDesc) * count);
    if (e != cudaSuccess) { batch2d_destroy(b); return e; }
    std::memset(b->host, 0, sizeof(BatchDesc) * count);

    // Offsets and scalars.
    std::vector<int64_t> off(count);
    int64_t acc_off = 0;
    for (int i = 0; i < count; ++i) {
        off[i] = acc_off;
        acc_off += batch2d_points(p[i]);
        BatchDesc& d = b->host[i];
        d.off = off[i];
        d.nx = (int)p[i].n[0];
        d.ny = (int)p[i].n[1];
        const double h = p[i].h, k = p[i].dt;
        d.inv_h2 = 1.0 / (h * h);
        d.inv_6h2 = 1.0 / (6.0 * h * h);
        d.a = p[i].a; d.s = p[i].s; d.inv_a = 1.0 / p[i].a;
        const double wa[5] = {0.0, k / 6.0, k / 3.0, k / 3.0, k / 6.0};
        const double wy[5] = {0.0, k / 2.0, k / 2.0, k, 0.0};
        for (int s = 0; s < 5; ++s) { d.c_acc[s] = wa[s]; d.c_y[s] = wy[s]; }
    }
    e = build_tiles(b, 64);
    if (e != cudaSuccess) { batch2d_destroy(b); return e; }
    *out = b;
    return cudaSuccess;
}

// (Re)encodes every instance's maps with `psi` as the Psi / stage-1 input
// buffer and uploads the table on the stream (synchronising it first).
cudaError_t batch2d_bind(BatchPlan* b, const void* psi, cudaStream_t st) {
    // The previous upload reads the pinned table asynchronously: let it finish
    // before the table is rewritten.
    cudaError_t e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return e;
    b->bases[0] = psi;
    for (int i = 0; i < b->count; ++i) {   // box widths follow the instance's tile group
        BatchDesc& d = b->host[i];
        const bool ok = b->prec == 0 ? encode_instance<float>(d, b->bases, d.off, d.nx, d.ny, d.nt)
                                     : encode_instance<double>(d, b->bases, d.off, d.nx, d.ny, d.nt);
        if (!ok) return cudaErrorInvalidValue;
    }
    return cudaMemcpyAsync(b->dev, b->host, sizeof(BatchDesc) * b->count, cudaMemcpyHostToDevice, st);
}

namespace {
cudaError_t launch_lists(BatchPlan* b, const StageLaunch& L, const int4* const lists[2], const int n[2],
                         cudaStream_t st) {
    // Same walk-direction alternation between stages as the single-grid kernel.
    const int dir = (L.stage % 2 == 0 && L.stage != 0) ? -1 : 1;
    for (int g = 0; g < 2; ++g) {
        if (!n[g]) continue;
        cudaError_t e;
        if (b->prec == 0) e = launch_stage_r<float>(L.stage, b->lap, b->nt[g], b->dev, lists[g], n[g],
                                                    make_io<float>(L), dir, st);
        else e = launch_stage_r<double>(L.stage, b->lap, b->nt[g], b->dev, lists[g], n[g],
                                        make_io<double>(L), dir, st);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}
}  // namespace

cudaError_t batch2d_launch(BatchPlan* b, const StageLaunch& L, cudaStream_t st) {
    const int4* lists[2] = {b->tiles, b->tiles + b->ntiles[0]};
    return launch_lists(b, L, lists, b->ntiles, st);
}

cudaError_t batch2d_launch_chunk(BatchPlan* b, const StageLaunch& L, int k, cudaStream_t st) {
    const int4* lists[2] = {b->chunk_tiles + b->chunk_off[2 * k], b->chunk_tiles + b->chunk_off[2 * k + 1]};
    const int n[2] = {b->chunk_n[2 * k], b->chunk_n[2 * k + 1]};
    return launch_lists(b, L, lists, n, st);
}

void batch2d_destroy(BatchPlan* b) {
    if (!b) return;
    cudaFreeHost(b->host);
    cudaFree(b->dev);
    cudaFree(b->tiles);
    cudaFree(b->chunk_tiles);
    delete b;
}

}  // namespace nlse
