// stage2d_tma.cuh -- the fused 2D RK4 stage (and standalone 2SHOC Laplacian)
// on one grid: a grid of CTAs, each running the TMA-fed y-streaming walk of
// stage2d_tile.cuh over TXC = 256 columns and TY rows.  TY is a tiling
// choice (8, 16 or 32; 16 by default: a 2048 x 2048 grid is then one wave of
// 1024 CTAs on 152 SMs at 7 CTAs per SM); each TY is instantiated in its own
// translation unit (stage2d_tma_r{8,16,32}.cu).
#pragma once

#include "stage2d_tile.cuh"
#include "tmap.cuh"

namespace nlse {
namespace tma2d {

constexpr int NT = 128;              // threads per CTA
constexpr int TXC = 2 * NT;          // columns per CTA
constexpr int HB = TXC;              // first input TMA box; the second is 4 points
constexpr int HB2 = 4;

template <typename R, int LP, int STAGE, int TY>
__global__ void __launch_bounds__(NT)
stage2d_tma_kernel(const __grid_constant__ CUtensorMap m_in, const __grid_constant__ CUtensorMap m_in2,
                   const __grid_constant__ CUtensorMap m_V,
                   const __grid_constant__ CUtensorMap m_psi, const __grid_constant__ CUtensorMap m_acc,
                   const __grid_constant__ CUtensorMap m_lo, const StageIO<R> io, const Coef<R> c,
                   const int nx, const int ny, const int dir) {
    tile2d::stage2d_tile<R, LP, STAGE, NT, TY>(&m_in, &m_in2, &m_V, &m_psi, &m_acc, &m_lo, io, c, nx, ny,
                                               blockIdx.x * TXC, blockIdx.y * TY, dir);
}

// ---- host side -------------------------------------------------------------

template <typename R, int LP, int STAGE, int TY>
cudaError_t launch_t(const StageLaunch& L, cudaStream_t st) {
    using tile2d::Lay;
    const int nx = (int)L.n[0], ny = (int)L.n[1];
    CUtensorMap m_in, m_in2, m_V, m_psi, m_acc, m_lo;
    if (!complex_map<R>(&m_in, L.yin, nx, ny, HB) || !complex_map<R>(&m_in2, L.yin, nx, ny, HB2))
        return cudaErrorInvalidValue;
    m_V = m_psi = m_acc = m_lo = m_in;
    const int rows1 = (int)(L.rows1 ? L.rows1 : ny);    // V has the rows of one stacked instance
    if (STAGE >= 1 && !real_map<R>(&m_V, L.V, nx, rows1, TXC)) return cudaErrorInvalidValue;
    if (STAGE >= 2) {
        if (!complex_map<R>(&m_psi, L.psi, nx, ny, TXC) || !complex_map<R>(&m_acc, L.acc, nx, ny, TXC))
            return cudaErrorInvalidValue;
    }
    if (STAGE == 4 && sizeof(R) == 4 && !complex_map<R>(&m_lo, L.lo, nx, ny, TXC)) return cudaErrorInvalidValue;
    auto kern = stage2d_tma_kernel<R, LP, STAGE, TY>;
    const int smem = Lay<R, NT, STAGE>::TOTAL;
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (e != cudaSuccess) return e;
    }
    dim3 grid((nx + TXC - 1) / TXC, (ny + TY - 1) / TY);
    // Consecutive stages walk the rows in opposite directions, so that each
    // stage starts on the rows the previous one wrote last (still in L2).
    const int dir = (STAGE % 2 == 0 && STAGE != 0) ? -1 : 1;
    kern<<<grid, NT, smem, st>>>(m_in, m_in2, m_V, m_psi, m_acc, m_lo, make_io<R>(L), make_coef<R>(L.h, L.a, L.s), nx,
                                 ny, dir);
    return cudaGetLastError();
}

template <typename R, int LP, int TY>
cudaError_t launch_stage(const StageLaunch& L, cudaStream_t st) {
    switch (L.stage) {
        case 0: return launch_t<R, LP, 0, TY>(L, st);
        case 1: return launch_t<R, LP, 1, TY>(L, st);
        case 2: return launch_t<R, LP, 2, TY>(L, st);
        case 3: return launch_t<R, LP, 3, TY>(L, st);
        case 4: return launch_t<R, LP, 4, TY>(L, st);
    }
    return cudaErrorInvalidValue;
}

template <typename R, int TY>
cudaError_t launch_lap(const StageLaunch& L, cudaStream_t st) {
    switch (L.lap) {
        case 0: return launch_stage<R, 0, TY>(L, st);
        case 1: return launch_stage<R, 1, TY>(L, st);
        case 2: return launch_stage<R, 2, TY>(L, st);
    }
    return cudaErrorInvalidValue;
}

template <int TY>
cudaError_t launch_rows(const StageLaunch& L, cudaStream_t st) {
    return L.prec == 0 ? launch_lap<float, TY>(L, st) : launch_lap<double, TY>(L, st);
}

}  // namespace tma2d
}  // namespace nlse
