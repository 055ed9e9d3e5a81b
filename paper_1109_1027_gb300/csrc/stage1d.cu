// stage1d.cu -- fused RK4 stage and standalone 2SHOC Laplacian on a 1D grid.
//
// One CTA owns T consecutive output points.  The stage input is staged with
// a 3-point halo so that F is also known one point outside the tile, which
// the MSD rule of Eq. (msdbc_ut) needs at a boundary point whose interior
// neighbour belongs to the next tile.  Sweeps, all in shared memory:
//   D   = (Psi_{i+1} - 2 Psi_i + Psi_{i-1}) / h^2           Eq. (2shoc1d)
//   D_b from Eq. (dbc_lap), or Eq. (msdbc_lap) once interior D is known
//   Lap = (7/6) D_i - (1/12)(D_{i+1} + D_{i-1})              Eq. (2shoc1d2)
//   F   = i[a Lap + (s|Psi|^2 - V) Psi]; F_b from Eq. (dbc_ut) or (msdbc_ut)
// and the RK4 stage epilogue.
#include "nlse_device.cuh"

namespace nlse {
namespace {

constexpr int T = 1024;      // output points per CTA
constexpr int NT = 256;
constexpr int NP = T + 6;    // stage input, 3-point halo
constexpr int ND = T + 4;    // D, 2-point halo
constexpr int NF = T + 2;    // F (or Lap), 1-point halo

template <typename R, bool CD, bool MSD, int STAGE>
__global__ void __launch_bounds__(NT)
stage1d_kernel(StageIO<R> io, Coef<R> c, int n) {
    using C = cplx<R>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* sP = reinterpret_cast<C*>(smem_raw);   // x0-3 .. x0+T+2
    C* sD = sP + NP;                          // x0-2 .. x0+T+1
    C* sF = sD + ND;                          // x0-1 .. x0+T
    const int x0 = blockIdx.x * T;
    const int tid = threadIdx.x;
    if constexpr (STAGE == 4) {
        if (refused(io.flag)) return;
    }

    for (int j = tid; j < NP; j += NT) {
        int g = x0 - 3 + j;
        sP[j] = (g >= 0 && g < n) ? io.yin[g] : czero<C>();
    }
    __syncthreads();

    // Step 1 (boundary points provisionally take the Dirichlet value).
    for (int j = tid; j < ND; j += NT) {
        int g = x0 - 2 + j;
        const C* q = sP + j + 1;
        C d = czero<C>();
        if (!NLSE_IDX(io.flag, j + 2, NP, kSiteStage1d)) continue;
        if ((g == 0 || g == n - 1) && NLSE_IDX(io.flag, g, n, kSiteStage1d)) d = dirichlet_D(c, q[0], io.V[g]);
        else if (g > 0 && g < n - 1)
            d = cscale(c.inv_h2, csub(cadd(q[1], q[-1]), cscale((R)2, q[0])));
        sD[j] = d;
    }
    __syncthreads();
    if constexpr (MSD) {
        // D_b needs D at the interior neighbour q (Eq. msdbc_lap).
        if (tid < 2) {
            int g = tid == 0 ? 0 : n - 1;
            int qg = tid == 0 ? 1 : n - 2;
            int j = g - (x0 - 2);
            if (j >= 0 && j < ND) {
                int jq = qg - (x0 - 2);
                if (NLSE_IDX(io.flag, jq, ND, kSiteStage1d) && NLSE_IDX(io.flag, j + 1, NP, kSiteStage1d) &&
                    NLSE_IDX(io.flag, jq + 1, NP, kSiteStage1d))
                    sD[j] = msd_D(c, sP[j + 1], io.V[g], sP[jq + 1], io.V[qg], sD[jq]);
            }
        }
        __syncthreads();
    }

    // Step 2 and F on the tile plus one point each side.
    for (int j = tid; j < NF; j += NT) {
        int g = x0 - 1 + j;
        const C* e = sD + j + 1;
        C out = czero<C>();
        if (!(NLSE_IDX(io.flag, j + 2, ND, kSiteStage1d) && NLSE_IDX(io.flag, j + 2, NP, kSiteStage1d))) continue;
        if (g >= 0 && g < n) {
            bool bnd = (g == 0 || g == n - 1);
            C lap = (bnd || CD) ? e[0]
                                : csub(cscale((R)(7.0 / 6.0), e[0]),
                                       cscale((R)(1.0 / 12.0), cadd(e[1], e[-1])));
            if constexpr (STAGE == 0) out = lap;
            else if (!bnd) out = rhs_point(c, sP[j + 2], lap, io.V[g]);
        }
        sF[j] = out;
    }
    __syncthreads();

    bool bad = false;
    for (int j = tid; j < T; j += NT) {
        int g = x0 + j;
        if (g >= n) break;
        if (!(NLSE_IDX(io.flag, j + 1, NF, kSiteStage1d) && NLSE_IDX(io.flag, j + 3, NP, kSiteStage1d))) continue;
        C v = sF[j + 1];
        if constexpr (STAGE == 0) {
            io.lap[g] = v;
        } else {
            const C y = sP[j + 3];
            if (MSD && (g == 0 || g == n - 1)) {
                int qg = g == 0 ? 1 : n - 2;
                if (NLSE_IDX(io.flag, qg - (x0 - 3), NP, kSiteStage1d) && NLSE_IDX(io.flag, qg - (x0 - 1), NF, kSiteStage1d))
                    v = msd_F(y, sP[qg - (x0 - 3)], sF[qg - (x0 - 1)]);
            }
            bad |= stage_epilogue<STAGE>(io, g, y, v);
        }
    }
    if constexpr (STAGE == 4) {
        if (__syncthreads_or(bad) && tid == 0) atomicOr(io.flag, 1);
    }
}

template <typename R, bool CD, bool MSD, int STAGE>
cudaError_t launch_t(const StageLaunch& L, cudaStream_t st) {
    const int n = (int)L.n[0];
    size_t smem = sizeof(cplx<R>) * (NP + ND + NF);
    auto kern = stage1d_kernel<R, CD, MSD, STAGE>;
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    kern<<<(n + T - 1) / T, NT, smem, st>>>(make_io<R>(L), make_coef<R>(L.h, L.a, L.s), n);
    return cudaGetLastError();
}

template <typename R, bool CD, bool MSD>
cudaError_t launch_stage(const StageLaunch& L, cudaStream_t st) {
    switch (L.stage) {
        case 0: return launch_t<R, CD, MSD, 0>(L, st);
        case 1: return launch_t<R, CD, MSD, 1>(L, st);
        case 2: return launch_t<R, CD, MSD, 2>(L, st);
        case 3: return launch_t<R, CD, MSD, 3>(L, st);
        case 4: return launch_t<R, CD, MSD, 4>(L, st);
    }
    return cudaErrorInvalidValue;
}

template <typename R>
cudaError_t launch_prec(const StageLaunch& L, cudaStream_t st) {
    const bool cd = L.lap == 1, msd = L.bc == 1;
    if (cd) return msd ? launch_stage<R, true, true>(L, st) : launch_stage<R, true, false>(L, st);
    return msd ? launch_stage<R, false, true>(L, st) : launch_stage<R, false, false>(L, st);
}

}  // namespace

cudaError_t launch_stage_1d(const StageLaunch& L, cudaStream_t st) {
    return L.prec == 0 ? launch_prec<float>(L, st) : launch_prec<double>(L, st);
}

}  // namespace nlse
