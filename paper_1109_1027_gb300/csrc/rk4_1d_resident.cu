// rk4_1d_resident.cu -- whole RK4 time loops on a small 1D grid inside one
// CTA.  One-dimensional problems (a few thousand points) are far too small to
// fill the GPU, so the four launches per step of the tiled path are pure
// latency.  Here one CTA of 1024 threads keeps the stage input, D and F in
// shared memory and each point's Psi^n, compensated part, accumulator and V
// in registers, and runs every stage of every step with CTA barriers between
// the sweeps: step 1 (Eq. 2shoc1d), the boundary value D_b (Eq. dbc_lap, or
// Eq. msdbc_lap once interior D is known), step 2 (Eq. 2shoc1d2), F with its
// boundary rule (Eq. dbc_ut / msdbc_ut) and the RK4 stage update.  The
// per-point arithmetic is the same device code as the tiled kernel
// (stage1d.cu), so the two give the same bits.
#include "nlse_device.cuh"

namespace nlse {
namespace {

constexpr int NT = 1024;
constexpr int PPT = 4;                        // points per thread: n <= 4096

// Stage weights, rounded from FP64 on the host exactly as for the tiled kernels.
template <typename R> struct Weights { R acc[5], y[5]; };

template <typename R, bool CD, bool MSD>
__global__ void __launch_bounds__(NT) rk4_1d_resident_kernel(cplx<R>* psi_g, cplx<R>* lo_g, const R* V_g,
                                                             Coef<R> c, Weights<R> w, int n, int64_t nsteps,
                                                             int* flag) {
    using C = cplx<R>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* sY = reinterpret_cast<C*>(smem_raw);   // stage input
    C* sD = sY + n;                           // step-1 field
    C* sF = sD + n;                           // F (MSD boundary rule needs F at b-1)
    const int tid = threadIdx.x;

    C psi[PPT], lo[PPT], acc[PPT];
    R V[PPT];
#pragma unroll
    for (int m = 0; m < PPT; ++m) {
        const int p = tid + m * NT;
        if (p < n) {
            psi[m] = psi_g[p];
            lo[m] = lo_g ? lo_g[p] : czero<C>();
            V[m] = V_g[p];
            sY[p] = psi[m];
        }
    }
    const R* wa = w.acc;
    const R* wy = w.y;
    bool bad = false;
    for (int64_t step = 0; step < nsteps; ++step) {
        for (int stage = 1; stage <= 4; ++stage) {
            __syncthreads();
            // Step 1: interior D; boundary D_b by Dirichlet (provisional for MSD).
#pragma unroll
            for (int m = 0; m < PPT; ++m) {
                const int p = tid + m * NT;
                if (p >= n) continue;
                C d;
                if (p == 0 || p == n - 1) d = dirichlet_D(c, sY[p], V[m]);
                else d = cscale(c.inv_h2, csub(cadd(sY[p + 1], sY[p - 1]), cscale((R)2, sY[p])));
                sD[p] = d;
            }
            __syncthreads();
            if constexpr (MSD) {
                if (tid < 2) {
                    const int b = tid == 0 ? 0 : n - 1, q = tid == 0 ? 1 : n - 2;
                    sD[b] = msd_D(c, sY[b], V_g[b], sY[q], V_g[q], sD[q]);
                }
                __syncthreads();
            }
            // Step 2 and F.
            C F[PPT];
#pragma unroll
            for (int m = 0; m < PPT; ++m) {
                const int p = tid + m * NT;
                F[m] = czero<C>();
                if (p >= n || p == 0 || p == n - 1) continue;
                const C lap = CD ? sD[p] : csub(cscale((R)(7.0 / 6.0), sD[p]),
                                                cscale((R)(1.0 / 12.0), cadd(sD[p + 1], sD[p - 1])));
                F[m] = rhs_point(c, sY[p], lap, V[m]);
                if (MSD) sF[p] = F[m];
            }
            if constexpr (MSD) {
                __syncthreads();
#pragma unroll
                for (int m = 0; m < PPT; ++m) {
                    const int p = tid + m * NT;
                    if (p == 0) F[m] = msd_F(sY[0], sY[1], sF[1]);
                    if (p == n - 1) F[m] = msd_F(sY[n - 1], sY[n - 2], sF[n - 2]);
                }
                __syncthreads();
            }
            // RK4 stage update (same algebra as the tiled kernels' epilogue).
#pragma unroll
            for (int m = 0; m < PPT; ++m) {
                const int p = tid + m * NT;
                if (p >= n) continue;
                if (stage == 1) {
                    acc[m] = cscale(wa[1], F[m]);
                    sY[p] = caxpy(psi[m], wy[1], F[m]);
                } else if (stage < 4) {
                    acc[m] = caxpy(acc[m], wa[stage], F[m]);
                    sY[p] = caxpy(psi[m], wy[stage], F[m]);
                } else {
                    const C d = caxpy(acc[m], wa[4], F[m]);
                    if constexpr (sizeof(R) == 4) {
                        kahan_add(psi[m].x, lo[m].x, d.x);
                        kahan_add(psi[m].y, lo[m].y, d.y);
                    } else {
                        psi[m] = cadd(psi[m], d);
                    }
                    sY[p] = psi[m];
                    bad |= !(isfinite(psi[m].x) && isfinite(psi[m].y));
                }
            }
        }
    }
#pragma unroll
    for (int m = 0; m < PPT; ++m) {
        const int p = tid + m * NT;
        if (p < n) {
            psi_g[p] = psi[m];
            if (lo_g) lo_g[p] = lo[m];
        }
    }
    if (__syncthreads_or(bad) && tid == 0) atomicOr(flag, 1);
}

template <typename R, bool CD, bool MSD>
cudaError_t launch_t(const ResidentLaunch& L, cudaStream_t st) {
    auto kern = rk4_1d_resident_kernel<R, CD, MSD>;
    const size_t smem = sizeof(cplx<R>) * 3 * (size_t)L.n;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    Weights<R> w;
    const double k = L.dt;
    const double wa[5] = {0.0, k / 6.0, k / 3.0, k / 3.0, k / 6.0};
    const double wy[5] = {0.0, k / 2.0, k / 2.0, k, 0.0};
    for (int s = 0; s < 5; ++s) { w.acc[s] = (R)wa[s]; w.y[s] = (R)wy[s]; }
    kern<<<1, NT, smem, st>>>((cplx<R>*)L.psi, (cplx<R>*)L.lo, (const R*)L.V, make_coef<R>(L.h, L.a, L.s), w,
                              (int)L.n, L.nsteps, L.flag);
    return cudaGetLastError();
}

template <typename R>
cudaError_t launch_r(const ResidentLaunch& L, cudaStream_t st) {
    const bool cd = L.lap == 1, msd = L.bc == 1;
    if (cd) return msd ? launch_t<R, true, true>(L, st) : launch_t<R, true, false>(L, st);
    return msd ? launch_t<R, false, true>(L, st) : launch_t<R, false, false>(L, st);
}

}  // namespace

bool rk4_1d_resident_fits(int64_t n) { return n >= 3 && n <= (int64_t)NT * PPT; }

cudaError_t launch_rk4_1d_resident(const ResidentLaunch& L, cudaStream_t st) {
    return L.prec == 0 ? launch_r<float>(L, st) : launch_r<double>(L, st);
}

}  // namespace nlse
