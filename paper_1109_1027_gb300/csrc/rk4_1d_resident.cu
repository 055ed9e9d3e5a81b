// rk4_1d_resident.cu -- whole RK4 time loops on a small 1D grid inside one
// thread-block cluster.  One-dimensional problems (a few thousand points) are
// far too small to fill the GPU, so the four launches per step of the tiled
// path are pure latency.  Here one launch runs every stage of every step: the
// grid is cut into CS contiguous chunks, one per CTA of a cluster (CS = 1 is a
// single CTA).  Each CTA keeps its chunk of the stage input Y (with a 2-point
// halo), D and F in shared memory and each point's Psi^n, compensated part,
// accumulator and V in registers.  Per stage: each CTA has written the two
// points at each edge of its new Y into the halo slots of its neighbours'
// shared memory, and a cluster barrier publishes them; then step 1 (Eq. 2shoc1d) with the boundary value D_b (Eq. dbc_lap, or Eq.
// msdbc_lap once interior D is known), step 2 (Eq. 2shoc1d2), F with its
// boundary rule (Eq. dbc_ut / msdbc_ut) and the RK4 stage update.  The
// per-point arithmetic is the same device code as the tiled kernel
// (stage1d.cu), so the two give the same bits for every CS.
//
// Spreading the chunk over several SMs matters most in FP64, whose per-SM
// rate on this part is a few FMAs per clock: one CTA is bound by it.
//
// Y is double-buffered when CS > 1: stage g reads buffer g % 2 and writes
// Y_{g+1}, own points and the neighbours' halo slots, to the other buffer; the
// barrier before stage g + 1 orders every read of buffer g % 2 before its
// rewrite at stage g + 1.  A first barrier makes sure every CTA runs before
// any writes into its shared memory, a last one that none exits while a
// neighbour may still write into it.  The cluster barrier is the hardware one,
// with all CTAs of a cluster co-scheduled by construction.
#include <cooperative_groups.h>

#include <atomic>

#include "nlse_device.cuh"

namespace cg = cooperative_groups;

namespace nlse {
namespace {

constexpr int MAX_T = 1024;
constexpr int MAX_PPT = 4;                    // points per thread: chunk <= 4096
constexpr int MAX_CS = 16;
constexpr int MIN_CHUNK = 32;                 // smallest chunk worth its own CTA

// Stage weights, rounded from FP64 on the host exactly as for the tiled kernels.
template <typename R> struct Weights { R acc[5], y[5]; };

template <typename R, bool CD, bool MSD, int PPT>
__global__ void __launch_bounds__(MAX_T) rk4_1d_resident_kernel(cplx<R>* psi_g, cplx<R>* lo_g, const R* V_g,
                                                                Coef<R> c, Weights<R> w, int n, int m,
                                                                int64_t nsteps, int* flag) {
    using C = cplx<R>;
    if (refused(flag)) return;                             // every CTA of the cluster, before any cluster barrier
    cg::cluster_group cl = cg::this_cluster();
    const int CS = (int)cl.num_blocks();
    const int r = (int)cl.block_rank();
    const int nbuf = CS > 1 ? 2 : 1;
    const int p0 = r * m;                                  // first own point
    const int mr = min(m, n - p0);                         // own points (>= 2)
    const bool first = r == 0, last = r == CS - 1;

    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* sY = reinterpret_cast<C*>(smem_raw);                // [nbuf][m + 4]: local j <-> point p0 - 2 + j
    C* sD = sY + nbuf * (m + 4);                           // [m + 2]: local j <-> point p0 - 1 + j
    C* sF = sD + (m + 2);                                  // [m] (MSD only): local j <-> point p0 + j
    const int tid = threadIdx.x, T = blockDim.x;

    // Writes own point j of buffer b and, for the two points at each chunk
    // edge, the matching halo slot of the neighbouring CTA.
    auto publish = [&](int b, int j, C v) {
        C* Yb = sY + b * (m + 4);
        Yb[j + 2] = v;
        if (CS > 1) {
            if (j < 2 && !first) cl.map_shared_rank(Yb, r - 1)[m + 2 + j] = v;
            if (j >= mr - 2 && !last) cl.map_shared_rank(Yb, r + 1)[j - mr + 2] = v;
        }
    };
    auto barrier = [&]() {
        if (CS > 1) cl.sync();
        else __syncthreads();
    };

#ifdef NLSE_BOUNDS_CHECK
    {
        // The chunk inside the grid and the three shared buffers inside the
        // launch's dynamic shared memory (recorded only: a CTA may not leave
        // before the cluster barriers its neighbours wait at).
        uint32_t dyn;
        asm("mov.u32 %0, %%dynamic_smem_size;" : "=r"(dyn));
        const int64_t need = (int64_t)(nbuf * (m + 4) + (m + 2) + (MSD ? m : 0)) * (int64_t)sizeof(C);
        (void)(NLSE_IDX(flag, p0 + mr - 1, n, kSiteResident1d) && NLSE_IDX(flag, mr - 2, m - 1, kSiteResident1d) &&
               NLSE_IDX(flag, need - 1, dyn, kSiteResident1d));
    }
#endif
    // Every CTA of the cluster must be running before any writes its shared memory.
    if (CS > 1) cl.sync();
    C psi[PPT], lo[PPT], acc[PPT];
    R V[PPT];
#pragma unroll
    for (int k = 0; k < PPT; ++k) {
        const int j = tid + k * T;
        if (j < mr && NLSE_IDX(flag, p0 + j, n, kSiteResident1d)) {
            psi[k] = psi_g[p0 + j];
            lo[k] = lo_g ? lo_g[p0 + j] : czero<C>();
            V[k] = V_g[p0 + j];
            publish(0, j, psi[k]);
        }
    }
    bool bad = false;
    int buf = 0;
    for (int64_t step = 0; step < nsteps; ++step) {
#pragma unroll
        for (int stage = 1; stage <= 4; ++stage) {
            barrier();
            const C* Y = sY + buf * (m + 4);
            // Step 1: own D (boundary D_b by Dirichlet, provisional for MSD) and
            // the interior D one point beyond each chunk edge.
#pragma unroll
            for (int k = 0; k < PPT; ++k) {
                const int j = tid + k * T;
                if (j >= mr) continue;
                const int p = p0 + j;
                const C* y = Y + j + 2;
                sD[j + 1] = (p == 0 || p == n - 1) ? dirichlet_D(c, y[0], V[k])
                                                   : cscale(c.inv_h2, csub(cadd(y[1], y[-1]), cscale((R)2, y[0])));
            }
            if (tid == 0 && !first) {
                const C* y = Y + 1;
                sD[0] = cscale(c.inv_h2, csub(cadd(y[1], y[-1]), cscale((R)2, y[0])));
            } else if (tid == 1 && !last) {
                const C* y = Y + mr + 2;
                sD[mr + 1] = cscale(c.inv_h2, csub(cadd(y[1], y[-1]), cscale((R)2, y[0])));
            }
            __syncthreads();
            if constexpr (MSD) {
                if (tid == 0 && first) sD[1] = msd_D(c, Y[2], V_g[0], Y[3], V_g[1], sD[2]);
                if (tid == 1 && last) sD[mr] = msd_D(c, Y[mr + 1], V_g[n - 1], Y[mr], V_g[n - 2], sD[mr - 1]);
                __syncthreads();
            }
            // Step 2 and F.
            C F[PPT];
#pragma unroll
            for (int k = 0; k < PPT; ++k) {
                const int j = tid + k * T;
                const int p = p0 + j;
                F[k] = czero<C>();
                if (j >= mr || p == 0 || p == n - 1) continue;
                const C* d = sD + j + 1;
                const C lap = CD ? d[0] : csub(cscale((R)(7.0 / 6.0), d[0]), cscale((R)(1.0 / 12.0), cadd(d[1], d[-1])));
                F[k] = rhs_point(c, Y[j + 2], lap, V[k]);
                if (MSD) sF[j] = F[k];
            }
            if constexpr (MSD) {
                __syncthreads();
#pragma unroll
                for (int k = 0; k < PPT; ++k) {
                    const int j = tid + k * T;
                    if (first && j == 0) F[k] = msd_F(Y[2], Y[3], sF[1]);
                    if (last && j == mr - 1) F[k] = msd_F(Y[mr + 1], Y[mr], sF[mr - 2]);
                }
                __syncthreads();
            }
            // RK4 stage update (same algebra as the tiled kernels' epilogue).
            const int nb = nbuf == 2 ? buf ^ 1 : buf;
#pragma unroll
            for (int k = 0; k < PPT; ++k) {
                const int j = tid + k * T;
                if (j >= mr) continue;
                if (stage == 1) {
                    acc[k] = cscale(w.acc[1], F[k]);
                    publish(nb, j, caxpy(psi[k], w.y[1], F[k]));
                } else if (stage < 4) {
                    acc[k] = caxpy(acc[k], w.acc[stage], F[k]);
                    publish(nb, j, caxpy(psi[k], w.y[stage], F[k]));
                } else {
                    const C d = caxpy(acc[k], w.acc[4], F[k]);
                    if constexpr (sizeof(R) == 4) {
                        kahan_add(psi[k].x, lo[k].x, d.x);
                        kahan_add(psi[k].y, lo[k].y, d.y);
                    } else {
                        psi[k] = cadd(psi[k], d);
                    }
                    publish(nb, j, psi[k]);
                    bad |= !(isfinite(psi[k].x) && isfinite(psi[k].y));
                }
            }
            buf = nb;
        }
    }
#pragma unroll
    for (int k = 0; k < PPT; ++k) {
        const int j = tid + k * T;
        if (j < mr && NLSE_IDX(flag, p0 + j, n, kSiteResident1d)) {
            psi_g[p0 + j] = psi[k];
            if (lo_g) lo_g[p0 + j] = lo[k];
        }
    }
    if (__syncthreads_or(bad) && tid == 0) atomicOr(flag, 1);
    if (CS > 1) cl.sync();
}

// Chunk length for a cluster of cs CTAs, or 0 when cs does not fit n: every
// chunk needs MIN_CHUNK points (the last one at least 2, so that the MSD
// boundary neighbours and every halo D point stay interior to one CTA) and at
// most PPT * MAX_T.
int chunk_for(int64_t n, int cs) {
    const int64_t m = (n + cs - 1) / cs;
    if (m > (int64_t)MAX_PPT * MAX_T) return 0;
    if (cs > 1 && (m < MIN_CHUNK || n - (int64_t)(cs - 1) * m < 2)) return 0;
    return (int)m;
}

size_t smem_bytes(int m, int cs, bool msd, size_t elem) {
    const int nbuf = cs > 1 ? 2 : 1;
    return elem * ((size_t)nbuf * (m + 4) + (m + 2) + (msd ? m : 0));
}

template <typename R, bool CD, bool MSD, int PPT>
cudaError_t launch_t(const ResidentLaunch& L, int cs, cudaStream_t st) {
    auto kern = rk4_1d_resident_kernel<R, CD, MSD, PPT>;
    // Whether a cluster of 2^i CTAs can be resident: -1 unknown, 0 no, 1 yes.
    static std::atomic<int> cluster_ok[5] = {-1, -1, -1, -1, -1};
    for (;; cs /= 2) {
        const int m = chunk_for(L.n, cs);
        const size_t smem = smem_bytes(m, cs, MSD, sizeof(cplx<R>));
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        if (cs > 8) {
            e = cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
            if (e != cudaSuccess) return e;
        }
        const int T = (int)std::min<int64_t>(MAX_T, (std::min(m, (int)((L.n + cs - 1) / cs)) + 31) / 32 * 32);
        cudaLaunchConfig_t cfg = {};
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = cs;
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
        cfg.gridDim = dim3(cs);
        cfg.blockDim = dim3(T);
        cfg.dynamicSmemBytes = smem;
        cfg.stream = st;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        if (cs > 1) {
            int lg = 0;
            while ((1 << lg) < cs) ++lg;
            int ok = cluster_ok[lg].load();
            if (ok < 0) {
                int clusters = 0;
                e = cudaOccupancyMaxActiveClusters(&clusters, kern, &cfg);
                if (e != cudaSuccess) {
                    (void)cudaGetLastError();
                    clusters = 0;
                }
                ok = clusters > 0 ? 1 : 0;
                cluster_ok[lg].store(ok);
            }
            if (!ok) continue;
        }
        Weights<R> w;
        const double k = L.dt;
        const double wa[5] = {0.0, k / 6.0, k / 3.0, k / 3.0, k / 6.0};
        const double wy[5] = {0.0, k / 2.0, k / 2.0, k, 0.0};
        for (int s = 0; s < 5; ++s) { w.acc[s] = (R)wa[s]; w.y[s] = (R)wy[s]; }
        return cudaLaunchKernelEx(&cfg, kern, (cplx<R>*)L.psi, (cplx<R>*)L.lo, (const R*)L.V,
                                  make_coef<R>(L.h, L.a, L.s), w, (int)L.n, m, L.nsteps, L.flag);
    }
}

// One point per thread where the chunk allows (no register pressure), else up to MAX_PPT.
template <typename R, bool CD, bool MSD>
cudaError_t launch_p(const ResidentLaunch& L, cudaStream_t st) {
    int cs = 1;
    while (cs * 2 <= L.max_cluster && chunk_for(L.n, cs * 2)) cs *= 2;
    if (chunk_for(L.n, cs) <= MAX_T) return launch_t<R, CD, MSD, 1>(L, cs, st);
    return launch_t<R, CD, MSD, MAX_PPT>(L, cs, st);
}

template <typename R>
cudaError_t launch_r(const ResidentLaunch& L, cudaStream_t st) {
    const bool cd = L.lap == 1, msd = L.bc == 1;
    if (cd) return msd ? launch_p<R, true, true>(L, st) : launch_p<R, true, false>(L, st);
    return msd ? launch_p<R, false, true>(L, st) : launch_p<R, false, false>(L, st);
}

}  // namespace

bool rk4_1d_resident_fits(int64_t n) { return n >= 3 && chunk_for(n, 1) > 0; }

int rk4_1d_max_cluster() { return MAX_CS; }

cudaError_t launch_rk4_1d_resident(const ResidentLaunch& L, cudaStream_t st) {
    if (L.max_cluster < 1 || L.max_cluster > MAX_CS || !rk4_1d_resident_fits(L.n)) return cudaErrorInvalidValue;
    return L.prec == 0 ? launch_r<float>(L, st) : launch_r<double>(L, st);
}

}  // namespace nlse
