// stage3d.cu -- fused RK4 stage and standalone 2SHOC Laplacian on a 3D grid:
// the generic kernel (FP64, and FP32 grids whose rows TMA cannot address);
// the TMA-fed FP32 kernel is in stage3d_tma.cu.
//
// One CTA owns a TX x TY column of the grid over TZ consecutive z planes and
// streams through them (2.5D blocking): shared memory holds a ring of three
// stage-input planes (z .. z+2, each with a 2-point xy halo) and three D
// planes (z-1 .. z+1, 1-point xy halo).  Per plane it loads input plane z+2,
// computes step 1, the seven-point D of Eq. (3d2shocs), for plane z+1
// (boundary points take D_b of Eq. dbc_lap), and evaluates step 2,
// Eq. (3d2shocs2),
//     Lap = -(1/12)[sum of the six axial D - 10 D_c]
//           + (1/(6h^2))[sum of the twelve edge neighbours of Psi - 12 Psi_c],
// then F, the Dirichlet rule F_b = 0 and the RK4 stage epilogue for plane z.
// Each input plane is read once per CTA, so the halo overhead is only the xy
// ring plus four planes per TZ.  Step 1 forms, at every point, the sum hx of
// its two x neighbours and the sum q of its four in-plane axial neighbours;
// rings keep them, and step 2 takes the x-z and y-z edge terms of plane z as
// q(z-1) + q(z+1) and the four in-plane diagonals as hx(y-1) + hx(y+1)
// instead of adding the values again (16 fewer FP64 additions per point and
// stage; FP64 arithmetic bounds the FP64 kernel on this GPU).  The FP64
// stages also carry a Lap: the a of F goes into the difference weights and the
// boundary value a D_b = -N_b Psi_b (Eq. dbc_lap), two multiplies fewer.
#include "nlse_device.cuh"
#include "tmap.cuh"

namespace nlse {
namespace {

constexpr int TX = 32, TY = 16, TZ = 32;
constexpr int NT = 256;
constexpr int PX = TX + 4, PY = TY + 4, PP = PX * PY;   // input plane with halo 2
constexpr int DX = TX + 2, DY = TY + 2, DP = DX * DY;   // D plane with halo 1

__device__ __forceinline__ int pslot(int z) { return (z + 4) & 3; }
__device__ __forceinline__ int dslot(int z) { return (z + 3) % 3; }

template <typename R, bool CD, int STAGE>
__global__ void __launch_bounds__(NT)
stage3d_kernel(StageIO<R> io, Coef<R> c, int nx, int ny, int nz) {
    using C = cplx<R>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* sP = reinterpret_cast<C*>(smem_raw);   // [3][PY][PX]
    C* sD = sP + 3 * PP;                      // [3][DY][DX]
    C* sQ = sD + 3 * DP;                      // [3][TY][TX]: in-plane axial sums of the tile's points
    C* sH = sQ + 3 * TX * TY;                 // [2][TY+2][TX]: x-neighbour sums, tile columns, rows y0-1 .. y0+TY
    // FP64 stages fold a into the weights (a Lap instead of Lap); FP32 and the
    // standalone Laplacian keep the unscaled form.
    constexpr bool SC = sizeof(R) == 8 && STAGE >= 1;
    const R wd = SC ? c.a * c.inv_h2 : c.inv_h2, we = SC ? c.a * c.inv_6h2 : c.inv_6h2;

    const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY, z0 = blockIdx.z * TZ;
    const int z1 = min(z0 + TZ, nz);
    const int tid = threadIdx.x;
    const int64_t plane = (int64_t)nx * ny;
    if constexpr (STAGE == 4) {
        if (refused(io.flag)) return;
    }

    auto load_plane = [&](int gz) {
        C* dst = sP + dslot(gz) * PP;
        const bool zin = gz >= 0 && gz < nz;
        for (int i = tid; i < PP; i += NT) {
            int ly = i / PX, lx = i - ly * PX;
            int gx = x0 - 2 + lx, gy = y0 - 2 + ly;
            C v = czero<C>();
            if (zin && gx >= 0 && gx < nx && gy >= 0 && gy < ny)
                v = io.yin[gz * plane + (int64_t)gy * nx + gx];
            dst[i] = v;
        }
    };
    auto d_plane = [&](int gz) {
        C* dst = sD + dslot(gz) * DP;
        C* qdst = sQ + dslot(gz) * (TX * TY);
        C* hdst = sH + ((gz + 2) & 1) * (TX * (TY + 2));
        const C* pm = sP + dslot(gz - 1) * PP;
        const C* pc = sP + dslot(gz) * PP;
        const C* pp = sP + dslot(gz + 1) * PP;
        const bool zin = gz >= 0 && gz < nz;
        const bool zb = gz == 0 || gz == nz - 1;
        for (int i = tid; i < DP; i += NT) {
            int ly = i / DX, lx = i - ly * DX;
            int gx = x0 - 1 + lx, gy = y0 - 1 + ly;
            int k = (ly + 1) * PX + (lx + 1);
            C d = czero<C>();
            if (!(NLSE_IDX(io.flag, k - PX, PP, kSiteStage3d) && NLSE_IDX(io.flag, k + PX, PP, kSiteStage3d))) continue;
            // in-plane neighbour sums (the values outside the grid read as zero)
            const C hx = cadd(pc[k + 1], pc[k - 1]);
            const C q = cadd(hx, cadd(pc[k + PX], pc[k - PX]));
            if (lx >= 1 && lx <= TX && NLSE_IDX(io.flag, ly * TX + lx - 1, TX * (TY + 2), kSiteStage3d))
                hdst[ly * TX + (lx - 1)] = hx;
            if (lx >= 1 && lx <= TX && ly >= 1 && ly <= TY &&
                NLSE_IDX(io.flag, (ly - 1) * TX + lx - 1, TX * TY, kSiteStage3d))
                qdst[(ly - 1) * TX + (lx - 1)] = q;
            if (zin && gx >= 0 && gx < nx && gy >= 0 && gy < ny) {
                C ctr = pc[k];
                if (zb || gx == 0 || gx == nx - 1 || gy == 0 || gy == ny - 1) {
                    if (NLSE_IDX(io.flag, gz * plane + (int64_t)gy * nx + gx, plane * nz, kSiteStage3d)) {
                        const R vb = io.V[gz * plane + (int64_t)gy * nx + gx];
                        d = SC ? cscale(-nonlin(c.s, ctr, vb), ctr) : dirichlet_D(c, ctr, vb);
                    }
                } else {
                    C sum = cadd(q, cadd(pp[k], pm[k]));
                    d = cscale(wd, csub(sum, cscale((R)6, ctr)));
                }
            }
            dst[i] = d;
        }
    };

    for (int gz = z0 - 2; gz <= z0; ++gz) load_plane(gz);
    __syncthreads();
    d_plane(z0 - 1);
    __syncthreads();
    load_plane(z0 + 1);                       // into the slot of plane z0 - 2
    __syncthreads();
    d_plane(z0);
    __syncthreads();

    bool bad = false;
    for (int gz = z0; gz < z1; ++gz) {
        load_plane(gz + 2);                   // into the slot of plane gz - 1
        __syncthreads();
        d_plane(gz + 1);
        __syncthreads();

        const C* pc = sP + dslot(gz) * PP;    // step 2 reads input plane gz only
        const C* hc = sH + ((gz + 2) & 1) * (TX * (TY + 2));
        const C* dm = sD + dslot(gz - 1) * DP;
        const C* dc = sD + dslot(gz) * DP;
        const C* dp = sD + dslot(gz + 1) * DP;
        const C* qm = sQ + dslot(gz - 1) * (TX * TY);
        const C* qp = sQ + dslot(gz + 1) * (TX * TY);
        const bool zb = gz == 0 || gz == nz - 1;
        for (int i = tid; i < TX * TY; i += NT) {
            int ly = i / TX, lx = i - ly * TX;
            int gx = x0 + lx, gy = y0 + ly;
            if (gx >= nx || gy >= ny) continue;
            const int64_t p = gz * plane + (int64_t)gy * nx + gx;
            const int k = (ly + 2) * PX + (lx + 2);
            const int kd = (ly + 1) * DX + (lx + 1);
            if (!(NLSE_IDX(io.flag, k - PX - 1, PP, kSiteStage3d) && NLSE_IDX(io.flag, k + PX + 1, PP, kSiteStage3d) &&
                  NLSE_IDX(io.flag, kd - DX, DP, kSiteStage3d) && NLSE_IDX(io.flag, kd + DX, DP, kSiteStage3d) &&
                  NLSE_IDX(io.flag, (ly + 2) * TX + lx, TX * (TY + 2), kSiteStage3d) &&
                  NLSE_IDX(io.flag, p, plane * nz, kSiteStage3d)))
                continue;
            const C y = pc[k];
            const bool bnd = zb || gx == 0 || gx == nx - 1 || gy == 0 || gy == ny - 1;
            C lap;
            if (bnd || CD) {
                lap = dc[kd];
            } else {
                C dsum = cadd(cadd(cadd(dc[kd + 1], dc[kd - 1]), cadd(dc[kd + DX], dc[kd - DX])),
                              cadd(dp[kd], dm[kd]));
                // the twelve edge neighbours, from the sums step 1 kept: the four
                // in-plane diagonals as hx(y+1) + hx(y-1), and the in-plane axial
                // sums of planes z -+ 1
                C exy = cadd(hc[(ly + 2) * TX + lx], hc[ly * TX + lx]);
                C edges = cadd(exy, cadd(qm[i], qp[i]));
                C dpart = cscale((R)(-1.0 / 12.0), csub(dsum, cscale((R)10, dc[kd])));
                C ppart = cscale(we, csub(edges, cscale((R)12, y)));
                lap = cadd(dpart, ppart);
            }
            if constexpr (STAGE == 0) {
                io.lap[p] = lap;
            } else {
                C F = czero<C>();
                if (!bnd) {
                    if constexpr (SC) {
                        const R N = nonlin(c.s, y, io.V[p]);           // F = i [a Lap + N y]
                        F = ctimesi(cmake<C>(lap.x + N * y.x, lap.y + N * y.y));
                    } else {
                        F = rhs_point(c, y, lap, io.V[p]);
                    }
                }
                bad |= stage_epilogue<STAGE>(io, p, y, F);
            }
        }
        __syncthreads();
    }
    if constexpr (STAGE == 4) {
        if (__syncthreads_or(bad) && tid == 0) atomicOr(io.flag, 1);
    }
}

// The multi-storage form, Eqs. (3d2shocMs1) and (3d2shocMs2), on the same
// 2.5D walk.  Per plane z: D^x and D^y of plane z on the tile plus a 1-point
// ring (one shared buffer each); D^z of this thread's two points of plane
// z+1 (registers, with those of z and z-1 kept from earlier planes);
//     Lap = (7/6)(D^x + D^y + D^z)_c - (1/12)(D^x_E + D^x_W + D^y_N + D^y_S
//                                             + D^z_{z+1} + D^z_{z-1}).
// At a point on the boundary of one axis only, that axis' D^a is D_b of
// Eq. (dbc_lap) minus the other axes' second differences; points on two or
// more boundaries take 0 (never used).
template <typename R, int STAGE>
__global__ void __launch_bounds__(NT)
stage3d_ms_kernel(StageIO<R> io, Coef<R> c, int nx, int ny, int nz) {
    using C = cplx<R>;
    constexpr int PPT = TX * TY / NT;         // points per thread (2)
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* sP = reinterpret_cast<C*>(smem_raw);   // [4][PY][PX]
    C* sDx = sP + 4 * PP;                     // [DY][DX]
    C* sDy = sDx + DP;                        // [DY][DX]

    const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY, z0 = blockIdx.z * TZ;
    const int z1 = min(z0 + TZ, nz);
    const int tid = threadIdx.x;
    const int64_t plane = (int64_t)nx * ny;
    if constexpr (STAGE == 4) {
        if (refused(io.flag)) return;
    }

    auto load_plane = [&](int gz) {
        C* dst = sP + pslot(gz) * PP;
        const bool zin = gz >= 0 && gz < nz;
        for (int i = tid; i < PP; i += NT) {
            int ly = i / PX, lx = i - ly * PX;
            int gx = x0 - 2 + lx, gy = y0 - 2 + ly;
            C v = czero<C>();
            if (zin && gx >= 0 && gx < nx && gy >= 0 && gy < ny)
                v = io.yin[gz * plane + (int64_t)gy * nx + gx];
            dst[i] = v;
        }
    };
    auto d2 = [&](C m, C ctr, C p) { return cscale(c.inv_h2, csub(cadd(m, p), cscale((R)2, ctr))); };
    // (D^x, D^y, D^z) at a grid point from its seven stencil values (k: index
    // in the input planes pm / pc / pp), with the boundary split.
    struct D3 { C x, y, z; };
    auto ms_point = [&](int gx, int gy, int gz, const C* pm, const C* pc, const C* pp, int k) -> D3 {
        const C zero = czero<C>();
        if (gz < 0 || gz >= nz || gx < 0 || gx >= nx || gy < 0 || gy >= ny) return {zero, zero, zero};
        const C ctr = pc[k];
        D3 d{d2(pc[k - 1], ctr, pc[k + 1]), d2(pc[k - PX], ctr, pc[k + PX]), d2(pm[k], ctr, pp[k])};
        const bool bx = gx == 0 || gx == nx - 1, by = gy == 0 || gy == ny - 1, bz = gz == 0 || gz == nz - 1;
        const int nb = (int)bx + (int)by + (int)bz;
        if (nb) {
            const C lb = dirichlet_D(c, ctr, io.V[gz * plane + (int64_t)gy * nx + gx]);
            if (nb > 1) d = {zero, zero, zero};
            else if (bx) d.x = csub(csub(lb, d.y), d.z);
            else if (by) d.y = csub(csub(lb, d.x), d.z);
            else d.z = csub(csub(lb, d.x), d.y);
        }
        return d;
    };
    auto on_bnd = [&](int gx, int gy, int gz) {
        return gx == 0 || gx == nx - 1 || gy == 0 || gy == ny - 1 || gz == 0 || gz == nz - 1;
    };
    // D^z of this thread's m-th point at plane gz (input planes gz-1 .. gz+1
    // loaded): the z difference alone, except at the boundary.
    auto dz_own = [&](int m, int gz) -> C {
        const int i = tid + m * NT, ly = i / TX, lx = i - ly * TX;
        const int k = (ly + 2) * PX + (lx + 2);
        const int gx = x0 + lx, gy = y0 + ly;
        if (gx >= nx || gy >= ny || gz < 0 || gz >= nz) return czero<C>();
        const C* pm = sP + pslot(gz - 1) * PP;
        const C* pc = sP + pslot(gz) * PP;
        const C* pp = sP + pslot(gz + 1) * PP;
        if (on_bnd(gx, gy, gz)) return ms_point(gx, gy, gz, pm, pc, pp, k).z;
        return d2(pm[k], pc[k], pp[k]);
    };

    for (int gz = z0 - 2; gz <= z0 + 1; ++gz) load_plane(gz);
    __syncthreads();
    C dzm[PPT], dz0[PPT];
#pragma unroll
    for (int m = 0; m < PPT; ++m) {
        dzm[m] = dz_own(m, z0 - 1);
        dz0[m] = dz_own(m, z0);
    }
    __syncthreads();                          // plane z0-2 is read above and overwritten below

    bool bad = false;
    for (int gz = z0; gz < z1; ++gz) {
        load_plane(gz + 2);
        // D^x, D^y of plane gz on the tile plus a 1-point ring.
        {
            const C* pm = sP + pslot(gz - 1) * PP;
            const C* pc = sP + pslot(gz) * PP;
            const C* pp = sP + pslot(gz + 1) * PP;
            for (int i = tid; i < DP; i += NT) {
                const int ly = i / DX, lx = i - ly * DX;
                const int gx = x0 - 1 + lx, gy = y0 - 1 + ly, k = (ly + 1) * PX + (lx + 1);
                C dx = czero<C>(), dy = czero<C>();
                if (gx < 0 || gx >= nx || gy < 0 || gy >= ny) {
                } else if (on_bnd(gx, gy, gz)) {
                    const D3 d = ms_point(gx, gy, gz, pm, pc, pp, k);
                    dx = d.x;
                    dy = d.y;
                } else {
                    dx = d2(pc[k - 1], pc[k], pc[k + 1]);
                    dy = d2(pc[k - PX], pc[k], pc[k + PX]);
                }
                sDx[i] = dx;
                sDy[i] = dy;
            }
        }
        __syncthreads();
        const C* pc = sP + pslot(gz) * PP;
        const bool zb = gz == 0 || gz == nz - 1;
#pragma unroll
        for (int m = 0; m < PPT; ++m) {
            const int i = tid + m * NT, ly = i / TX, lx = i - ly * TX;
            const int gx = x0 + lx, gy = y0 + ly;
            const C dz1 = dz_own(m, gz + 1);
            if (gx < nx && gy < ny &&
                NLSE_IDX(io.flag, gz * plane + (int64_t)gy * nx + gx, plane * nz, kSiteStage3d) &&
                NLSE_IDX(io.flag, (ly + 1) * DX + lx + 1 + DX, DP, kSiteStage3d) &&
                NLSE_IDX(io.flag, (ly + 2) * PX + lx + 2, PP, kSiteStage3d)) {
                const int64_t p = gz * plane + (int64_t)gy * nx + gx;
                const int k = (ly + 2) * PX + (lx + 2);
                const int kd = (ly + 1) * DX + (lx + 1);
                const C y = pc[k];
                const bool bnd = zb || gx == 0 || gx == nx - 1 || gy == 0 || gy == ny - 1;
                C lap;
                if (bnd) {
                    lap = dirichlet_D(c, y, io.V[p]);
                } else {
                    const C nbs = cadd(cadd(cadd(sDx[kd - 1], sDx[kd + 1]), cadd(sDy[kd - DX], sDy[kd + DX])),
                                       cadd(dzm[m], dz1));
                    const C ctr = cadd(cadd(sDx[kd], sDy[kd]), dz0[m]);
                    lap = csub(cscale((R)(7.0 / 6.0), ctr), cscale((R)(1.0 / 12.0), nbs));
                }
                if constexpr (STAGE == 0) {
                    io.lap[p] = lap;
                } else {
                    C F = bnd ? czero<C>() : rhs_point(c, y, lap, io.V[p]);
                    bad |= stage_epilogue<STAGE>(io, p, y, F);
                }
            }
            dzm[m] = dz0[m];
            dz0[m] = dz1;
        }
        __syncthreads();
    }
    if constexpr (STAGE == 4) {
        if (__syncthreads_or(bad) && tid == 0) atomicOr(io.flag, 1);
    }
}

template <typename R, int STAGE>
cudaError_t launch_ms(const StageLaunch& L, cudaStream_t st) {
    const int nx = (int)L.n[0], ny = (int)L.n[1], nz = (int)L.n[2];
    dim3 grid((nx + TX - 1) / TX, (ny + TY - 1) / TY, (nz + TZ - 1) / TZ);
    size_t smem = sizeof(cplx<R>) * (4 * PP + 2 * DP);
    auto kern = stage3d_ms_kernel<R, STAGE>;
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    kern<<<grid, NT, smem, st>>>(make_io<R>(L), make_coef<R>(L.h, L.a, L.s), nx, ny, nz);
    return cudaGetLastError();
}

template <typename R, bool CD, int STAGE>
cudaError_t launch_t(const StageLaunch& L, cudaStream_t st) {
    if (!CD && L.lap == 2) return launch_ms<R, STAGE>(L, st);
    const int nx = (int)L.n[0], ny = (int)L.n[1], nz = (int)L.n[2];
    dim3 grid((nx + TX - 1) / TX, (ny + TY - 1) / TY, (nz + TZ - 1) / TZ);
    size_t smem = sizeof(cplx<R>) * (3 * PP + 3 * DP + 3 * TX * TY + 2 * TX * (TY + 2));
    auto kern = stage3d_kernel<R, CD, STAGE>;
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    kern<<<grid, NT, smem, st>>>(make_io<R>(L), make_coef<R>(L.h, L.a, L.s), nx, ny, nz);
    return cudaGetLastError();
}

template <typename R, bool CD>
cudaError_t launch_stage(const StageLaunch& L, cudaStream_t st) {
    switch (L.stage) {
        case 0: return launch_t<R, CD, 0>(L, st);
        case 1: return launch_t<R, CD, 1>(L, st);
        case 2: return launch_t<R, CD, 2>(L, st);
        case 3: return launch_t<R, CD, 3>(L, st);
        case 4: return launch_t<R, CD, 4>(L, st);
    }
    return cudaErrorInvalidValue;
}

}  // namespace

// FP32 Dirichlet grids whose rows TMA can address (nx a multiple of 4) and
// 16-byte aligned buffers; other 3D grids use the generic kernel.
bool stage_3d_tma_eligible(const StageLaunch& L) {
    if (L.prec != 0 || L.bc != 0 || L.n[0] % 4 != 0) return false;
    const void* ptrs[8] = {L.yin, L.V, L.psi, L.psi_out, L.acc, L.lo, L.yout, L.lap_out};
    for (const void* p : ptrs)
        if ((uintptr_t)p % 16) return false;
    return encoder() != nullptr;
}

cudaError_t launch_stage_3d_tma(const StageLaunch& L, cudaStream_t st) {
    switch (L.tile_planes) {
        case 64: return launch_stage_3d_tma_planes64(L, st);
        case 128: return launch_stage_3d_tma_planes128(L, st);
        default: return launch_stage_3d_tma_planes32(L, st);
    }
}

cudaError_t launch_stage_3d(const StageLaunch& L, cudaStream_t st) {
    if (stage_3d_tma_eligible(L)) return launch_stage_3d_tma(L, st);
    const bool cd = L.lap == 1;
    if (L.prec == 0) return cd ? launch_stage<float, true>(L, st) : launch_stage<float, false>(L, st);
    return cd ? launch_stage<double, true>(L, st) : launch_stage<double, false>(L, st);
}

}  // namespace nlse
