// stage2d.cu -- fused RK4 stage and standalone 2SHOC Laplacian on a 2D grid,
// generic tile kernel for grids whose rows TMA cannot address (row pitch not
// a multiple of 16 bytes); the TMA-fed kernel in stage2d_tma.cu serves the rest.
//
// One CTA owns a TX x TY tile of output points.  It stages the stage input
// with a 2-point halo in shared memory, computes step 1 of the 2SHOC scheme,
// the second-order D of Eq. (2d2shocs1), on the tile plus a 1-point ring
// (boundary points take D_b of Eq. (dbc_lap)), and then step 2,
// Eq. (2d2shocs2):
//     Lap = -(1/12)[D_E + D_W + D_N + D_S - 12 D_c]
//           + (1/(6h^2))[Psi_NE + Psi_NW + Psi_SE + Psi_SW - 4 Psi_c],
// followed by F (Sec. 3.1), the Dirichlet rule F_b = 0 (Eq. dbc_ut) and the
// stage epilogue.  D lives only in shared memory.  The multi-storage form
// (LP = 2) keeps D^x and D^y apart, Eq. (2d2shocMs1), with the Dirichlet
// split of D_b at points on the boundary of one axis (D^a_b = D_b minus the
// other axis' second difference), and takes step 2 from Eq. (2d2shocMs2):
//     Lap = (7/6)(D^x_c + D^y_c) - (1/12)(D^x_E + D^x_W + D^y_N + D^y_S).
#include "nlse_device.cuh"
#include "tmap.cuh"

namespace nlse {
namespace {

constexpr int TX = 64;       // tile width (x, contiguous)
constexpr int TY = 16;       // tile height
constexpr int NT = 256;      // threads per CTA
constexpr int PX = TX + 4, PY = TY + 4;   // stage input with a 2-point halo
constexpr int DX = TX + 2, DY = TY + 2;   // D with a 1-point halo

// STAGE 0 writes the Laplacian (boundary = D_b); STAGE 1..4 are RK4 stages.
// LP: 0 single-storage 2SHOC, 1 CD, 2 multi-storage 2SHOC.
template <typename R, int LP, int STAGE>
__global__ void __launch_bounds__(NT)
stage2d_kernel(StageIO<R> io, Coef<R> c, int nx, int ny) {
    using C = cplx<R>;
    constexpr bool CD = LP == 1, MS = LP == 2;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* sP = reinterpret_cast<C*>(smem_raw);          // [PY][PX]
    C* sD = sP + PX * PY;                            // [DY][DX]; multi storage: D^x
    C* sDy = sD + DX * DY;                           // multi storage: D^y [DY][DX]

    const int x0 = blockIdx.x * TX;
    const int y0 = blockIdx.y * TY;
    const int tid = threadIdx.x;
    if constexpr (STAGE == 4) {
        if (refused(io.flag)) return;
    }

    // Stage input tile with halo; points outside the grid read as zero (never used).
    for (int i = tid; i < PX * PY; i += NT) {
        int ly = i / PX, lx = i - ly * PX;
        int gx = x0 - 2 + lx, gy = y0 - 2 + ly;
        C v = czero<C>();
        if (gx >= 0 && gx < nx && gy >= 0 && gy < ny) v = io.yin[(int64_t)gy * nx + gx];
        sP[i] = v;
    }
    __syncthreads();

    // Step 1: D on the tile plus a 1-point ring.
    for (int i = tid; i < DX * DY; i += NT) {
        int ly = i / DX, lx = i - ly * DX;
        int gx = x0 - 1 + lx, gy = y0 - 1 + ly;
        const C* q = sP + (ly + 1) * PX + (lx + 1);
        // (the five-point window q -+ 1, q -+ PX inside the staged tile)
        if (!(NLSE_IDX(io.flag, (ly + 1) * PX + lx + 1 - PX, PX * PY, kSiteStage2d) &&
              NLSE_IDX(io.flag, (ly + 1) * PX + lx + 1 + PX, PX * PY, kSiteStage2d)))
            continue;
        C d = czero<C>();
        if constexpr (MS) {
            C dx = czero<C>(), dy = czero<C>();
            if (gx >= 0 && gx < nx && gy >= 0 && gy < ny) {
                const C pc = q[0];
                dx = cscale(c.inv_h2, csub(cadd(q[-1], q[1]), cscale((R)2, pc)));
                dy = cscale(c.inv_h2, csub(cadd(q[-PX], q[PX]), cscale((R)2, pc)));
                const int gyl = inst_row(gy, io.rows1);
                const bool bx = gx == 0 || gx == nx - 1, by = gyl == 0 || gyl == io.rows1 - 1;
                if ((bx || by) && NLSE_IDX(io.flag, (int64_t)gyl * nx + gx, (int64_t)io.rows1 * nx, kSiteStage2d)) {
                    const C lb = dirichlet_D(c, pc, io.V[(int64_t)gyl * nx + gx]);
                    if (bx && by) dx = dy = czero<C>();
                    else if (bx) dx = csub(lb, dy);
                    else dy = csub(lb, dx);
                }
            }
            sD[i] = dx;
            sDy[i] = dy;
            continue;
        }
        if (gx >= 0 && gx < nx && gy >= 0 && gy < ny) {
            C pc = q[0];
            const int gyl = inst_row(gy, io.rows1);
            if (gx == 0 || gx == nx - 1 || gyl == 0 || gyl == io.rows1 - 1) {
                if (NLSE_IDX(io.flag, (int64_t)gyl * nx + gx, (int64_t)io.rows1 * nx, kSiteStage2d))
                    d = dirichlet_D(c, pc, io.V[(int64_t)gyl * nx + gx]);
            } else {
                C sum = cadd(cadd(q[1], q[-1]), cadd(q[PX], q[-PX]));
                d = cscale(c.inv_h2, csub(sum, cscale((R)4, pc)));
            }
        }
        sD[i] = d;
    }
    __syncthreads();

    // Step 2, F and the stage epilogue on the tile.
    bool bad = false;
    for (int i = tid; i < TX * TY; i += NT) {
        int ly = i / TX, lx = i - ly * TX;
        int gx = x0 + lx, gy = y0 + ly;
        if (gx >= nx || gy >= ny) continue;
        const int64_t p = (int64_t)gy * nx + gx;
        const C* q = sP + (ly + 2) * PX + (lx + 2);
        const C* e = sD + (ly + 1) * DX + (lx + 1);
        const C y = q[0];
        const int gyl = inst_row(gy, io.rows1);
        const int64_t pv = (int64_t)gyl * nx + gx;     // V is shared by stacked instances
        // (the windows in the staged tile and in D, the output and V indices)
        if (!(NLSE_IDX(io.flag, (ly + 2) * PX + lx + 2 - PX - 1, PX * PY, kSiteStage2d) &&
              NLSE_IDX(io.flag, (ly + 2) * PX + lx + 2 + PX + 1, PX * PY, kSiteStage2d) &&
              NLSE_IDX(io.flag, (ly + 1) * DX + lx + 1 - DX, DX * DY, kSiteStage2d) &&
              NLSE_IDX(io.flag, (ly + 1) * DX + lx + 1 + DX, DX * DY, kSiteStage2d) &&
              NLSE_IDX(io.flag, p, (int64_t)nx * ny, kSiteStage2d) &&
              NLSE_IDX(io.flag, pv, (int64_t)io.rows1 * nx, kSiteStage2d)))
            continue;
        const bool bnd = (gx == 0 || gx == nx - 1 || gyl == 0 || gyl == io.rows1 - 1);
        C lap;
        if (MS) {
            const C* ey = sDy + (ly + 1) * DX + (lx + 1);
            if (bnd) {
                lap = dirichlet_D(c, y, io.V[pv]);
            } else {
                const C nb = cadd(cadd(e[-1], e[1]), cadd(ey[-DX], ey[DX]));
                lap = csub(cscale((R)(7.0 / 6.0), cadd(e[0], ey[0])), cscale((R)(1.0 / 12.0), nb));
            }
        } else if (bnd || CD) {
            lap = e[0];
        } else {
            C dsum = cadd(cadd(e[1], e[-1]), cadd(e[DX], e[-DX]));
            C corners = cadd(cadd(q[PX + 1], q[PX - 1]), cadd(q[-PX + 1], q[-PX - 1]));
            C dpart = cscale((R)(-1.0 / 12.0), csub(dsum, cscale((R)12, e[0])));
            C ppart = cscale(c.inv_6h2, csub(corners, cscale((R)4, y)));
            lap = cadd(dpart, ppart);
        }
        if constexpr (STAGE == 0) {
            io.lap[p] = lap;
        } else {
            C F = bnd ? czero<C>() : rhs_point(c, y, lap, io.V[pv]);
            bad |= stage_epilogue<STAGE>(io, p, y, F);
        }
    }
    if constexpr (STAGE == 4) {
        if (__syncthreads_or(bad) && tid == 0) atomicOr(io.flag, 1);
    }
}

template <typename R, int LP, int STAGE>
cudaError_t launch_t(const StageLaunch& L, cudaStream_t st) {
    const int nx = (int)L.n[0], ny = (int)L.n[1];
    dim3 grid((nx + TX - 1) / TX, (ny + TY - 1) / TY);
    size_t smem = sizeof(cplx<R>) * (PX * PY + (LP == 2 ? 2 : 1) * DX * DY);
    auto kern = stage2d_kernel<R, LP, STAGE>;
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    kern<<<grid, NT, smem, st>>>(make_io<R>(L), make_coef<R>(L.h, L.a, L.s), nx, ny);
    return cudaGetLastError();
}

template <typename R, int LP>
cudaError_t launch_stage(const StageLaunch& L, cudaStream_t st) {
    switch (L.stage) {
        case 0: return launch_t<R, LP, 0>(L, st);
        case 1: return launch_t<R, LP, 1>(L, st);
        case 2: return launch_t<R, LP, 2>(L, st);
        case 3: return launch_t<R, LP, 3>(L, st);
        case 4: return launch_t<R, LP, 4>(L, st);
    }
    return cudaErrorInvalidValue;
}

template <typename R>
cudaError_t launch_lap(const StageLaunch& L, cudaStream_t st) {
    switch (L.lap) {
        case 0: return launch_stage<R, 0>(L, st);
        case 1: return launch_stage<R, 1>(L, st);
        case 2: return launch_stage<R, 2>(L, st);
    }
    return cudaErrorInvalidValue;
}

}  // namespace

bool keep_v_in_l2(size_t v_bytes) {
    static int l2 = -1;
    if (l2 < 0) {
        int dev = 0, bytes = 0;
        if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&bytes, cudaDevAttrL2CacheSize, dev) != cudaSuccess)
            bytes = 0;
        l2 = bytes;
    }
    return v_bytes <= (size_t)l2 / 4;
}

// TMA needs 16-byte aligned bases and row pitches: nx a multiple of 4
// (complex64 rows and float V rows) or of 2 (complex128 rows, double V).
// The column pairs also need nx even.
bool stage_2d_tma_eligible(const StageLaunch& L) {
    if (L.bc != 0) return false;
    const int64_t nx = L.n[0];
    if (nx % (L.prec == 0 ? 4 : 2) != 0) return false;
    const void* ptrs[8] = {L.yin, L.V, L.psi, L.psi_out, L.acc, L.lo, L.yout, L.lap_out};
    for (const void* p : ptrs)
        if ((uintptr_t)p % 16) return false;
    return encoder() != nullptr;
}

cudaError_t launch_stage_2d_tma(const StageLaunch& L, cudaStream_t st) {
    switch (L.tile_rows) {
        case 8: return launch_stage_2d_tma_rows8(L, st);
        case 32: return launch_stage_2d_tma_rows32(L, st);
        default: return launch_stage_2d_tma_rows16(L, st);
    }
}

cudaError_t launch_stage_2d(const StageLaunch& L, cudaStream_t st) {
    if (stage_2d_tma_eligible(L)) return launch_stage_2d_tma(L, st);
    return L.prec == 0 ? launch_lap<float>(L, st) : launch_lap<double>(L, st);
}

}  // namespace nlse
