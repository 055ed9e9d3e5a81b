// stage2d_tma.cu -- the fused 2D RK4 stage (and standalone 2SHOC Laplacian)
// as a y-streaming kernel fed by the tensor memory accelerator.
//
// One CTA of TX threads owns TX consecutive columns and walks down TY rows.
// A ring of S row slots in shared memory is filled by TMA tile loads (one
// mbarrier per slot), S rows ahead of use:
//   * the stage input row with a 2-point x halo,
//   * the potential V row (x halo 4, for the boundary rule),
//   * on output rows: Psi^n, the accumulator and (stage 4, FP32) the
//     compensated low part.
// Each thread keeps its column's stage input and D in registers as a sliding
// window; only the x neighbours of D travel through a two-row shared ring.
// Per output row y, with D(x, y+1) computed one row ahead:
//   step 1 (Eq. 2d2shocs1): D = (sum of the four axial Psi - 4 Psi_c) / h^2,
//                           boundary points D_b of Eq. (dbc_lap);
//   step 2 (Eq. 2d2shocs2): Lap = D_c - (1/12) sum of the four axial D
//                           + (1/(6h^2)) (four corner Psi - 4 Psi_c);
//   F = i[a Lap + (s|Psi|^2 - V) Psi] (Sec. 3.1), F_b = 0 (Eq. dbc_ut);
//   the RK4 stage epilogue (Eq. RK4, accumulated-increment form).
// Complex64 arithmetic uses the packed f32x2 instructions.  Every mbarrier
// wait is bounded (1 s); on timeout the CTA sets bit 2 of the status flag,
// drains its own copies in flight and returns.
#include <mutex>

#include "nlse_device.cuh"
#include "tma.cuh"

namespace nlse {
namespace {

constexpr int TX = 128;              // columns per CTA (= threads)
constexpr int TY = 32;               // rows per CTA
constexpr int S = 6;                 // row slots in flight
constexpr uint64_t kWaitNs = 1000000000ull;
constexpr uint64_t kDrainNs = 50000000ull;

constexpr int al128(int v) { return (v + 127) / 128 * 128; }

template <typename R>
struct Lay {
    static constexpr int CB = (int)sizeof(cplx<R>);
    static constexpr int P_BYTES = (TX + 4) * CB;            // stage input row, x0-2 .. x0+TX+1
    static constexpr int V_BYTES = (TX + 8) * (int)sizeof(R);  // V row, x0-4 .. x0+TX+3
    static constexpr int T_BYTES = TX * CB;                  // Psi^n / acc / lo rows, x0 .. x0+TX-1
    static constexpr int P_OFF = 0;
    static constexpr int V_OFF = al128(P_BYTES);
    static constexpr int PSI_OFF = V_OFF + al128(V_BYTES);
    static constexpr int ACC_OFF = PSI_OFF + T_BYTES;
    static constexpr int LO_OFF = ACC_OFF + T_BYTES;
    static constexpr int SLOT = LO_OFF + (sizeof(R) == 4 ? T_BYTES : 0);
    static constexpr int D_ROW = TX + 2;                     // D row, x0-1 .. x0+TX
    static constexpr int D_OFF = S * SLOT;
    static constexpr int BAR_OFF = al128(D_OFF + 2 * D_ROW * CB);
    static constexpr int TOTAL = BAR_OFF + 8 * S + 128;      // +128: base alignment slack
};

template <typename R>
__device__ __forceinline__ void load_cplx_row(uint32_t dst, const CUtensorMap* m, int x, int r, uint32_t bar) {
    if constexpr (sizeof(R) == 4) tma_load_2d(dst, m, x, r, bar);       // complex64 as 8-byte elements
    else tma_load_3d(dst, m, 0, x, r, bar);                             // complex128 as (re, im) doubles
}

template <typename C> __device__ __forceinline__ C pair(decltype(C::x) a, decltype(C::x) b) {
    C z; z.x = a; z.y = b; return z;
}

template <typename R, bool CD, int STAGE>
__global__ void __launch_bounds__(TX)
stage2d_tma_kernel(const __grid_constant__ CUtensorMap m_in, const __grid_constant__ CUtensorMap m_V,
                   const __grid_constant__ CUtensorMap m_psi, const __grid_constant__ CUtensorMap m_acc,
                   const __grid_constant__ CUtensorMap m_lo, const StageIO<R> io, const Coef<R> c,
                   const int nx, const int ny) {
    using C = cplx<R>;
    using L = Lay<R>;
    constexpr bool NEED_PA = STAGE >= 2;
    constexpr bool NEED_LO = STAGE == 4 && sizeof(R) == 4;
    extern __shared__ unsigned char smem_raw[];
    unsigned char* smem = smem_raw + ((128 - (smem_u32(smem_raw) & 127)) & 127);

    const int tx = threadIdx.x;
    const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY;
    const int nrows = min(TY, ny - y0);
    const int jmax = nrows + 4;                 // rows j = 0 .. jmax-1 are y0-2 .. y0+nrows+1
    const uint32_t sbase = smem_u32(smem);
    const uint32_t bar0 = sbase + L::BAR_OFF;

    if (tx == 0) {
        tma_prefetch_desc(&m_in);
        tma_prefetch_desc(&m_V);
        for (int s = 0; s < S; ++s) mbar_init(bar0 + 8 * s, 1);
        mbar_init_fence();
    }
    __syncthreads();

    auto issue = [&](int j) {
        const int s = j % S;
        const uint32_t slot = sbase + s * L::SLOT;
        const uint32_t bar = bar0 + 8 * s;
        const int r = y0 - 2 + j;
        const bool outrow = j >= 2 && j < nrows + 2;
        uint32_t bytes = L::P_BYTES + L::V_BYTES;
        if (NEED_PA && outrow) bytes += 2 * L::T_BYTES;
        if (NEED_LO && outrow) bytes += L::T_BYTES;
        mbar_expect_tx(bar, bytes);
        load_cplx_row<R>(slot + L::P_OFF, &m_in, x0 - 2, r, bar);
        tma_load_2d(slot + L::V_OFF, &m_V, x0 - 4, r, bar);
        if (NEED_PA && outrow) {
            load_cplx_row<R>(slot + L::PSI_OFF, &m_psi, x0, r, bar);
            load_cplx_row<R>(slot + L::ACC_OFF, &m_acc, x0, r, bar);
        }
        if (NEED_LO && outrow) load_cplx_row<R>(slot + L::LO_OFF, &m_lo, x0, r, bar);
    };
    int next = 0;                                // rows issued so far (thread 0)
    if (tx == 0)
        for (; next < S && next < jmax; ++next) issue(next);

    auto prow = [&](int j) { return reinterpret_cast<const C*>(smem + (j % S) * L::SLOT + L::P_OFF); };
    auto vrow = [&](int j) { return reinterpret_cast<const R*>(smem + (j % S) * L::SLOT + L::V_OFF); };
    auto trow = [&](int j, int off) { return reinterpret_cast<const C*>(smem + (j % S) * L::SLOT + off); };
    C* dring = reinterpret_cast<C*>(smem + L::D_OFF);

    bool ok = true;
    auto wait_row = [&](int j) {
        if (ok) ok = mbar_wait(bar0 + 8 * (j % S), (uint32_t)((j / S) & 1), kWaitNs);
    };

    const C m4 = pair<C>(-4, -4), m12 = pair<C>(R(-1.0 / 12.0), R(-1.0 / 12.0));
    const C ih2 = pair<C>(c.inv_h2, c.inv_h2), i6h2 = pair<C>(c.inv_6h2, c.inv_6h2);
    const C a2 = pair<C>(c.a, c.a);
    const C ca2 = pair<C>(-io.c_acc, io.c_acc), cy2 = pair<C>(-io.c_y, io.c_y);

    // D at an arbitrary grid point (x, r) from its five stencil values; used
    // for the two halo columns x0-1 and x0+TX.
    auto halo_d = [&](int x, int r, C ctr, C up, C dn, C lf, C rt) -> C {
        if (x < 0 || x >= nx || r < 0 || r >= ny) return czero<C>();
        if (x == 0 || x == nx - 1 || r == 0 || r == ny - 1)
            return dirichlet_D(c, ctr, io.V[(int64_t)r * nx + x]);
        return mul2(fma2(m4, ctr, add2(add2(lf, rt), add2(up, dn))), ih2);
    };

    const int gx = x0 + tx;
    const int k = tx + 2;                        // this column in the row buffers
    const bool xin = gx < nx;
    const bool xb = gx == 0 || gx == nx - 1;
    // D at (gx, r) from the register window (cm, cc, cp: rows r-1, r, r+1; cl, cr: x neighbours).
    auto d_reg = [&](int r, int j, C cm, C cc, C cp, C cl, C cr) -> C {
        if (!xin || r < 0 || r >= ny) return czero<C>();
        if (xb || r == 0 || r == ny - 1) return dirichlet_D(c, cc, vrow(j)[tx + 4]);
        return mul2(fma2(m4, cc, add2(add2(cl, cr), add2(cm, cp))), ih2);
    };

    // Prologue: rows y0-2 .. y0+1 give D(y0-1) (registers) and D(y0) (registers + ring).
    wait_row(0); wait_row(1); wait_row(2); wait_row(3);
    bool alive = __syncthreads_and(ok);
    C lm, rm, l0, r0, c0, c1, dm, d0;
    if (alive) {
        lm = prow(1)[k - 1]; rm = prow(1)[k + 1];
        l0 = prow(2)[k - 1]; r0 = prow(2)[k + 1];
        const C cm = prow(1)[k];
        c0 = prow(2)[k];
        c1 = prow(3)[k];
        dm = d_reg(y0 - 1, 1, prow(0)[k], cm, c0, lm, rm);
        d0 = d_reg(y0, 2, cm, c0, c1, l0, r0);
        dring[tx + 1] = d0;                                  // row j = 2 -> ring row 0
        if (tx == 0) dring[0] = halo_d(x0 - 1, y0, l0, lm, prow(3)[1], prow(2)[0], c0);
        if (tx == TX - 1) dring[TX + 1] = halo_d(x0 + TX, y0, r0, rm, prow(3)[TX + 2], c0, prow(2)[TX + 3]);
    }
    __syncthreads();

    bool bad = false;
    for (int i = 0; alive && i < nrows; ++i) {
        const int j = i + 2;                                 // buffer row of y
        const int y = y0 + i;
        wait_row(j + 2);
        if (!__syncthreads_and(ok)) { alive = false; break; }
        if (tx == 0 && next < jmax) { issue(next); ++next; }

        // D(gx, y+1), one row ahead.
        const C* p1 = prow(j + 1);
        const C l1 = p1[k - 1], r1 = p1[k + 1];
        const C c2 = prow(j + 2)[k];
        const C d1 = d_reg(y + 1, j + 1, c0, c1, c2, l1, r1);
        C* dnext = dring + ((j + 1) & 1) * L::D_ROW;
        dnext[tx + 1] = d1;
        if (tx == 0) dnext[0] = halo_d(x0 - 1, y + 1, l1, l0, prow(j + 2)[1], p1[0], c1);
        if (tx == TX - 1) dnext[TX + 1] = halo_d(x0 + TX, y + 1, r1, r0, prow(j + 2)[TX + 2], c1, p1[TX + 3]);
        __syncthreads();

        if (xin) {
            const C* dr = dring + (j & 1) * L::D_ROW + tx;   // dr[0] = D(gx-1, y), dr[2] = D(gx+1, y)
            const bool bnd = xb || y == 0 || y == ny - 1;
            C lap = d0;
            if (!CD && !bnd) {
                const C dsum = add2(add2(dr[0], dr[2]), add2(dm, d1));
                const C corners = add2(add2(lm, rm), add2(l1, r1));
                lap = fma2(i6h2, fma2(m4, c0, corners), fma2(m12, dsum, d0));
            }
            const int64_t p = (int64_t)y * nx + gx;
            if constexpr (STAGE == 0) {
                io.lap[p] = lap;
            } else {
                // w = a Lap + (s|Psi|^2 - V) Psi, F = i w; F_b = 0.
                C sw = czero<C>();
                if (!bnd) {
                    const R v = vrow(j)[tx + 4];
                    const R N = c.s * (c0.x * c0.x + c0.y * c0.y) - v;
                    const C w = fma2(pair<C>(N, N), c0, mul2(a2, lap));
                    sw = pair<C>(w.y, w.x);                  // c * F = (-c w.y, c w.x) = (-c, c) * swap(w)
                }
                if constexpr (STAGE == 1) {
                    io.acc[p] = mul2(ca2, sw);
                    io.yout[p] = fma2(cy2, sw, c0);
                } else if constexpr (STAGE == 2 || STAGE == 3) {
                    const C pn = trow(j, L::PSI_OFF)[tx];
                    const C ac = trow(j, L::ACC_OFF)[tx];
                    io.acc[p] = fma2(ca2, sw, ac);
                    io.yout[p] = fma2(cy2, sw, pn);
                } else {
                    C pn = trow(j, L::PSI_OFF)[tx];
                    const C d = fma2(ca2, sw, trow(j, L::ACC_OFF)[tx]);
                    if constexpr (sizeof(R) == 4) {
                        C lo = trow(j, L::LO_OFF)[tx];
                        kahan_add(pn.x, lo.x, d.x);
                        kahan_add(pn.y, lo.y, d.y);
                        io.lo[p] = lo;
                    } else {
                        pn = add2(pn, d);
                    }
                    io.psi_out[p] = pn;
                    bad |= !(isfinite(pn.x) && isfinite(pn.y));
                }
            }
        }
        lm = l0; rm = r0; l0 = l1; r0 = r1;
        c0 = c1; c1 = c2;
        dm = d0; d0 = d1;
    }

    if (!alive) {
        // A row never arrived: report, let this CTA's copies in flight land, leave.
        if (tx == 0) {
            atomicOr(io.flag, 2);
            for (int j = next > S ? next - S : 0; j < next; ++j)
                mbar_wait(bar0 + 8 * (j % S), (uint32_t)((j / S) & 1), kDrainNs);
        }
        return;
    }
    if constexpr (STAGE == 4) {
        if (__syncthreads_or(bad) && tx == 0) atomicOr(io.flag, 1);
    }
}

// ---- host side -------------------------------------------------------------

using EncodeTiled = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                 const cuuint64_t*, const cuuint32_t*, const cuuint32_t*,
                                 CUtensorMapInterleave, CUtensorMapSwizzle, CUtensorMapL2promotion,
                                 CUtensorMapFloatOOBfill);

EncodeTiled encoder() {
    static EncodeTiled fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess && q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiled>(p);
    });
    return fn;
}

bool encode(CUtensorMap* m, CUtensorMapDataType t, int rank, const void* base, const cuuint64_t* dims,
            const cuuint64_t* strides, const cuuint32_t* box) {
    EncodeTiled fn = encoder();
    if (!fn || !base) return false;
    const cuuint32_t ones[3] = {1, 1, 1};
    return fn(m, t, (cuuint32_t)rank, const_cast<void*>(base), dims, strides, box, ones,
              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// A complex row map over an nx x ny grid with boxes `width` points wide.
template <typename R>
bool complex_map(CUtensorMap* m, const void* base, int nx, int ny, int width) {
    if constexpr (sizeof(R) == 4) {
        cuuint64_t dims[2] = {(cuuint64_t)nx, (cuuint64_t)ny};
        cuuint64_t strides[1] = {(cuuint64_t)nx * 8};
        cuuint32_t box[2] = {(cuuint32_t)width, 1};
        return encode(m, CU_TENSOR_MAP_DATA_TYPE_UINT64, 2, base, dims, strides, box);
    } else {
        cuuint64_t dims[3] = {2, (cuuint64_t)nx, (cuuint64_t)ny};
        cuuint64_t strides[2] = {16, (cuuint64_t)nx * 16};
        cuuint32_t box[3] = {2, (cuuint32_t)width, 1};
        return encode(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 3, base, dims, strides, box);
    }
}

template <typename R>
bool real_map(CUtensorMap* m, const void* base, int nx, int ny, int width) {
    cuuint64_t dims[2] = {(cuuint64_t)nx, (cuuint64_t)ny};
    cuuint64_t strides[1] = {(cuuint64_t)nx * sizeof(R)};
    cuuint32_t box[2] = {(cuuint32_t)width, 1};
    return encode(m, sizeof(R) == 4 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 2, base,
                  dims, strides, box);
}

template <typename R, bool CD, int STAGE>
cudaError_t launch_t(const StageLaunch& L, cudaStream_t st) {
    const int nx = (int)L.n[0], ny = (int)L.n[1];
    CUtensorMap m_in, m_V, m_psi, m_acc, m_lo;
    if (!complex_map<R>(&m_in, L.yin, nx, ny, TX + 4) || !real_map<R>(&m_V, L.V, nx, ny, TX + 8))
        return cudaErrorInvalidValue;
    m_psi = m_acc = m_lo = m_in;
    if (STAGE >= 2) {
        if (!complex_map<R>(&m_psi, L.psi, nx, ny, TX) || !complex_map<R>(&m_acc, L.acc, nx, ny, TX))
            return cudaErrorInvalidValue;
    }
    if (STAGE == 4 && sizeof(R) == 4 && !complex_map<R>(&m_lo, L.lo, nx, ny, TX)) return cudaErrorInvalidValue;
    auto kern = stage2d_tma_kernel<R, CD, STAGE>;
    const int smem = Lay<R>::TOTAL;
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (e != cudaSuccess) return e;
    }
    dim3 grid((nx + TX - 1) / TX, (ny + TY - 1) / TY);
    kern<<<grid, TX, smem, st>>>(m_in, m_V, m_psi, m_acc, m_lo, make_io<R>(L), make_coef<R>(L.h, L.a, L.s), nx, ny);
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

// TMA needs 16-byte aligned bases and row pitches: nx a multiple of 4
// (complex64 rows and float V rows) or of 2 (complex128 rows, double V).
bool stage_2d_tma_eligible(const StageLaunch& L) {
    if (L.bc != 0) return false;
    const int64_t nx = L.n[0];
    if (nx % (L.prec == 0 ? 4 : 2) != 0) return false;
    const void* ptrs[6] = {L.yin, L.V, L.psi, L.acc, L.lo, L.yout};
    for (const void* p : ptrs)
        if ((uintptr_t)p % 16) return false;
    return encoder() != nullptr;
}

cudaError_t launch_stage_2d_tma(const StageLaunch& L, cudaStream_t st) {
    const bool cd = L.lap == 1;
    if (L.prec == 0) return cd ? launch_stage<float, true>(L, st) : launch_stage<float, false>(L, st);
    return cd ? launch_stage<double, true>(L, st) : launch_stage<double, false>(L, st);
}

}  // namespace nlse
