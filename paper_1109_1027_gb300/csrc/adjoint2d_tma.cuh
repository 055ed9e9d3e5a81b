// adjoint2d_tma.cuh -- one reversed RK4 stage of the 2D Dirichlet adjoint
// (the operator is derived in adjoint2d.cu) as a y-streaming row walk fed by
// the tensor memory accelerator, the structure of the forward stage walk
// (stage2d_tile.cuh) with the transposed stencil.
//
// One CTA of NT threads owns TXC = 2 NT columns (two per thread) and walks TY
// rows.  Two rings of shared-memory row slots are filled by TMA tile loads,
// each slot completing on its own mbarrier:
//   * the input ring (S slots): the stored cotangent w with a 2-point x halo;
//   * the epilogue ring (2 slots, one output row ahead): Y_j and V on the
//     output row; lam' (stages 3 and 2; stage 4's w is lam' itself) and the
//     running lam (stages 3, 2, 1); for stage 1 also the dL/dV contributions
//     of stages 4, 3, 2 and the running dL/dV (8 bytes a point).
// Each thread keeps u = -i a w (0 off the interior) of its two columns and
// their outer x neighbours, and E = u - (1/12)(axial u), as three-row
// register windows; the x neighbours of E travel through a two-row shared
// ring.  Per output row y, with E formed one row ahead:
//   Ybar = (axial interior E - 4 E_c) / h^2 + (corner u - 4 u_c) / (6 h^2)
//          + the pointwise terms (adjoint2d.cuh),
//   lam  = lam (or lam' at stage 4) + Ybar,   w_next = cw lam' + cy Ybar,
//   stages 4..2 store their dL/dV contribution; stage 1 adds the four to
//   the running dL/dV in the order 4, 3, 2, 1 (adjoint2d.cuh).
// The arithmetic is that of the shared-memory tile kernel, operation for
// operation, so the two give the same bits.  Every mbarrier wait is bounded
// (1 s); on timeout the CTA sets the timeout bit of the status, lets its
// copies in flight land and returns.
#pragma once

#include "adjoint2d.cuh"
#include "stage2d_tile.cuh"
#include "tmap.cuh"

namespace nlse {
namespace adjtma {

constexpr int NT = 128;              // threads per CTA
constexpr int TXC = 2 * NT;          // columns per CTA
constexpr int HB = TXC;              // first input TMA box (x0-2 .. x0+TXC-3); the second: 4 points
constexpr int HB2 = 4;
constexpr int S = 6;                 // input ring slots
constexpr uint64_t kWaitNs = 1000000000ull;
constexpr uint64_t kDrainNs = 50000000ull;

constexpr int al128(int v) { return (v + 127) / 128 * 128; }

// Shared-memory layout.  Input rows and E rows are indexed by column
// x - (x0 - 2); every TMA destination is 128-byte aligned.
template <typename R, int J>
struct Lay {
    static constexpr int CB = (int)sizeof(cplx<R>);
    static constexpr int RB = (int)sizeof(R);
    static constexpr int ROW = TXC + 4;
    static constexpr int IN_BYTES = ROW * CB;
    static constexpr int IN_SLOT = al128(IN_BYTES);
    static constexpr int T = TXC * CB;                   // one complex row
    static constexpr int VB = TXC * RB;                  // one real row
    static constexpr bool LAMP = J == 3 || J == 2;       // lam' from its own array
    static constexpr bool LAM = J < 4;                   // the running lam
    static constexpr bool G = J == 1;                    // dL/dV and the stored contributions
    static constexpr int E_Y = 0;
    static constexpr int E_LAMP = T;
    static constexpr int E_LAM = E_LAMP + (LAMP ? T : 0);
    static constexpr int E_V = E_LAM + (LAM ? T : 0);
    static constexpr int E_G = E_V + VB;                 // stages 4, 3, 2 contributions
    static constexpr int E_GV = E_G + (G ? 3 * VB : 0);  // the running dL/dV (8 bytes a point)
    static constexpr int E_BYTES = E_GV + (G ? TXC * 8 : 0);
    static constexpr int E_SLOT = al128(E_BYTES);
    static constexpr int E_OFF = S * IN_SLOT;
    static constexpr int R_OFF = E_OFF + 2 * E_SLOT;    // the E ring, two rows
    static constexpr int BAR_OFF = al128(R_OFF + 2 * ROW * CB);
    static constexpr int TOTAL = BAR_OFF + 8 * (S + 2) + 128;   // +128: base alignment slack
};

template <typename R>
struct WalkIO {
    cplx<R>* lam;          // running dL/dPsi_n
    cplx<R>* w_next;       // stages 4..2: cotangent of the previous stage's K
    R* g_out;              // stages 4..2: this stage's dL/dV contribution
    adj::gacc<R>* gV;      // stage 1: the running dL/dV
    int* flag;             // status bits
    int rows1;             // rows per stacked instance
};

template <typename R, bool CD, int J, int TY>
__global__ void __launch_bounds__(NT)
adj2d_walk_kernel(const __grid_constant__ CUtensorMap m_w, const __grid_constant__ CUtensorMap m_w2,
                  const __grid_constant__ CUtensorMap m_Y, const __grid_constant__ CUtensorMap m_lamp,
                  const __grid_constant__ CUtensorMap m_lam, const __grid_constant__ CUtensorMap m_V,
                  const __grid_constant__ CUtensorMap m_g4, const __grid_constant__ CUtensorMap m_g3,
                  const __grid_constant__ CUtensorMap m_g2, const __grid_constant__ CUtensorMap m_gV,
                  const WalkIO<R> io, const adj::Coef<R> c, const int nx, const int ny, const int dir) {
    using C = cplx<R>;
    using L = Lay<R, J>;
    using T2 = tile2d::Two<C>;
    using tile2d::ld2;
    using tile2d::st2;
    extern __shared__ unsigned char smem_raw[];
    unsigned char* smem = smem_raw + ((128 - (smem_u32(smem_raw) & 127)) & 127);

    const int t = threadIdx.x;
    const int x0 = blockIdx.x * TXC, y0 = blockIdx.y * TY;
    const int nrows = min(TY, ny - y0);
    const int jmax = nrows + 4;                  // input rows j = 0 .. jmax-1
    // Output row e is grid row ybase + dir * e, input row j is ybase + dir * (j - 2).
    const int ybase = dir > 0 ? y0 : y0 + nrows - 1;
    const uint32_t sbase = smem_u32(smem);
    const uint32_t ibar0 = sbase + L::BAR_OFF;   // S input barriers, then 2 epilogue barriers
    const uint32_t ebar0 = ibar0 + 8 * S;
    auto rstep = [&](int rl, int d) {
        rl += d;
        return rl < 0 ? io.rows1 - 1 : (rl == io.rows1 ? 0 : rl);
    };
    const int rl_base = ybase % io.rows1;

#ifdef NLSE_BOUNDS_CHECK
    {
        const int kk = 2 * t + 2;
        uint32_t dyn;
        asm("mov.u32 %0, %%dynamic_smem_size;" : "=r"(dyn));
        const bool okb = NLSE_IDX(io.flag, kk - 1, L::ROW, kSiteAdj2d) && NLSE_IDX(io.flag, kk + 2, L::ROW, kSiteAdj2d) &&
                         NLSE_IDX(io.flag, TXC + 3, L::ROW, kSiteAdj2d) && NLSE_IDX(io.flag, 2 * t + 1, TXC, kSiteAdj2d) &&
                         NLSE_IDX(io.flag, x0, nx, kSiteAdj2d) && NLSE_IDX(io.flag, y0, ny, kSiteAdj2d) &&
                         NLSE_ALIGN16(io.flag, (int64_t)(x0 - 2) * L::CB, kSiteAdj2d) &&
                         NLSE_ALIGN16(io.flag, (int64_t)(x0 - 2 + HB) * L::CB, kSiteAdj2d) &&
                         NLSE_ALIGN16(io.flag, (int64_t)x0 * L::CB, kSiteAdj2d) &&
                         NLSE_ALIGN16(io.flag, (int64_t)x0 * L::RB, kSiteAdj2d) &&
                         NLSE_ALIGN16(io.flag, (int64_t)x0 * 8, kSiteAdj2d) &&
                         NLSE_IDX(io.flag, L::TOTAL - 1, dyn, kSiteAdj2d);
        if (__syncthreads_or(!okb)) return;
    }
#endif

    if (t == 0) {
        tma_prefetch_desc(&m_w);
        tma_prefetch_desc(&m_w2);
        for (int s = 0; s < S + 2; ++s) mbar_init(ibar0 + 8 * s, 1);
        mbar_init_fence();
    }
    __syncthreads();

    // Input rows are issued by the first lane of warp 1, epilogue rows by the
    // first lane of warp 2; warp 0 and the last warp form the halo E.
    constexpr int PIN = 32, PE = 64;
    auto issue_in = [&](int j) {
        const int s = j % S;
        const uint32_t dst = sbase + s * L::IN_SLOT;
        const uint32_t bar = ibar0 + 8 * s;
        const int r = ybase + dir * (j - 2);
        mbar_expect_tx(bar, L::IN_BYTES);
        tile2d::load_cplx_box<R>(dst, &m_w, x0 - 2, r, bar);
        tile2d::load_cplx_box<R>(dst + HB * L::CB, &m_w2, x0 - 2 + HB, r, bar);
    };
    int erl = rl_base;                           // instance row of the next epilogue row
    auto issue_e = [&](int e) {
        const uint32_t dst = sbase + L::E_OFF + (e & 1) * L::E_SLOT;
        const uint32_t bar = ebar0 + 8 * (e & 1);
        const int r = ybase + dir * e;
        (void)(NLSE_IDX(io.flag, r, ny, kSiteAdj2d) && NLSE_IDX(io.flag, erl, io.rows1, kSiteAdj2d));
        mbar_expect_tx(bar, L::E_BYTES);
        tile2d::load_cplx_box<R>(dst + L::E_Y, &m_Y, x0, r, bar);
        if (L::LAMP) tile2d::load_cplx_box<R>(dst + L::E_LAMP, &m_lamp, x0, r, bar);
        if (L::LAM) tile2d::load_cplx_box<R>(dst + L::E_LAM, &m_lam, x0, r, bar);
        tma_load_2d(dst + L::E_V, &m_V, x0, erl, bar);
        erl = rstep(erl, dir);
        if (L::G) {
            tma_load_2d(dst + L::E_G, &m_g4, x0, r, bar);
            tma_load_2d(dst + L::E_G + L::VB, &m_g3, x0, r, bar);
            tma_load_2d(dst + L::E_G + 2 * L::VB, &m_g2, x0, r, bar);
            tma_load_2d(dst + L::E_GV, &m_gV, x0, r, bar);
        }
    };
    int next = 0, enext = 0;
    if (t == PIN)
        for (; next < S && next < jmax; ++next) issue_in(next);
    if (t == PE) issue_e(enext++);

    auto irow = [&](int j) { return reinterpret_cast<const C*>(smem + (j % S) * L::IN_SLOT); };
    auto erow = [&](int e) { return smem + L::E_OFF + (e & 1) * L::E_SLOT; };
    C* ering = reinterpret_cast<C*>(smem + L::R_OFF);

    bool ok = true;
    auto wait_in = [&](int j) {
        if (ok) ok = mbar_wait(ibar0 + 8 * (j % S), (uint32_t)((j / S) & 1), kWaitNs);
    };
    auto wait_e = [&](int e) {
        if (ok) ok = mbar_wait(ebar0 + 8 * (e & 1), (uint32_t)((e >> 1) & 1), kWaitNs);
    };

    // Interior tests: a column x, and grid row r whose instance row is rl.
    auto colin = [&](int x) { return x > 0 && x < nx - 1; };
    auto rowin = [&](int r, int rl) { return r >= 0 && r < ny && rl > 0 && rl < io.rows1 - 1; };
    auto u = [&](C stored, bool inner) { return adj::u_of(c, stored, inner); };

    const int xa = x0 + 2 * t;                   // this thread's columns xa, xa + 1
    const int k = 2 * t + 2;                     // xa in the row buffers
    const bool xin = xa < nx;                    // nx is even: then xa + 1 < nx too
    const bool ca = colin(xa), cb = colin(xa + 1), cl = colin(xa - 1), cr = colin(xa + 2);
    const bool cll = colin(x0 - 2), crr = colin(x0 + TXC + 1);   // halo columns of the CTA

    // Prologue: input rows y-2 .. y+1 (y = ybase) give E(., y-1) and E(., y).
    wait_in(0); wait_in(1); wait_in(2); wait_in(3);
    bool alive = __syncthreads_and(ok);
    int yla = rstep(rl_base, dir);               // instance row of y + dir
    bool fm, f0, f1;                             // rows y - dir, y, y + dir interior
    T2 um, u0, u1, em, e0;
    C lm, rm, l0, r0;
    {
        const int rl1 = rstep(rl_base, -dir), rl0 = rstep(rl1, -dir);
        const bool f_ = rowin(ybase - 2 * dir, rl0);
        fm = rowin(ybase - dir, rl1);
        f0 = rowin(ybase, rl_base);
        f1 = rowin(ybase + dir, yla);
        if (alive) {
            const C* q0 = irow(0); const C* q1 = irow(1); const C* q2 = irow(2); const C* q3 = irow(3);
            const T2 w0 = ld2(q0 + k), w1 = ld2(q1 + k), w2 = ld2(q2 + k), w3 = ld2(q3 + k);
            const T2 umm{u(w0.a, ca && f_), u(w0.b, cb && f_)};
            um = T2{u(w1.a, ca && fm), u(w1.b, cb && fm)};
            u0 = T2{u(w2.a, ca && f0), u(w2.b, cb && f0)};
            u1 = T2{u(w3.a, ca && f1), u(w3.b, cb && f1)};
            lm = u(q1[k - 1], cl && fm); rm = u(q1[k + 2], cr && fm);
            l0 = u(q2[k - 1], cl && f0); r0 = u(q2[k + 2], cr && f0);
            em = T2{adj::e_of<CD>(um.a, um.b, lm, u0.a, umm.a), adj::e_of<CD>(um.b, rm, um.a, u0.b, umm.b)};
            e0 = T2{adj::e_of<CD>(u0.a, u0.b, l0, u1.a, um.a), adj::e_of<CD>(u0.b, r0, u0.a, u1.b, um.b)};
            C* er = ering;                                   // input row 2 -> E ring row 0
            st2(er + k, e0);
            if (t == 0) er[1] = adj::e_of<CD>(l0, u0.a, u(q2[0], cll && f0), u(q3[1], cl && f1), lm);
            if (t == NT - 1)
                er[TXC + 2] = adj::e_of<CD>(r0, u(q2[TXC + 3], crr && f0), u0.b, u(q3[TXC + 2], cr && f1), rm);
        }
    }
    __syncthreads();

#pragma unroll 1
    for (int i = 0; i < TY; ++i) {
        if (!alive || i >= nrows) break;
        const int j = i + 2;                     // input row of y
        const int y = ybase + dir * i;
        const int ylb = rstep(yla, dir);         // instance row of y + 2 dir
        wait_in(j + 2);
        if (!__syncthreads_and(ok)) { alive = false; break; }
        if (t == PIN && next < jmax) issue_in(next++);
        if (t == PE && enext < nrows) issue_e(enext++);

        // u of rows y + dir (outer neighbours) and y + 2 dir, then E(., y + dir).
        const bool f2 = rowin(y + 2 * dir, ylb);
        const C* q1 = irow(j + 1);
        const C* q2 = irow(j + 2);
        const C l1 = u(q1[k - 1], cl && f1), r1 = u(q1[k + 2], cr && f1);
        const T2 w2 = ld2(q2 + k);
        const T2 u2{u(w2.a, ca && f2), u(w2.b, cb && f2)};
        const T2 e1{adj::e_of<CD>(u1.a, u1.b, l1, u2.a, u0.a), adj::e_of<CD>(u1.b, r1, u1.a, u2.b, u0.b)};
        C* en = ering + ((j + 1) & 1) * L::ROW;
        st2(en + k, e1);
        if (t == 0) en[1] = adj::e_of<CD>(l1, u1.a, u(q1[0], cll && f1), u(q2[1], cl && f2), l0);
        if (t == NT - 1)
            en[TXC + 2] = adj::e_of<CD>(r1, u(q1[TXC + 3], crr && f1), u1.b, u(q2[TXC + 2], cr && f2), r0);
        // No barrier here: the step below reads the E ring row written in the
        // previous iteration, ordered by the barrier at the top of the loop.
        wait_e(i);

        if (xin && NLSE_IDX(io.flag, (int64_t)y * nx + xa + 1, (int64_t)nx * ny, kSiteAdj2d)) {
            const C* er = ering + (j & 1) * L::ROW;          // er[k-1] = E(xa-1, y), er[k+2] = E(xa+2, y)
            const bool ia = ca && f0, ib = cb && f0;
            const C z = czero<C>();
            const C eca = ia ? e0.a : z, ecb = ib ? e0.b : z;
            C ya = adj::ybar_stencil<CD>(c, eca, ecb, (cl && f0) ? er[k - 1] : z, (ca && f1) ? e1.a : z,
                                         (ca && fm) ? em.a : z, u0.a, u1.b, l1, um.b, lm);
            C yb = adj::ybar_stencil<CD>(c, ecb, (cr && f0) ? er[k + 2] : z, eca, (cb && f1) ? e1.b : z,
                                         (cb && fm) ? em.b : z, u0.b, r1, u1.a, rm, um.a);
            const unsigned char* es = erow(i);
            const T2 w0 = ld2(irow(j) + k);                  // the stored cotangent at (xa, y), (xa+1, y)
            const T2 Y = ld2(reinterpret_cast<const C*>(es + L::E_Y) + 2 * t);
            const R* vv = reinterpret_cast<const R*>(es + L::E_V) + 2 * t;
            const R ga = adj::pointwise(c, ia, adj::wscale(c, w0.a), e0.a, Y.a, vv[0], ya);
            const R gb = adj::pointwise(c, ib, adj::wscale(c, w0.b), e0.b, Y.b, vv[1], yb);
            const int64_t p = (int64_t)y * nx + xa;
            T2 lamp = w0;                                    // stage 4: w holds lam'
            if constexpr (L::LAMP) lamp = ld2(reinterpret_cast<const C*>(es + L::E_LAMP) + 2 * t);
            T2 lam = lamp;
            if constexpr (L::LAM) lam = ld2(reinterpret_cast<const C*>(es + L::E_LAM) + 2 * t);
            st2(io.lam + p, T2{add2(lam.a, ya), add2(lam.b, yb)});
            if constexpr (J > 1) {
                st2(io.w_next + p, T2{adj::w_next(c, lamp.a, ya), adj::w_next(c, lamp.b, yb)});
                *reinterpret_cast<C*>(io.g_out + p) = adj::two<C>(ga, gb);
            } else {
                using A = adj::gacc<R>;
                const R* g = reinterpret_cast<const R*>(es + L::E_G) + 2 * t;
                const A* gv = reinterpret_cast<const A*>(es + L::E_GV) + 2 * t;
                io.gV[p] = adj::gv_total(gv[0], g[0], g[TXC], g[2 * TXC], ga);
                io.gV[p + 1] = adj::gv_total(gv[1], g[1], g[TXC + 1], g[2 * TXC + 1], gb);
            }
        }
        lm = l0; rm = r0; l0 = l1; r0 = r1;
        um = u0; u0 = u1; u1 = u2;
        em = e0; e0 = e1;
        fm = f0; f0 = f1; f1 = f2;
        yla = ylb;
    }

    if (!alive) {
        // A transfer never arrived: report, let this CTA's copies in flight land, leave.
        if (t == 0) atomicOr(io.flag, kStatusTimeout);
        if (t == PIN)
            for (int j = next > S ? next - S : 0; j < next; ++j)
                mbar_wait(ibar0 + 8 * (j % S), (uint32_t)((j / S) & 1), kDrainNs);
        if (t == PE)
            for (int e = enext > 2 ? enext - 2 : 0; e < enext; ++e)
                mbar_wait(ebar0 + 8 * (e & 1), (uint32_t)((e >> 1) & 1), kDrainNs);
    }
}

// ---- host side -------------------------------------------------------------

template <typename R, bool CD, int J, int TY>
cudaError_t launch_t(const AdjLaunch& A, cudaStream_t st) {
    const int nx = (int)A.nx, ny = (int)A.ny;
    const int rows1 = (int)(A.rows1 ? A.rows1 : A.ny);
    CUtensorMap m_w, m_w2, m_Y, m_lamp, m_lam, m_V, m_g4, m_g3, m_g2, m_gV;
    if (!complex_map<R>(&m_w, A.w, nx, ny, HB) || !complex_map<R>(&m_w2, A.w, nx, ny, HB2) ||
        !complex_map<R>(&m_Y, A.Y, nx, ny, TXC) || !real_map<R>(&m_V, A.V, nx, rows1, TXC))
        return cudaErrorInvalidValue;
    m_lamp = m_lam = m_g4 = m_g3 = m_g2 = m_gV = m_w;
    if ((J == 3 || J == 2) && !complex_map<R>(&m_lamp, A.lamp, nx, ny, TXC)) return cudaErrorInvalidValue;
    if (J < 4 && !complex_map<R>(&m_lam, A.lam, nx, ny, TXC)) return cudaErrorInvalidValue;
    if (J == 1 && (!real_map<R>(&m_g4, A.g_in[0], nx, ny, TXC) || !real_map<R>(&m_g3, A.g_in[1], nx, ny, TXC) ||
                   !real_map<R>(&m_g2, A.g_in[2], nx, ny, TXC) || !real_map<double>(&m_gV, A.gV, nx, ny, TXC)))
        return cudaErrorInvalidValue;
    WalkIO<R> io;
    io.lam = (cplx<R>*)A.lam;
    io.w_next = (cplx<R>*)A.w_next;
    io.g_out = (R*)A.g_out;
    io.gV = (adj::gacc<R>*)A.gV;
    io.flag = A.flag;
    io.rows1 = rows1;
    auto kern = adj2d_walk_kernel<R, CD, J, TY>;
    const int smem = Lay<R, J>::TOTAL;
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (e != cudaSuccess) return e;
    }
    dim3 grid((nx + TXC - 1) / TXC, (ny + TY - 1) / TY);
    // Consecutive stages walk the rows in opposite directions.
    const int dir = (J % 2 == 0) ? 1 : -1;
    kern<<<grid, NT, smem, st>>>(m_w, m_w2, m_Y, m_lamp, m_lam, m_V, m_g4, m_g3, m_g2, m_gV, io,
                                 adj::make_coef<R>(A.h, A.a, A.s, A.scale_w, A.cw, A.cy), nx, ny, dir);
    return cudaGetLastError();
}

template <typename R, bool CD, int TY>
cudaError_t launch_j(const AdjLaunch& A, cudaStream_t st) {
    switch (A.j) {
        case 4: return launch_t<R, CD, 4, TY>(A, st);
        case 3: return launch_t<R, CD, 3, TY>(A, st);
        case 2: return launch_t<R, CD, 2, TY>(A, st);
        case 1: return launch_t<R, CD, 1, TY>(A, st);
    }
    return cudaErrorInvalidValue;
}

template <int TY>
cudaError_t launch_rows(const AdjLaunch& A, cudaStream_t st) {
    const bool cd = A.lap == 1;
    if (A.prec == 0) return cd ? launch_j<float, true, TY>(A, st) : launch_j<float, false, TY>(A, st);
    return cd ? launch_j<double, true, TY>(A, st) : launch_j<double, false, TY>(A, st);
}

}  // namespace adjtma
}  // namespace nlse
