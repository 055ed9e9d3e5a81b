// stage2d_tile.cuh -- one CTA's work of the fused 2D RK4 stage (and of the
// standalone 2SHOC Laplacian): a y-streaming walk fed by the tensor memory
// accelerator.  Used by the single-grid kernel (stage2d_tma.cu) and by the
// batched kernel over many grids (batch2d.cu).
//
// One CTA of NT threads owns TXC = 2 NT consecutive columns (two per thread)
// and walks down TY rows.  Two rings of shared-memory row slots are filled by
// TMA tile loads, each slot completing on its own mbarrier:
//   * the input ring (S slots, up to S rows ahead): the stage input row with
//     a 2-point x halo (a TXC-point and a 4-point TMA box, so that both land
//     on 128-byte aligned shared addresses);
//   * the epilogue ring (2 slots, one output row ahead): V, and for stages
//     2-4 Psi^n and the RK4 accumulator (stage 4 in FP32: the compensated
//     part too) on the output row.  When V fits in a quarter of L2 its loads
//     carry an evict-last policy, so that V, read by every stage, stays in L2
//     while the other fields stream through.
// Each thread keeps its two columns' stage input, their outer x neighbours
// and D in registers as a sliding window; the x neighbours of D travel
// through a two-row shared ring.  The walk runs down the grid on odd stages
// and up on even ones, so each stage starts on the rows the previous stage
// wrote last (still in L2).  Per output row y, with D formed one row ahead:
//   step 1 (Eq. 2d2shocs1): D = (sum of the four axial Psi - 4 Psi_c) / h^2,
//                           boundary points D_b of Eq. (dbc_lap);
//   step 2 (Eq. 2d2shocs2): Lap = D_c - (1/12) sum of the four axial D
//                           + (1/(6h^2)) (four corner Psi - 4 Psi_c);
// in FP64 the corner sum of row y is hx(y-1) + hx(y+1), with hx the sum of a
// point's two x neighbours that step 1 formed for D on those rows, kept in
// the register window (the same additions, two fewer per point; FP32 forms
// them again, which keeps its walk within 64 registers);
// With the multi-storage form (LP = 2) step 1 keeps the two second
// differences apart, Eq. (2d2shocMs1), D^y in the register window and D^x in
// the shared ring, and step 2 is Eq. (2d2shocMs2):
//   Lap = (7/6)(D^x_c + D^y_c) - (1/12)(D^x of the two x neighbours + D^y of
//   the two y neighbours);
// at a point on the boundary of one axis only, that axis' D^a is D_b of
// Eq. (dbc_lap) minus the other axis' second difference.
//   F = i[a Lap + (s|Psi|^2 - V) Psi] (Sec. 3.1), F_b = 0 (Eq. dbc_ut);
//   the RK4 stage epilogue (Eq. RK4, accumulated-increment form).
// Complex64 arithmetic uses the packed f32x2 instructions.  Every mbarrier
// wait is bounded (1 s); on timeout the CTA sets the timeout bit of the status,
// lets its own copies in flight land and returns.
#pragma once

#include "nlse_device.cuh"
#include "tma.cuh"

namespace nlse {
namespace tile2d {

constexpr int S = 6;                 // input ring slots
constexpr uint64_t kWaitNs = 1000000000ull;
constexpr uint64_t kDrainNs = 50000000ull;

constexpr int al128(int v) { return (v + 127) / 128 * 128; }

// Shared-memory layout.  Input rows and D rows are indexed by column
// x - (x0 - 2), so a thread's column pair (xa, xa+1) sits at the 16-byte
// aligned index 2t + 2.  Every TMA destination is 128-byte aligned.  The
// epilogue slots hold only what the stage reads (stage 1: V; stages 2, 3:
// Psi^n, the accumulator and V; stage 4 in FP32 also the compensated part), so
// the earlier stages need less shared memory and fit one more CTA per SM.
template <typename R, int NT, int STAGE>
struct Lay {
    static constexpr int TXC = 2 * NT;
    static constexpr int CB = (int)sizeof(cplx<R>);
    static constexpr int ROW = TXC + 4;                       // x0-2 .. x0+TXC+1
    static constexpr int IN_BYTES = ROW * CB;
    static constexpr int IN_SLOT = al128(IN_BYTES);
    static constexpr int T_BYTES = TXC * CB;                  // one complex output row
    static constexpr int V_BYTES = TXC * (int)sizeof(R);
    static constexpr bool PA = STAGE >= 2;                    // Psi^n and the accumulator
    static constexpr bool LO = STAGE == 4 && sizeof(R) == 4;  // the compensated part
    static constexpr int E_PSI = 0, E_ACC = T_BYTES, E_LO = 2 * T_BYTES;
    static constexpr int E_V = (PA ? 2 * T_BYTES : 0) + (LO ? T_BYTES : 0);
    static constexpr int E_SLOT = STAGE >= 1 ? al128(E_V + V_BYTES) : 0;
    static constexpr int IN_OFF = 0;
    static constexpr int E_OFF = S * IN_SLOT;
    static constexpr int D_OFF = E_OFF + 2 * E_SLOT;
    static constexpr int BAR_OFF = al128(D_OFF + 2 * ROW * CB);
    static constexpr int TOTAL = BAR_OFF + 8 * (S + 2) + 128;   // +128: base alignment slack
};

template <typename R>
__device__ __forceinline__ void load_cplx_box(uint32_t dst, const CUtensorMap* m, int x, int r, uint32_t bar) {
    if constexpr (sizeof(R) == 4) tma_load_2d(dst, m, x, r, bar);       // complex64 as 8-byte elements
    else tma_load_3d(dst, m, 0, x, r, bar);                             // complex128 as (re, im) doubles
}

template <typename C> __device__ __forceinline__ C pair(decltype(C::x) a, decltype(C::x) b) {
    C z; z.x = a; z.y = b; return z;
}

// Two adjacent complex values (columns x, x+1).
template <typename C> struct Two { C a, b; };
__device__ __forceinline__ Two<float2> ld2(const float2* p) {
    const float4 v = *reinterpret_cast<const float4*>(p);
    return {make_float2(v.x, v.y), make_float2(v.z, v.w)};
}
__device__ __forceinline__ Two<double2> ld2(const double2* p) { return {p[0], p[1]}; }
__device__ __forceinline__ void st2(float2* p, Two<float2> v) {
    *reinterpret_cast<float4*>(p) = make_float4(v.a.x, v.a.y, v.b.x, v.b.y);
}
__device__ __forceinline__ void st2(double2* p, Two<double2> v) { p[0] = v.a; p[1] = v.b; }

// LP: 0 single-storage 2SHOC, 1 CD, 2 multi-storage 2SHOC.  INNER: every
// point whose D or output the CTA forms is an interior grid point, so the
// per-point boundary and grid-edge tests drop out (the arithmetic is the same).
template <typename R, int LP, int STAGE, int NT, int TY, bool INNER>
__device__ __forceinline__ void stage2d_walk(const CUtensorMap* m_in, const CUtensorMap* m_in2,
                                             const CUtensorMap* m_V, const CUtensorMap* m_psi,
                                             const CUtensorMap* m_acc, const CUtensorMap* m_lo,
                                             const StageIO<R>& io, const Coef<R>& c, const int nx, const int ny,
                                             const int x0, const int y0, const int dir) {
    constexpr bool CD = LP == 1, MS = LP == 2;
    constexpr int TXC = 2 * NT;          // columns per CTA
    constexpr int HB = TXC;              // first input TMA box: x0-2 .. x0+TXC-3; the second: 4 points
    using C = cplx<R>;
    using L = Lay<R, NT, STAGE>;
    using T2 = Two<C>;
    constexpr bool NEED_E = STAGE >= 1;          // V on the output row
    constexpr bool NEED_PA = STAGE >= 2;
    constexpr bool NEED_LO = STAGE == 4 && sizeof(R) == 4;
    extern __shared__ unsigned char smem_raw[];
    unsigned char* smem = smem_raw + ((128 - (smem_u32(smem_raw) & 127)) & 127);

    const int t = threadIdx.x;
    const int nrows = min(TY, ny - y0);
    const int jmax = nrows + 4;                  // input rows j = 0 .. jmax-1
    // The CTA walks its rows downwards (dir = +1) or upwards (dir = -1):
    // output row e is grid row ybase + dir * e, input row j is ybase + dir * (j - 2).
    const int ybase = dir > 0 ? y0 : y0 + nrows - 1;
    const uint32_t sbase = smem_u32(smem);
    const uint32_t ibar0 = sbase + L::BAR_OFF;   // S input barriers, then 2 epilogue barriers
    const uint32_t ebar0 = ibar0 + 8 * S;
    // Row within its stacked instance (the grid row itself without a stack),
    // one division per CTA and then stepped along the walk.
    auto rstep = [&](int rl, int d) {
        rl += d;
        return rl < 0 ? io.rows1 - 1 : (rl == io.rows1 ? 0 : rl);
    };
    const int rl_base = ybase % io.rows1;

#ifdef NLSE_BOUNDS_CHECK
    {
        // This thread's column window k-1 .. k+2 and the CTA's halo columns in
        // the row buffers, its epilogue slots, the tile origin, the TMA x
        // coordinates' 16-byte alignment, and the dynamic shared memory the
        // launch gave against the layout.
        const int kk = 2 * t + 2;
        uint32_t dyn;
        asm("mov.u32 %0, %%dynamic_smem_size;" : "=r"(dyn));
        const bool okb = NLSE_IDX(io.flag, kk - 1, L::ROW, kSiteTile2d) && NLSE_IDX(io.flag, kk + 2, L::ROW, kSiteTile2d) &&
                         NLSE_IDX(io.flag, TXC + 3, L::ROW, kSiteTile2d) && NLSE_IDX(io.flag, 2 * t + 1, TXC, kSiteTile2d) &&
                         NLSE_IDX(io.flag, x0, nx, kSiteTile2d) && NLSE_IDX(io.flag, y0, ny, kSiteTile2d) &&
                         NLSE_ALIGN16(io.flag, (int64_t)(x0 - 2) * L::CB, kSiteTile2d) &&
                         NLSE_ALIGN16(io.flag, (int64_t)(x0 - 2 + HB) * L::CB, kSiteTile2d) &&
                         NLSE_ALIGN16(io.flag, (int64_t)x0 * L::CB, kSiteTile2d) &&
                         NLSE_ALIGN16(io.flag, (int64_t)x0 * (int64_t)sizeof(R), kSiteTile2d) &&
                         NLSE_IDX(io.flag, L::TOTAL - 1, dyn, kSiteTile2d);
        if (__syncthreads_or(!okb)) return;
    }
#endif

    if (t == 0) {
        tma_prefetch_desc(m_in);
        tma_prefetch_desc(m_in2);
        for (int s = 0; s < S + 2; ++s) mbar_init(ibar0 + 8 * s, 1);
        mbar_init_fence();
    }
    __syncthreads();

    // Producer side: input rows are issued by the first lane of warp 1 (PIN),
    // epilogue rows by the first lane of warp 2 (PE), while warp 0 forms the
    // left halo D and the last warp the right one: with four warps each
    // carries one extra task per row, and no warp waits at the row barrier for
    // another's two.
    constexpr int PIN = NT >= 64 ? 32 : 0;
    constexpr int PE = NT >= 96 ? 64 : 0;
    auto issue_in = [&](int j) {
        const int s = j % S;
        const uint32_t dst = sbase + L::IN_OFF + s * L::IN_SLOT;
        const uint32_t bar = ibar0 + 8 * s;
        const int r = ybase + dir * (j - 2);
        mbar_expect_tx(bar, L::IN_BYTES);
        load_cplx_box<R>(dst, m_in, x0 - 2, r, bar);
        load_cplx_box<R>(dst + HB * L::CB, m_in2, x0 - 2 + HB, r, bar);
    };
    int erl = rl_base;                           // instance row of the next epilogue row
    auto issue_e = [&](int e) {
        const uint32_t dst = sbase + L::E_OFF + (e & 1) * L::E_SLOT;
        const uint32_t bar = ebar0 + 8 * (e & 1);
        const int r = ybase + dir * e;
        // (TMA loads outside the grid read the fill value; the rows are checked for the record only.)
        (void)(NLSE_IDX(io.flag, r, ny, kSiteTile2d) && NLSE_IDX(io.flag, erl, io.rows1, kSiteTile2d));
        uint32_t bytes = L::V_BYTES;
        if (NEED_PA) bytes += 2 * L::T_BYTES;
        if (NEED_LO) bytes += L::T_BYTES;
        mbar_expect_tx(bar, bytes);
        if (io.keep_v) tma_load_2d_hint(dst + L::E_V, m_V, x0, erl, bar, l2_evict_last());
        else tma_load_2d(dst + L::E_V, m_V, x0, erl, bar);
        erl = rstep(erl, dir);
        if (NEED_PA) {
            load_cplx_box<R>(dst + L::E_PSI, m_psi, x0, r, bar);
            load_cplx_box<R>(dst + L::E_ACC, m_acc, x0, r, bar);
        }
        if (NEED_LO) load_cplx_box<R>(dst + L::E_LO, m_lo, x0, r, bar);
    };
    int next = 0, enext = 0;                     // rows issued so far (by PIN, by PE)
    if (t == PIN)
        for (; next < S && next < jmax; ++next) issue_in(next);
    if (NEED_E && t == PE) issue_e(enext++);

    auto irow = [&](int j) { return reinterpret_cast<const C*>(smem + L::IN_OFF + (j % S) * L::IN_SLOT); };
    auto erow = [&](int e) { return smem + L::E_OFF + (e & 1) * L::E_SLOT; };
    C* dring = reinterpret_cast<C*>(smem + L::D_OFF);

    bool ok = true;
    auto wait_in = [&](int j) {
        if (ok) ok = mbar_wait(ibar0 + 8 * (j % S), (uint32_t)((j / S) & 1), kWaitNs);
    };
    auto wait_e = [&](int e) {
        if (ok) ok = mbar_wait(ebar0 + 8 * (e & 1), (uint32_t)((e >> 1) & 1), kWaitNs);
    };

    const C m4 = pair<C>(-4, -4), m2 = pair<C>(-2, -2), m12 = pair<C>(R(-1.0 / 12.0), R(-1.0 / 12.0));
    const C c76 = pair<C>(R(7.0 / 6.0), R(7.0 / 6.0));
    // FP64 stages carry a Lap instead of Lap: the a of F folds into the
    // difference weights and the boundary value a D_b = -N Psi_b (Eq. dbc_lap),
    // two FP64 multiplies fewer per point.  FP64 runs at its arithmetic rate
    // on this GPU; FP32 and the standalone Laplacian keep the unscaled form.
    constexpr bool SC = sizeof(R) == 8 && STAGE >= 1;
    const R wd = SC ? c.a * c.inv_h2 : c.inv_h2, we = SC ? c.a * c.inv_6h2 : c.inv_6h2;
    const C ih2 = pair<C>(wd, wd), i6h2 = pair<C>(we, we);
    const C a2 = pair<C>(c.a, c.a);
    auto bnd_D = [&](C ctr, R v) -> C {
        if constexpr (SC) return cscale(-nonlin(c.s, ctr, v), ctr);
        else return dirichlet_D(c, ctr, v);
    };
    const C ca2 = pair<C>(-io.c_acc, io.c_acc), cy2 = pair<C>(-io.c_y, io.c_y);

    // D at grid point (x, r), rl its row within its instance, from its five
    // stencil values (boundary: Eq. dbc_lap, V read from global memory;
    // outside the grid: 0, never used).
    // V at (x, row rl of its instance), read from global memory at boundary points.
    auto vat = [&](int rl, int x) -> R {
        const int64_t q = (int64_t)rl * nx + x;
        return NLSE_IDX(io.flag, q, (int64_t)io.rows1 * nx, kSiteTile2d) ? io.V[q] : R(0);
    };
    auto dpoint = [&](int x, int r, int rl, C ctr, C up, C dn, C lf, C rt) -> C {
        if constexpr (!INNER) {
            if (x < 0 || x >= nx || r < 0 || r >= ny) return czero<C>();
            if (x == 0 || x == nx - 1 || rl == 0 || rl == io.rows1 - 1)
                return bnd_D(ctr, vat(rl, x));
        }
        return mul2(fma2(m4, ctr, add2(add2(lf, rt), add2(up, dn))), ih2);
    };
    // The same from the sum hx of the two x neighbours (FP64, which keeps hx).
    auto dpoint_h = [&](int x, int r, int rl, C ctr, C up, C dn, C hx) -> C {
        if constexpr (!INNER) {
            if (x < 0 || x >= nx || r < 0 || r >= ny) return czero<C>();
            if (x == 0 || x == nx - 1 || rl == 0 || rl == io.rows1 - 1)
                return bnd_D(ctr, vat(rl, x));
        }
        return mul2(fma2(m4, ctr, add2(hx, add2(up, dn))), ih2);
    };
    // The x-neighbour sums of this thread's pair on a row (its values, the outer left and right ones).
    auto hpair = [&](const T2& cc, C l, C r) { return T2{add2(l, cc.b), add2(cc.a, r)}; };

    // Multi-storage step 1 at grid point (x, r): (D^x, D^y).  Outside the grid:
    // 0; on the boundary of both axes: 0 (never used).
    auto ms_point = [&](int x, int r, int rl, C ctr, C up, C dn, C lf, C rt) -> Two<C> {
        if (!INNER && (x < 0 || x >= nx || r < 0 || r >= ny)) return {czero<C>(), czero<C>()};
        Two<C> d{mul2(fma2(m2, ctr, add2(lf, rt)), ih2), mul2(fma2(m2, ctr, add2(up, dn)), ih2)};
        if constexpr (INNER) return d;
        const bool bx = x == 0 || x == nx - 1, by = rl == 0 || rl == io.rows1 - 1;
        if (bx || by) {
            const C lb = bnd_D(ctr, vat(rl, x));
            if (bx && by) d = {czero<C>(), czero<C>()};
            else if (bx) d.a = sub2(lb, d.b);
            else d.b = sub2(lb, d.a);
        }
        return d;
    };

    const int xa = x0 + 2 * t;                   // this thread's columns xa, xa + 1
    const int k = 2 * t + 2;                     // xa in the row buffers
    const bool xin = INNER || xa < nx;           // nx is even: then xa + 1 < nx too

    // Prologue: input rows y0-2 .. y0+1 give D(., y0-1) and D(., y0).
    wait_in(0); wait_in(1); wait_in(2); wait_in(3);
    bool alive = __syncthreads_and(ok);
    T2 cm, c0, c1, dm, d0;
    // FP64 single-storage 2SHOC keeps the x-neighbour sums of rows y - 1, y.
    constexpr bool KEEPH = sizeof(R) == 8 && !MS && !CD;
    T2 hm, h0;
    C lm, rm, l0, r0;
    T2 dx0;                                      // multi storage: D^x of row y (D^y is in dm, d0, d1)
    if (alive && MS) {
        const C* q0 = irow(0); const C* q1 = irow(1); const C* q2 = irow(2); const C* q3 = irow(3);
        const T2 cmm = ld2(q0 + k);
        cm = ld2(q1 + k); c0 = ld2(q2 + k); c1 = ld2(q3 + k);
        lm = q1[k - 1]; rm = q1[k + 2];
        l0 = q2[k - 1]; r0 = q2[k + 2];
        const int yb = ybase - dir, rlb = rstep(rl_base, -dir);
        dm.a = ms_point(xa, yb, rlb, cm.a, cmm.a, c0.a, lm, cm.b).b;
        dm.b = ms_point(xa + 1, yb, rlb, cm.b, cmm.b, c0.b, cm.a, rm).b;
        const Two<C> pa = ms_point(xa, ybase, rl_base, c0.a, cm.a, c1.a, l0, c0.b);
        const Two<C> pb = ms_point(xa + 1, ybase, rl_base, c0.b, cm.b, c1.b, c0.a, r0);
        dx0 = T2{pa.a, pb.a};
        d0 = T2{pa.b, pb.b};
        C* drow = dring;                                   // D^x of input row 2 -> ring row 0
        st2(drow + k, dx0);
        if (t == 0) drow[1] = ms_point(x0 - 1, ybase, rl_base, l0, q1[1], q3[1], q2[0], c0.a).a;
        if (t == NT - 1) drow[TXC + 2] = ms_point(x0 + TXC, ybase, rl_base, r0, q1[TXC + 2], q3[TXC + 2], c0.b, q2[TXC + 3]).a;
    } else if (alive) {
        const C* q0 = irow(0); const C* q1 = irow(1); const C* q2 = irow(2); const C* q3 = irow(3);
        const T2 cmm = ld2(q0 + k);
        cm = ld2(q1 + k); c0 = ld2(q2 + k); c1 = ld2(q3 + k);
        lm = q1[k - 1]; rm = q1[k + 2];
        l0 = q2[k - 1]; r0 = q2[k + 2];
        const int yb = ybase - dir, rlb = rstep(rl_base, -dir);   // the row before the first output row
        if constexpr (KEEPH) {
            hm = hpair(cm, lm, rm);
            h0 = hpair(c0, l0, r0);
            dm.a = dpoint_h(xa, yb, rlb, cm.a, cmm.a, c0.a, hm.a);
            dm.b = dpoint_h(xa + 1, yb, rlb, cm.b, cmm.b, c0.b, hm.b);
            d0.a = dpoint_h(xa, ybase, rl_base, c0.a, cm.a, c1.a, h0.a);
            d0.b = dpoint_h(xa + 1, ybase, rl_base, c0.b, cm.b, c1.b, h0.b);
        } else {
            dm.a = dpoint(xa, yb, rlb, cm.a, cmm.a, c0.a, lm, cm.b);
            dm.b = dpoint(xa + 1, yb, rlb, cm.b, cmm.b, c0.b, cm.a, rm);
            d0.a = dpoint(xa, ybase, rl_base, c0.a, cm.a, c1.a, l0, c0.b);
            d0.b = dpoint(xa + 1, ybase, rl_base, c0.b, cm.b, c1.b, c0.a, r0);
        }
        C* drow = dring;                                   // input row 2 -> D ring row 0
        st2(drow + k, d0);
        if (t == 0) drow[1] = dpoint(x0 - 1, ybase, rl_base, l0, q1[1], q3[1], q2[0], c0.a);
        if (t == NT - 1) drow[TXC + 2] = dpoint(x0 + TXC, ybase, rl_base, r0, q1[TXC + 2], q3[TXC + 2], c0.b, q2[TXC + 3]);
    }
    __syncthreads();

    bool bad = false;
    int yl = rl_base;                            // instance row of y
    // Unrolled by 3, the period of the three-row register windows, so that
    // sliding them is register renaming rather than moves.
#pragma unroll 3
    for (int i = 0; i < TY; ++i) {
        if (!alive || i >= nrows) break;
        const int j = i + 2;                     // input row of y
        const int y = ybase + dir * i;
        const int ya = y + dir;                  // the row after y in walk order
        const int yla = rstep(yl, dir);
        wait_in(j + 2);
        if (!__syncthreads_and(ok)) { alive = false; break; }
        if (t == PIN && next < jmax) issue_in(next++);
        if (NEED_E && t == PE && enext < nrows) issue_e(enext++);

        // D(., ya), one row ahead.
        const C* q1 = irow(j + 1);
        const C* q2 = irow(j + 2);
        const T2 c2 = ld2(q2 + k);
        const C l1 = q1[k - 1], r1 = q1[k + 2];
        T2 d1, dx1, h1;
        C* dn = dring + ((j + 1) & 1) * L::ROW;
        if constexpr (MS) {
            const Two<C> pa = ms_point(xa, ya, yla, c1.a, c0.a, c2.a, l1, c1.b);
            const Two<C> pb = ms_point(xa + 1, ya, yla, c1.b, c0.b, c2.b, c1.a, r1);
            dx1 = T2{pa.a, pb.a};
            d1 = T2{pa.b, pb.b};
            st2(dn + k, dx1);
            if (t == 0) dn[1] = ms_point(x0 - 1, ya, yla, l1, l0, q2[1], q1[0], c1.a).a;
            if (t == NT - 1) dn[TXC + 2] = ms_point(x0 + TXC, ya, yla, r1, r0, q2[TXC + 2], c1.b, q1[TXC + 3]).a;
        } else {
            if constexpr (KEEPH) {
                h1 = hpair(c1, l1, r1);
                d1.a = dpoint_h(xa, ya, yla, c1.a, c0.a, c2.a, h1.a);
                d1.b = dpoint_h(xa + 1, ya, yla, c1.b, c0.b, c2.b, h1.b);
            } else {
                d1.a = dpoint(xa, ya, yla, c1.a, c0.a, c2.a, l1, c1.b);
                d1.b = dpoint(xa + 1, ya, yla, c1.b, c0.b, c2.b, c1.a, r1);
            }
            st2(dn + k, d1);
            if (t == 0) dn[1] = dpoint(x0 - 1, ya, yla, l1, l0, q2[1], q1[0], c1.a);
            if (t == NT - 1) dn[TXC + 2] = dpoint(x0 + TXC, ya, yla, r1, r0, q2[TXC + 2], c1.b, q1[TXC + 3]);
        }
        // No barrier here: the step below reads the D ring slot written in the
        // previous iteration and this thread's own registers, both ordered by
        // the barrier at the top of the loop, and a thread whose wait gave up
        // carries ok = false to that barrier, where the CTA stops together.
        if (NEED_E) wait_e(i);

        if (xin && NLSE_IDX(io.flag, (int64_t)y * nx + xa + 1, (int64_t)nx * ny, kSiteTile2d)) {
            const C* dr = dring + (j & 1) * L::ROW;          // dr[k-1] = D(xa-1, y), dr[k+2] = D(xa+2, y)
            const bool rowb = !INNER && (yl == 0 || yl == io.rows1 - 1);
            const bool ba = !INNER && (rowb || xa == 0), bb = !INNER && (rowb || xa + 1 == nx - 1);
            T2 lap = d0;
            if constexpr (MS) {
                // dr holds D^x of row y; d0 / dm / d1 hold D^y of rows y, y -+ 1.
                const C sa = add2(add2(dr[k - 1], dx0.b), add2(dm.a, d1.a));
                const C sb = add2(add2(dx0.a, dr[k + 2]), add2(dm.b, d1.b));
                lap.a = fma2(c76, add2(dx0.a, d0.a), mul2(m12, sa));
                lap.b = fma2(c76, add2(dx0.b, d0.b), mul2(m12, sb));
                if (STAGE == 0) {
                    if (ba) lap.a = dirichlet_D(c, c0.a, vat(yl, xa));
                    if (bb) lap.b = dirichlet_D(c, c0.b, vat(yl, xa + 1));
                }
            } else if (!CD) {
                const C dsa = add2(add2(dr[k - 1], d0.b), add2(dm.a, d1.a));
                const C dsb = add2(add2(d0.a, dr[k + 2]), add2(dm.b, d1.b));
                // corners: the x-neighbour sums of rows y -+ 1
                C cna, cnb;
                if constexpr (KEEPH) {
                    cna = add2(hm.a, h1.a);
                    cnb = add2(hm.b, h1.b);
                } else {
                    cna = add2(add2(lm, cm.b), add2(l1, c1.b));
                    cnb = add2(add2(cm.a, rm), add2(c1.a, r1));
                }
                if (!ba) lap.a = fma2(i6h2, fma2(m4, c0.a, cna), fma2(m12, dsa, d0.a));
                if (!bb) lap.b = fma2(i6h2, fma2(m4, c0.b, cnb), fma2(m12, dsb, d0.b));
            }
            const int64_t p = (int64_t)y * nx + xa;
            if constexpr (STAGE == 0) {
                st2(io.lap + p, lap);
            } else {
                const unsigned char* es = erow(i);
                const R* vv = reinterpret_cast<const R*>(es + L::E_V) + 2 * t;
                // w = a Lap + (s|Psi|^2 - V) Psi; c F = (-c, c) * swap(w); F_b = 0.
                auto swapped_w = [&](C y_, C lap_, R v_, bool b_) -> C {
                    if (b_) return czero<C>();
                    const R N = nonlin(c.s, y_, v_);
                    const C w = SC ? fma2(pair<C>(N, N), y_, lap_) : fma2(pair<C>(N, N), y_, mul2(a2, lap_));
                    return pair<C>(w.y, w.x);
                };
                const C swa = swapped_w(c0.a, lap.a, vv[0], ba);
                const C swb = swapped_w(c0.b, lap.b, vv[1], bb);
                if constexpr (STAGE == 1) {
                    st2(io.acc + p, T2{mul2(ca2, swa), mul2(ca2, swb)});
                    st2(io.yout + p, T2{fma2(cy2, swa, c0.a), fma2(cy2, swb, c0.b)});
                } else {
                    const T2 pn = ld2(reinterpret_cast<const C*>(es + L::E_PSI) + 2 * t);
                    const T2 ac = ld2(reinterpret_cast<const C*>(es + L::E_ACC) + 2 * t);
                    if constexpr (STAGE == 2 || STAGE == 3) {
                        st2(io.acc + p, T2{fma2(ca2, swa, ac.a), fma2(ca2, swb, ac.b)});
                        st2(io.yout + p, T2{fma2(cy2, swa, pn.a), fma2(cy2, swb, pn.b)});
                    } else {
                        const C da = fma2(ca2, swa, ac.a), db = fma2(ca2, swb, ac.b);
                        T2 out = pn;
                        if constexpr (sizeof(R) == 4) {
                            T2 lo = ld2(reinterpret_cast<const C*>(es + L::E_LO) + 2 * t);
                            kahan_add(out.a.x, lo.a.x, da.x);
                            kahan_add(out.a.y, lo.a.y, da.y);
                            kahan_add(out.b.x, lo.b.x, db.x);
                            kahan_add(out.b.y, lo.b.y, db.y);
                            st2(io.lo + p, lo);
                        } else {
                            out.a = add2(out.a, da);
                            out.b = add2(out.b, db);
                        }
                        st2(io.psi_out + p, out);
                        bad |= !(isfinite(out.a.x) && isfinite(out.a.y) && isfinite(out.b.x) && isfinite(out.b.y));
                    }
                }
            }
        }
        lm = l0; rm = r0; l0 = l1; r0 = r1;
        cm = c0; c0 = c1; c1 = c2;
        dm = d0; d0 = d1;
        if constexpr (KEEPH) { hm = h0; h0 = h1; }
        if constexpr (MS) dx0 = dx1;
        yl = yla;
    }

    if (!alive) {
        // A transfer never arrived: report, let this CTA's copies in flight land, leave.
        if (t == 0) atomicOr(io.flag, 2);
        if (t == PIN)
            for (int j = next > S ? next - S : 0; j < next; ++j)
                mbar_wait(ibar0 + 8 * (j % S), (uint32_t)((j / S) & 1), kDrainNs);
        if (t == PE)
            for (int e = enext > 2 ? enext - 2 : 0; e < enext; ++e)
                mbar_wait(ebar0 + 8 * (e & 1), (uint32_t)((e >> 1) & 1), kDrainNs);
        return;
    }
    if constexpr (STAGE == 4) {
        if (__syncthreads_or(bad) && t == 0) atomicOr(io.flag, 1);
    }
}

// One CTA's walk.  In FP64, whose rate on this GPU bounds the walk, CTAs in
// which no point whose D the CTA forms (columns x0-1 .. x0+TXC, rows y0-1 ..
// y0+nrows) is a boundary point of its instance or lies outside the grid take
// the variant without per-point boundary tests (5% faster).  In FP32 the
// walk is bound by memory and latency; there the second variant gained
// nothing on single grids and cost 20% on batches, so FP32 has one.
template <typename R, int LP, int STAGE, int NT, int TY>
__device__ __forceinline__ void stage2d_tile(const CUtensorMap* m_in, const CUtensorMap* m_in2,
                                             const CUtensorMap* m_V, const CUtensorMap* m_psi,
                                             const CUtensorMap* m_acc, const CUtensorMap* m_lo,
                                             const StageIO<R>& io, const Coef<R>& c, const int nx, const int ny,
                                             const int x0, const int y0, const int dir) {
    if constexpr (STAGE == 4) {
        if (refused(io.flag)) return;              // before any barrier or copy
    }
    if constexpr (sizeof(R) == 4) {
        stage2d_walk<R, LP, STAGE, NT, TY, false>(m_in, m_in2, m_V, m_psi, m_acc, m_lo, io, c, nx, ny, x0, y0, dir);
    } else {
        const int ylo = y0 - 1, yhi = y0 + min(TY, ny - y0);
        const bool inner = x0 >= 2 && x0 + 2 * NT <= nx - 2 && ylo >= 1 && yhi <= ny - 2 &&
                           ylo / io.rows1 == yhi / io.rows1 && ylo % io.rows1 >= 1 &&
                           yhi % io.rows1 <= io.rows1 - 2;
        if (inner)
            stage2d_walk<R, LP, STAGE, NT, TY, true>(m_in, m_in2, m_V, m_psi, m_acc, m_lo, io, c, nx, ny, x0, y0,
                                                     dir);
        else
            stage2d_walk<R, LP, STAGE, NT, TY, false>(m_in, m_in2, m_V, m_psi, m_acc, m_lo, io, c, nx, ny, x0, y0,
                                                      dir);
    }
}

}  // namespace tile2d
}  // namespace nlse
