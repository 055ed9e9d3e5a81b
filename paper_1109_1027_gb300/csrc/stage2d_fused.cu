// stage2d_fused.cu -- temporal blocking of the 2D RK4 step: two stages per
// launch (stages 1+2, then 3+4), so that the intermediate stage input Y_s
// never leaves the SM.
//
// Eq. (RK4) makes stage s+1 at a point depend on Y_s at the point and its two
// neighbours along each axis (the 2SHOC stencil reads Y_s at distance 2:
// step 1 at distance 1, step 2 at distance 1 of D).  So a CTA that is to
// produce stage B = s+1 on a TXC x TY block produces stage A = s on the block
// widened by 2 points on each side, from its input widened by 4.  The CTA
// walks its block row by row like the single-stage walk (stage2d_tile.cuh):
//   * stage A runs 5 rows ahead of stage B.  Its input rows (264 points:
//     columns x0-4 .. x0+TXC+3) come through a TMA ring, its D through a
//     two-row shared ring, and each output row Y_A (260 points) goes into a
//     shared ring of 5 rows that is stage B's input;
//   * stage B is the single-stage walk reading that ring instead of global
//     memory, and writes the step's arrays;
//   * F of stage A at the block's own points waits for stage B in a per-thread
//     shared fifo (the accumulated increment of stage A is formed from it when
//     stage B runs, with the same roundings as the separate launches);
//   * the 6 extra columns of D_A, the 4 extra columns of Y_A and the 2 extra
//     columns of D_B are computed by a fifth warp, one column per lane, which
//     also issues the TMA copies.
// Per update this moves 28 B for stages 1+2 (read Psi^n, V; write acc, Y_2)
// and 52 B for stages 3+4 (read Y_2, V, Psi^n, acc, lo; write Psi^n+1, lo):
// 80 B per RK4 step instead of 168.  The redundant work is the 4 extra rows
// and 4 extra columns of stage A per block.
//
// Every point value goes through the same operations in the same order as in
// the single-stage kernel (packed f32x2 instructions and explicitly rounded
// intrinsics, which the compiler cannot fuse or reorder), so the two paths
// give identical bits.  FP32 with the compensated state only; Dirichlet
// boundaries (single grids and stacks); the single-storage 2SHOC and CD.
// Every mbarrier wait is bounded (1 s): on timeout the CTA sets bit 2 of the
// status flag, lets its copies in flight land and returns.
#include "nlse_internal.h"
#include "stage2d_tile.cuh"
#include "tmap.cuh"

#include <mutex>

namespace nlse {
namespace fused2d {

using tile2d::al128;
using tile2d::ld2;
using tile2d::pair;
using tile2d::st2;
using tile2d::Two;
using C = float2;
using T2 = Two<float2>;

constexpr int NT = 128;            // main threads, two columns each
constexpr int NTH = NT + 32;       // plus the edge-column warp
constexpr int TXC = 2 * NT;        // output columns per CTA
constexpr int W = TXC + 8;         // row buffers hold columns x0-4 .. x0+TXC+3
constexpr int SA = 6;              // stage-A input ring
constexpr int SY = 5;              // ring of stage-A outputs (stage-B inputs)
constexpr int LAG = 5;             // stage B's first row runs this many iterations after stage A's
constexpr int NF = 4;              // slots of the F_A fifo
constexpr int PRODUCER = NTH - 1;  // last lane of the edge warp issues the copies
constexpr uint64_t kWaitNs = tile2d::kWaitNs;
constexpr uint64_t kDrainNs = tile2d::kDrainNs;

// Shared-memory layout.  Row buffers are indexed by x - (x0 - 4): a main
// thread's column pair sits at 2t + 4 (16-byte aligned).  TMA destinations
// are 128-byte aligned.
template <int PAIR>
struct Lay {
    static constexpr int ROWB = al128(W * 8);          // complex row with halo
    static constexpr int VROWB = al128(W * 4);         // real row with halo
    static constexpr int T = TXC * 8, TV = TXC * 4;    // rows of the block's own columns
    // Stage-A epilogue slot: V (W wide), stages 3+4 also Psi^n (W wide).
    static constexpr int EA_V = 0, EA_PSI = VROWB;
    static constexpr int EA_SLOT = PAIR ? VROWB + ROWB : VROWB;
    // Stage-B epilogue slot: Psi^n, V, and for stages 3+4 acc and lo.
    static constexpr int EB_PSI = 0, EB_V = T, EB_ACC = T + TV, EB_LO = 2 * T + TV;
    static constexpr int EB_SLOT = al128(PAIR ? 3 * T + TV : T + TV);
    static constexpr int IN_OFF = 0;
    static constexpr int Y_OFF = IN_OFF + SA * ROWB;
    static constexpr int EA_OFF = Y_OFF + SY * ROWB;
    static constexpr int EB_OFF = EA_OFF + 2 * EA_SLOT;
    static constexpr int DA_OFF = EB_OFF + 2 * EB_SLOT;
    static constexpr int DB_OFF = DA_OFF + 2 * W * 8;
    static constexpr int F_OFF = DB_OFF + 2 * W * 8;
    static constexpr int BAR_OFF = al128(F_OFF + NF * T);
    static constexpr int NBAR = SA + 4;                // input ring, 2 A epilogue, 2 B epilogue
    static constexpr int TOTAL = BAR_OFF + 8 * NBAR + 128;
};

// What the two stages write and their weights (Eq. RK4).
struct FusedIO {
    const float* V;
    C* acc;           // stages 1+2: acc after stage 2
    C* yout;          // stages 1+2: Y_2
    C* psi_out;       // stages 3+4: Psi^{n+1}
    C* lo;            // stages 3+4: compensated part (read through TMA, written here)
    int* flag;
    float ca_a, cy_a; // stage A: weight of F in acc and in Y_A
    float ca_b, cy_b; // stage B: weight of F in acc and in Y_B
    int keep_v;
    int rows1;
};

// D at grid point (x, r), rl its row within its instance (Eq. 2d2shocs1;
// boundary: Eq. dbc_lap; outside the grid: 0, never used).  The same
// operations as the single-stage walk.
__device__ __forceinline__ C dpt(const Coef<float>& c, const FusedIO& io, int nx, int ny, int x, int r, int rl,
                                 C ctr, C up, C dn, C lf, C rt) {
    if (x < 0 || x >= nx || r < 0 || r >= ny) return czero<C>();
    if (x == 0 || x == nx - 1 || rl == 0 || rl == io.rows1 - 1)
        return NLSE_IDX(io.flag, (int64_t)rl * nx + x, (int64_t)io.rows1 * nx, kSiteFused)
                   ? dirichlet_D(c, ctr, io.V[(int64_t)rl * nx + x]) : czero<C>();
    return mul2(fma2(pair<C>(-4, -4), ctr, add2(add2(lf, rt), add2(up, dn))), pair<C>(c.inv_h2, c.inv_h2));
}

// Step 2 at an interior point (Eq. 2d2shocs2): ctr and d the point's value
// and D, dl / dr the D of its x-neighbours, dp / dn those of the previous and
// next rows, cpl, cpr / cnl, cnr the corner values of the previous / next row.
// CD (LP = 1): Lap = D.
template <int LP>
__device__ __forceinline__ C lap_pt(const Coef<float>& c, C ctr, C d, C dl, C dr, C dp, C dn, C cpl, C cpr,
                                    C cnl, C cnr) {
    if constexpr (LP == 1) {
        return d;
    } else {
        const C ds = add2(add2(dl, dr), add2(dp, dn));
        const C cn = add2(add2(cpl, cpr), add2(cnl, cnr));
        return fma2(pair<C>(c.inv_6h2, c.inv_6h2), fma2(pair<C>(-4, -4), ctr, cn),
                    fma2(pair<C>((float)(-1.0 / 12.0), (float)(-1.0 / 12.0)), ds, d));
    }
}

// (a Lap + N y) with its parts swapped, so that (-c, c) * it is c i(...) =
// c F (Sec. 3.1); 0 at boundary points (Eq. dbc_ut).
__device__ __forceinline__ C swapped_w(const Coef<float>& c, C y, C lap, float v, bool b) {
    if (b) return czero<C>();
    const float N = nonlin(c.s, y, v);
    const C w = fma2(pair<C>(N, N), y, mul2(pair<C>(c.a, c.a), lap));
    return pair<C>(w.y, w.x);
}

__device__ __forceinline__ int rstep(int rl, int d, int rows1) {
    rl += d;
    return rl < 0 ? rows1 - 1 : (rl == rows1 ? 0 : rl);
}

// PAIR 0: stages 1+2; PAIR 1: stages 3+4.  LP 0: 2SHOC, 1: CD.
template <int LP, int PAIR>
__global__ void __launch_bounds__(NTH, 3)
rk4_2d_fused_kernel(const __grid_constant__ CUtensorMap m_in, const __grid_constant__ CUtensorMap m_in8,
                    const __grid_constant__ CUtensorMap m_v, const __grid_constant__ CUtensorMap m_v8,
                    const __grid_constant__ CUtensorMap m_psi, const __grid_constant__ CUtensorMap m_psi8,
                    const __grid_constant__ CUtensorMap m_acc, const __grid_constant__ CUtensorMap m_lo,
                    const FusedIO io, const Coef<float> c, const int nx, const int ny, const int ty,
                    const int dir) {
    using L = Lay<PAIR>;
    if constexpr (PAIR == 1) {
        if (refused(io.flag)) return;              // stages 3+4 write the state; before any barrier or copy
    }
    extern __shared__ unsigned char smem_raw[];
    unsigned char* smem = smem_raw + ((128 - (smem_u32(smem_raw) & 127)) & 127);
    const uint32_t sbase = smem_u32(smem);
    const uint32_t bar0 = sbase + L::BAR_OFF;          // SA input, 2 A-epilogue, 2 B-epilogue

    const int t = threadIdx.x;
    const int x0 = blockIdx.x * TXC, y0 = blockIdx.y * ty;
    const int nrows = min(ty, ny - y0);
    const int nA = nrows + 4;                          // stage-A output rows q = 0 .. nA-1
    const int mA = nA + 4;                             // stage-A input rows m = 0 .. mA-1
    // Walk order: stage-B output row e is grid row ybase + dir e; stage-A
    // output row q (= stage-B input row j) is ybase + dir (q - 2); stage-A
    // input row m is ybase + dir (m - 4).
    const int ybase = dir > 0 ? y0 : y0 + nrows - 1;
    const int rows1 = io.rows1;
    const int rl_base = ybase % rows1;                 // row within its instance
    const int rl_q0 = ((ybase - 2 * dir) % rows1 + rows1) % rows1;

    if (t == PRODUCER) {
        tma_prefetch_desc(&m_in);
        tma_prefetch_desc(&m_v);
        for (int s = 0; s < L::NBAR; ++s) mbar_init(bar0 + 8 * s, 1);
        mbar_init_fence();
    }
    __syncthreads();

    // ---- producer (one lane of the edge warp) ----------------------------
    uint64_t pol = 0;
    if (io.keep_v && t == PRODUCER) pol = l2_evict_last();
    auto load_v = [&](uint32_t dst, const CUtensorMap* m, int x, int r, uint32_t bar) {
        if (io.keep_v) tma_load_2d_hint(dst, m, x, r, bar, pol);
        else tma_load_2d(dst, m, x, r, bar);
    };
    auto issue_in = [&](int m) {
        const uint32_t dst = sbase + L::IN_OFF + (m % SA) * L::ROWB;
        const uint32_t bar = bar0 + 8 * (m % SA);
        const int r = ybase + dir * (m - 4);
        mbar_expect_tx(bar, W * 8);
        tma_load_2d(dst, &m_in, x0 - 4, r, bar);
        tma_load_2d(dst + TXC * 8, &m_in8, x0 + TXC - 4, r, bar);
    };
    int ea_rl = rl_q0;                                 // instance row of the next A-epilogue row
    int ea_n = 0, eb_n = 0;                            // epilogue rows issued
    auto issue_ea = [&](int q) {
        const uint32_t dst = sbase + L::EA_OFF + (q & 1) * L::EA_SLOT;
        const uint32_t bar = bar0 + 8 * (SA + (q & 1));
        const int r = ybase + dir * (q - 2);
        mbar_expect_tx(bar, W * 4 + (PAIR ? W * 8 : 0));
        load_v(dst + L::EA_V, &m_v, x0 - 4, ea_rl, bar);
        load_v(dst + L::EA_V + TXC * 4, &m_v8, x0 + TXC - 4, ea_rl, bar);
        if (PAIR) {
            tma_load_2d(dst + L::EA_PSI, &m_psi, x0 - 4, r, bar);
            tma_load_2d(dst + L::EA_PSI + TXC * 8, &m_psi8, x0 + TXC - 4, r, bar);
        }
        ea_rl = rstep(ea_rl, dir, rows1);
        ++ea_n;
    };
    int eb_rl = rl_base;
    auto issue_eb = [&](int e) {
        const uint32_t dst = sbase + L::EB_OFF + (e & 1) * L::EB_SLOT;
        const uint32_t bar = bar0 + 8 * (SA + 2 + (e & 1));
        const int r = ybase + dir * e;
        mbar_expect_tx(bar, TXC * 8 + TXC * 4 + (PAIR ? 2 * TXC * 8 : 0));
        // Psi^n again (stage A read it a few rows earlier: an L2 hit).
        tma_load_2d(dst + L::EB_PSI, PAIR ? &m_psi : &m_in, x0, r, bar);
        load_v(dst + L::EB_V, &m_v, x0, eb_rl, bar);
        if (PAIR) {
            tma_load_2d(dst + L::EB_ACC, &m_acc, x0, r, bar);
            tma_load_2d(dst + L::EB_LO, &m_lo, x0, r, bar);
        }
        eb_rl = rstep(eb_rl, dir, rows1);
        ++eb_n;
    };
    int next_in = 0;
    if (t == PRODUCER) {
        for (; next_in < SA && next_in < mA; ++next_in) issue_in(next_in);
        issue_ea(0);
    }

    auto inrow = [&](int m) { return reinterpret_cast<const C*>(smem + L::IN_OFF + (m % SA) * L::ROWB); };
    auto yrow = [&](int q) { return reinterpret_cast<C*>(smem + L::Y_OFF + (q % SY) * L::ROWB); };
    auto darow = [&](int q) { return reinterpret_cast<C*>(smem + L::DA_OFF + (q & 1) * W * 8); };
    auto dbrow = [&](int j) { return reinterpret_cast<C*>(smem + L::DB_OFF + (j & 1) * W * 8); };
    auto fifo = [&](int q) { return reinterpret_cast<C*>(smem + L::F_OFF + (q & (NF - 1)) * L::T); };
    auto earow = [&](int q) { return smem + L::EA_OFF + (q & 1) * L::EA_SLOT; };
    auto ebrow = [&](int e) { return smem + L::EB_OFF + (e & 1) * L::EB_SLOT; };

    bool ok = true;
    auto wait_in = [&](int m) {
        if (ok) ok = mbar_wait(bar0 + 8 * (m % SA), (uint32_t)((m / SA) & 1), kWaitNs);
    };
    auto wait_ea = [&](int q) {
        if (ok) ok = mbar_wait(bar0 + 8 * (SA + (q & 1)), (uint32_t)((q >> 1) & 1), kWaitNs);
    };
    auto wait_eb = [&](int e) {
        if (ok) ok = mbar_wait(bar0 + 8 * (SA + 2 + (e & 1)), (uint32_t)((e >> 1) & 1), kWaitNs);
    };

    const bool main_t = t < NT;
    const int lane = t - NT;                           // edge warp lane
    // Main threads: columns xa, xa + 1 at buffer index k.  Edge lanes 0..5:
    // column xh at index kh (x0-3, x0-2, x0-1, x0+TXC, x0+TXC+1, x0+TXC+2).
    const int xa = x0 + 2 * t, k = 2 * t + 4;
    const bool xin = xa < nx;
    const int kh = lane < 3 ? 1 + lane : TXC + 1 + lane;
    const int xh = x0 - 4 + kh;
    const bool h_da = !main_t && lane < 6;             // D_A at xh
    const bool h_ya = !main_t && lane >= 1 && lane < 5;  // Y_A at xh
    const bool h_db = !main_t && (lane == 2 || lane == 3);  // D_B at xh

    const C ca_a2 = pair<C>(-io.ca_a, io.ca_a), cy_a2 = pair<C>(-io.cy_a, io.cy_a);
    const C ca_b2 = pair<C>(-io.ca_b, io.ca_b), cy_b2 = pair<C>(-io.cy_b, io.cy_b);

    // Stage-A register windows (main: two columns; edge lanes: D of one column).
    T2 aCm, aC0, aC1, aDm, aD0;
    C aLm, aRm, aL0, aR0;
    C hDm = czero<C>(), hD0 = czero<C>();
    // Stage-B windows.
    T2 bCm, bC0, bC1, bDm, bD0;
    C bLm, bRm, bL0, bR0;
    int rlA = rl_q0;                                   // instance row of A output row qa
    int rlB = rl_base;                                 // instance row of B output row ib

    // Stage-A prologue: input rows 0..3 give D_A of output rows -1 and 0.
    wait_in(0); wait_in(1); wait_in(2); wait_in(3);
    bool alive = __syncthreads_and(ok);
    if (alive) {
        const C* p0 = inrow(0); const C* p1 = inrow(1); const C* p2 = inrow(2); const C* p3 = inrow(3);
        const int r0 = ybase - 2 * dir, rm1 = r0 - dir;
        const int rlm1 = rstep(rl_q0, -dir, rows1);
        if (main_t) {
            const T2 cmm = ld2(p0 + k);
            aCm = ld2(p1 + k); aC0 = ld2(p2 + k); aC1 = ld2(p3 + k);
            aLm = p1[k - 1]; aRm = p1[k + 2];
            aL0 = p2[k - 1]; aR0 = p2[k + 2];
            aDm.a = dpt(c, io, nx, ny, xa, rm1, rlm1, aCm.a, cmm.a, aC0.a, aLm, aCm.b);
            aDm.b = dpt(c, io, nx, ny, xa + 1, rm1, rlm1, aCm.b, cmm.b, aC0.b, aCm.a, aRm);
            aD0.a = dpt(c, io, nx, ny, xa, r0, rl_q0, aC0.a, aCm.a, aC1.a, aL0, aC0.b);
            aD0.b = dpt(c, io, nx, ny, xa + 1, r0, rl_q0, aC0.b, aCm.b, aC1.b, aC0.a, aR0);
            st2(darow(0) + k, aD0);
        } else if (h_da) {
            hDm = dpt(c, io, nx, ny, xh, rm1, rlm1, p1[kh], p0[kh], p2[kh], p1[kh - 1], p1[kh + 1]);
            hD0 = dpt(c, io, nx, ny, xh, r0, rl_q0, p2[kh], p1[kh], p3[kh], p2[kh - 1], p2[kh + 1]);
            darow(0)[kh] = hD0;
        }
    }

    bool bad = false;
    const int nit = nA + LAG - 1;                      // B's last row runs at nrows - 1 + LAG
    for (int it = 0; it <= nit; ++it) {
        if (!alive) break;
        const int qa = it;
        const bool a_on = qa < nA;
        if (a_on) wait_in(qa + 4);
        if (!__syncthreads_and(ok)) { alive = false; break; }
        if (t == PRODUCER) {
            if (a_on && next_in < mA) issue_in(next_in++);
            if (qa + 1 < nA) issue_ea(qa + 1);
            if (it >= LAG - 1 && it - (LAG - 1) < nrows) issue_eb(it - (LAG - 1));
        }

        // ---- stage A: D_A of output row qa+1, then Y_A of row qa ----------
        if (a_on) {
            const int rA = ybase + dir * (qa - 2), rA1 = rA + dir;
            const int rlA1 = rstep(rlA, dir, rows1);
            const bool rowin = rA >= 0 && rA < ny;
            const bool rowb = rlA == 0 || rlA == rows1 - 1;
            if (main_t) {
                const C* q1 = inrow(qa + 3);
                const C* q2 = inrow(qa + 4);
                const T2 c2 = ld2(q2 + k);
                const C l1 = q1[k - 1], r1 = q1[k + 2];
                T2 d1;
                d1.a = dpt(c, io, nx, ny, xa, rA1, rlA1, aC1.a, aC0.a, c2.a, l1, aC1.b);
                d1.b = dpt(c, io, nx, ny, xa + 1, rA1, rlA1, aC1.b, aC0.b, c2.b, aC1.a, r1);
                st2(darow(qa + 1) + k, d1);
                wait_ea(qa);
                const C* dr = darow(qa);
                const unsigned char* ea = earow(qa);
                const float* vv = reinterpret_cast<const float*>(ea + L::EA_V) + k;
                const bool ba = rowb || xa == 0, bb = rowb || xa + 1 == nx - 1;
                T2 lap = aD0;
                if (!ba) lap.a = lap_pt<LP>(c, aC0.a, aD0.a, dr[k - 1], aD0.b, aDm.a, d1.a, aLm, aCm.b, l1, aC1.b);
                if (!bb) lap.b = lap_pt<LP>(c, aC0.b, aD0.b, aD0.a, dr[k + 2], aDm.b, d1.b, aCm.a, aRm, aC1.a, r1);
                const C swa = swapped_w(c, aC0.a, lap.a, vv[0], ba);
                const C swb = swapped_w(c, aC0.b, lap.b, vv[1], bb);
                T2 base = aC0;                       // stage 1: Y_1 = Psi^n + k/2 F (Psi^n is the input)
                if constexpr (PAIR == 1) base = ld2(reinterpret_cast<const C*>(ea + L::EA_PSI) + k);
                T2 ya{fma2(cy_a2, swa, base.a), fma2(cy_a2, swb, base.b)};
                if (!(rowin && xin)) ya = T2{czero<C>(), czero<C>()};
                st2(yrow(qa) + k, ya);
                st2(fifo(qa) + 2 * t, T2{swa, swb});
                aLm = aL0; aRm = aR0; aL0 = l1; aR0 = r1;
                aCm = aC0; aC0 = aC1; aC1 = c2;
                aDm = aD0; aD0 = d1;
            } else {
                const C* q0 = inrow(qa + 1);
                const C* q1 = inrow(qa + 2);
                const C* q2 = inrow(qa + 3);
                const C* q3 = inrow(qa + 4);
                C hD1 = czero<C>();
                if (h_da) {
                    hD1 = dpt(c, io, nx, ny, xh, rA1, rlA1, q2[kh], q1[kh], q3[kh], q2[kh - 1], q2[kh + 1]);
                    darow(qa + 1)[kh] = hD1;
                }
                wait_ea(qa);
                if (h_ya) {
                    const C* dr = darow(qa);
                    const unsigned char* ea = earow(qa);
                    const float v = reinterpret_cast<const float*>(ea + L::EA_V)[kh];
                    const bool b = rowb || xh == 0 || xh == nx - 1;
                    const C ctr = q1[kh];
                    const C lap = b ? hD0 : lap_pt<LP>(c, ctr, hD0, dr[kh - 1], dr[kh + 1], hDm, hD1, q0[kh - 1],
                                                       q0[kh + 1], q2[kh - 1], q2[kh + 1]);
                    const C sw = swapped_w(c, ctr, lap, v, b);
                    C base = ctr;
                    if constexpr (PAIR == 1) base = reinterpret_cast<const C*>(ea + L::EA_PSI)[kh];
                    C y = fma2(cy_a2, sw, base);
                    if (!(rowin && xh >= 0 && xh < nx)) y = czero<C>();
                    yrow(qa)[kh] = y;
                }
                hDm = hD0; hD0 = hD1;
            }
            rlA = rlA1;
        }

        // ---- stage B -------------------------------------------------------
        if (it == LAG - 1) {
            // Prologue: stage-A rows 0..3 give D_B of input rows 1 and 2.
            const C* p0 = yrow(0); const C* p1 = yrow(1); const C* p2 = yrow(2); const C* p3 = yrow(3);
            const int yb = ybase - dir;
            const int rlb = rstep(rl_base, -dir, rows1);
            if (main_t) {
                const T2 cmm = ld2(p0 + k);
                bCm = ld2(p1 + k); bC0 = ld2(p2 + k); bC1 = ld2(p3 + k);
                bLm = p1[k - 1]; bRm = p1[k + 2];
                bL0 = p2[k - 1]; bR0 = p2[k + 2];
                bDm.a = dpt(c, io, nx, ny, xa, yb, rlb, bCm.a, cmm.a, bC0.a, bLm, bCm.b);
                bDm.b = dpt(c, io, nx, ny, xa + 1, yb, rlb, bCm.b, cmm.b, bC0.b, bCm.a, bRm);
                bD0.a = dpt(c, io, nx, ny, xa, ybase, rl_base, bC0.a, bCm.a, bC1.a, bL0, bC0.b);
                bD0.b = dpt(c, io, nx, ny, xa + 1, ybase, rl_base, bC0.b, bCm.b, bC1.b, bC0.a, bR0);
                st2(dbrow(2) + k, bD0);
            } else if (h_db) {
                dbrow(2)[kh] = dpt(c, io, nx, ny, xh, ybase, rl_base, p2[kh], p1[kh], p3[kh], p2[kh - 1], p2[kh + 1]);
            }
        } else if (it >= LAG && it - LAG < nrows) {
            const int ib = it - LAG, j = ib + 2;
            const int y = ybase + dir * ib, ya = y + dir;
            const int rly = rlB, rlya = rstep(rlB, dir, rows1);
            const C* q1 = yrow(j + 1);
            const C* q2 = yrow(j + 2);
            if (main_t) {
                const T2 c2 = ld2(q2 + k);
                const C l1 = q1[k - 1], r1 = q1[k + 2];
                T2 d1;
                d1.a = dpt(c, io, nx, ny, xa, ya, rlya, bC1.a, bC0.a, c2.a, l1, bC1.b);
                d1.b = dpt(c, io, nx, ny, xa + 1, ya, rlya, bC1.b, bC0.b, c2.b, bC1.a, r1);
                st2(dbrow(j + 1) + k, d1);
                wait_eb(ib);
                if (xin && NLSE_IDX(io.flag, (int64_t)y * nx + xa + 1, (int64_t)nx * ny, kSiteFused)) {
                    const C* dr = dbrow(j);
                    const bool rowb = rly == 0 || rly == rows1 - 1;
                    const bool ba = rowb || xa == 0, bb = rowb || xa + 1 == nx - 1;
                    T2 lap = bD0;
                    if (!ba) lap.a = lap_pt<LP>(c, bC0.a, bD0.a, dr[k - 1], bD0.b, bDm.a, d1.a, bLm, bCm.b, l1, bC1.b);
                    if (!bb) lap.b = lap_pt<LP>(c, bC0.b, bD0.b, bD0.a, dr[k + 2], bDm.b, d1.b, bCm.a, bRm, bC1.a, r1);
                    const unsigned char* eb = ebrow(ib);
                    const float* vv = reinterpret_cast<const float*>(eb + L::EB_V) + 2 * t;
                    const C swa = swapped_w(c, bC0.a, lap.a, vv[0], ba);
                    const C swb = swapped_w(c, bC0.b, lap.b, vv[1], bb);
                    const T2 sA = ld2(fifo(j) + 2 * t);
                    const T2 pn = ld2(reinterpret_cast<const C*>(eb + L::EB_PSI) + 2 * t);
                    const int64_t p = (int64_t)y * nx + xa;
                    if constexpr (PAIR == 0) {
                        // acc after stage 1 (k/6 F_1), then stage 2.
                        const C a1a = mul2(ca_a2, sA.a), a1b = mul2(ca_a2, sA.b);
                        st2(io.acc + p, T2{fma2(ca_b2, swa, a1a), fma2(ca_b2, swb, a1b)});
                        st2(io.yout + p, T2{fma2(cy_b2, swa, pn.a), fma2(cy_b2, swb, pn.b)});
                    } else {
                        const T2 ac = ld2(reinterpret_cast<const C*>(eb + L::EB_ACC) + 2 * t);
                        const C a3a = fma2(ca_a2, sA.a, ac.a), a3b = fma2(ca_a2, sA.b, ac.b);
                        const C da = fma2(ca_b2, swa, a3a), db = fma2(ca_b2, swb, a3b);
                        T2 lo = ld2(reinterpret_cast<const C*>(eb + L::EB_LO) + 2 * t);
                        T2 out = pn;
                        kahan_add(out.a.x, lo.a.x, da.x);
                        kahan_add(out.a.y, lo.a.y, da.y);
                        kahan_add(out.b.x, lo.b.x, db.x);
                        kahan_add(out.b.y, lo.b.y, db.y);
                        st2(io.lo + p, lo);
                        st2(io.psi_out + p, out);
                        bad |= !(isfinite(out.a.x) && isfinite(out.a.y) && isfinite(out.b.x) && isfinite(out.b.y));
                    }
                }
                bLm = bL0; bRm = bR0; bL0 = l1; bR0 = r1;
                bCm = bC0; bC0 = bC1; bC1 = c2;
                bDm = bD0; bD0 = d1;
            } else if (h_db) {
                const C* q0 = yrow(j);
                dbrow(j + 1)[kh] = dpt(c, io, nx, ny, xh, ya, rlya, q1[kh], q0[kh], q2[kh], q1[kh - 1], q1[kh + 1]);
            }
            rlB = rlya;
        }
    }

    if (!alive) {
        // A transfer never arrived: report, let this CTA's copies in flight land, leave.
        if (t == PRODUCER) {
            atomicOr(io.flag, 2);
            for (int m = next_in > SA ? next_in - SA : 0; m < next_in; ++m)
                mbar_wait(bar0 + 8 * (m % SA), (uint32_t)((m / SA) & 1), kDrainNs);
            for (int q = ea_n > 2 ? ea_n - 2 : 0; q < ea_n; ++q)
                mbar_wait(bar0 + 8 * (SA + (q & 1)), (uint32_t)((q >> 1) & 1), kDrainNs);
            for (int e = eb_n > 2 ? eb_n - 2 : 0; e < eb_n; ++e)
                mbar_wait(bar0 + 8 * (SA + 2 + (e & 1)), (uint32_t)((e >> 1) & 1), kDrainNs);
        }
        return;
    }
    if constexpr (PAIR == 1) {
        if (__syncthreads_or(bad) && t == 0) atomicOr(io.flag, 1);
    }
}

// ---- host side ---------------------------------------------------------------

template <int LP, int PAIR>
int blocks_per_sm() {
    static int n = -1;
    static std::once_flag once;
    std::call_once(once, [] {
        auto kern = rk4_2d_fused_kernel<LP, PAIR>;
        const int smem = Lay<PAIR>::TOTAL;
        if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) != cudaSuccess) {
            n = 0;
            return;
        }
        int b = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, kern, NTH, smem) != cudaSuccess) b = 0;
        n = b;
    });
    return n;
}

int sm_count() {
    static int n = 0;
    static std::once_flag once;
    std::call_once(once, [] {
        int dev = 0;
        if (cudaGetDevice(&dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
            n = 0;
    });
    return n;
}

template <int LP, int PAIR>
cudaError_t launch_t(const StageLaunch& L, cudaStream_t st) {
    const int nx = (int)L.n[0], ny = (int)L.n[1];
    const int rows1 = (int)(L.rows1 ? L.rows1 : ny);
    const void* yin = PAIR ? L.yin : L.psi;
    CUtensorMap m_in, m_in8, m_v, m_v8, m_psi, m_psi8, m_acc, m_lo;
    if (!complex_map<float>(&m_in, yin, nx, ny, TXC) || !complex_map<float>(&m_in8, yin, nx, ny, 8) ||
        !real_map<float>(&m_v, L.V, nx, rows1, TXC) || !real_map<float>(&m_v8, L.V, nx, rows1, 8))
        return cudaErrorInvalidValue;
    m_psi = m_psi8 = m_acc = m_lo = m_in;
    if (PAIR) {
        if (!complex_map<float>(&m_psi, L.psi, nx, ny, TXC) || !complex_map<float>(&m_psi8, L.psi, nx, ny, 8) ||
            !complex_map<float>(&m_acc, L.acc, nx, ny, TXC) || !complex_map<float>(&m_lo, L.lo, nx, ny, TXC))
            return cudaErrorInvalidValue;
    }
    const int per_sm = blocks_per_sm<LP, PAIR>();
    const int nsm = sm_count();
    if (per_sm <= 0 || nsm <= 0) return cudaErrorInvalidConfiguration;
    // Rows per CTA: the grid as one wave of resident CTAs, and at least 8.
    const int strips = (nx + TXC - 1) / TXC;
    const int per_strip = std::max(1, nsm * per_sm / strips);
    const int ty = std::max(8, (ny + per_strip - 1) / per_strip);

    FusedIO io;
    io.V = (const float*)L.V;
    io.acc = (C*)L.acc;
    io.yout = (C*)L.yout;
    io.psi_out = (C*)L.psi_out;
    io.lo = (C*)L.lo;
    io.flag = L.flag;
    const double kk = L.dt;
    // The stage weights of Eq. (RK4), rounded as the single-stage launches round them.
    io.ca_a = (float)(PAIR ? kk / 3.0 : kk / 6.0);
    io.cy_a = (float)(PAIR ? kk : kk / 2.0);
    io.ca_b = (float)(PAIR ? kk / 6.0 : kk / 3.0);
    io.cy_b = (float)(PAIR ? 0.0 : kk / 2.0);
    io.keep_v = L.keep_v;
    io.rows1 = rows1;
    dim3 grid(strips, (ny + ty - 1) / ty);
    const int dir = PAIR ? -1 : 1;
    rk4_2d_fused_kernel<LP, PAIR><<<grid, NTH, Lay<PAIR>::TOTAL, st>>>(
        m_in, m_in8, m_v, m_v8, m_psi, m_psi8, m_acc, m_lo, io, make_coef<float>(L.h, L.a, L.s), nx, ny, ty, dir);
    return cudaGetLastError();
}

}  // namespace fused2d

bool rk4_2d_fused_eligible(const StageLaunch& L) {
    return L.dim == 2 && L.prec == 0 && (L.lap == 0 || L.lap == 1) && stage_2d_tma_eligible(L);
}

cudaError_t launch_rk4_2d_fused(const StageLaunch& L, int pair, cudaStream_t st) {
    if (L.lap == 0) return pair ? fused2d::launch_t<0, 1>(L, st) : fused2d::launch_t<0, 0>(L, st);
    return pair ? fused2d::launch_t<1, 1>(L, st) : fused2d::launch_t<1, 0>(L, st);
}

}  // namespace nlse
