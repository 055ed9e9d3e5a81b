// stage3d_tma.cuh -- the fused 3D RK4 stage (and standalone 2SHOC Laplacian) in
// FP32 as a z-streaming kernel fed by the tensor memory accelerator.
//
// One CTA of 256 threads owns a TX x TY = 32 x 16 column of the grid (two
// x-adjacent points per thread) and walks TZ planes along z (TZ a tiling
// choice, 32, 64 or 128; each in its own translation unit
// stage3d_tma_z{32,64,128}.cu).  Two rings of
// shared-memory plane slots are filled by TMA tile loads, each completing on
// its own mbarrier:
//   * the input ring (S slots): the stage-input plane with a 2-point xy halo
//     (one 36 x 20 box);
//   * the epilogue ring (2 slots, one output plane ahead): V, and for stages
//     2-4 Psi^n and the RK4 accumulator (stage 4: the compensated part too).
// Each thread keeps its two columns' stage input and D along z in registers
// (planes z-1 .. z+2); in-plane neighbours come from the rings.  D of the
// plane ahead is written to a two-plane shared ring, with its 96-point xy
// halo computed by warps 0-2.  Per output plane z:
//   step 1 (Eq. 3d2shocs): D = (sum of the six axial Psi - 6 Psi_c) / h^2,
//                          boundary points D_b of Eq. (dbc_lap);
//   step 2 (Eq. 3d2shocs2): Lap = (10/12) D_c - (1/12) sum of the six axial D
//                          + (1/(6h^2)) (sum of the twelve edge Psi - 12 Psi_c);
//   F = i[a Lap + (s|Psi|^2 - V) Psi] (Sec. 3.1), F_b = 0 (Eq. dbc_ut);
//   the RK4 stage epilogue (Eq. RK4, accumulated-increment form).
// With the multi-storage form (LP = 2), step 1 keeps the three second
// differences apart, Eq. (3d2shocMs1): D^z in the register window, D^x and
// D^y in two shared rings (with the x and the y halo respectively), the
// Dirichlet D_b split over them at points on the boundary of one axis
// (D^a_b = D_b minus the other axes' second differences); step 2 is
// Eq. (3d2shocMs2): Lap = (7/6)(D^x + D^y + D^z)_c - (1/12)(the two axial
// neighbours of each D^a along its own axis).  Its step 2 reads no input
// plane, so a 4-slot input ring suffices and the two D rings fit.
// Consecutive stages walk z in opposite directions so that each starts on
// planes the previous one wrote last.  Every mbarrier wait is bounded (1 s);
// on timeout the CTA sets the timeout bit of the status, lets its copies land and
// returns.
#pragma once

#include "nlse_device.cuh"
#include "tma.cuh"
#include "tmap.cuh"

namespace nlse {
namespace tma3d {

constexpr int TX = 32, TY = 16;
constexpr int TXP = TX / 2;                  // thread columns (pairs)
constexpr int NT = TXP * TY;                 // 256 threads
constexpr int PW = TX + 4, PH = TY + 4;      // input plane with a 2-point halo (36 x 20)
constexpr uint64_t kWaitNs = 1000000000ull;
constexpr uint64_t kDrainNs = 50000000ull;

constexpr int al128(int v) { return (v + 127) / 128 * 128; }

// S input-ring slots, ND D-plane buffers.
template <int S, int ND>
struct Lay3 {
    static constexpr int CB = 8;                                  // complex64
    static constexpr int IN_BYTES = PW * PH * CB;                 // 5760
    static constexpr int IN_SLOT = al128(IN_BYTES);
    static constexpr int T_BYTES = TX * TY * CB;                  // 4096
    static constexpr int V_BYTES = TX * TY * 4;
    static constexpr int E_PSI = 0, E_ACC = T_BYTES, E_LO = 2 * T_BYTES, E_V = 3 * T_BYTES;
    static constexpr int E_SLOT = al128(E_V + V_BYTES);
    static constexpr int IN_OFF = 0;
    static constexpr int E_OFF = S * IN_SLOT;
    static constexpr int D_OFF = E_OFF + 2 * E_SLOT;              // D planes use the input-plane indexing
    static constexpr int BAR_OFF = al128(D_OFF + ND * IN_BYTES);
    static constexpr int TOTAL = BAR_OFF + 8 * (S + 2) + 128;
};

template <typename C> __device__ __forceinline__ C pair(float a, float b) { C z; z.x = a; z.y = b; return z; }

struct Two { float2 a, b; };
__device__ __forceinline__ Two ld2(const float2* p) {
    const float4 v = *reinterpret_cast<const float4*>(p);
    return {make_float2(v.x, v.y), make_float2(v.z, v.w)};
}
__device__ __forceinline__ void st2(float2* p, Two v) {
    *reinterpret_cast<float4*>(p) = make_float4(v.a.x, v.a.y, v.b.x, v.b.y);
}

// LP: 0 single-storage 2SHOC, 1 CD, 2 multi-storage 2SHOC.
template <int LP> struct Ring3 {
    static constexpr int S = LP == 2 ? 4 : 5;                     // input ring slots
    using L = Lay3<S, LP == 2 ? 4 : 2>;
};

template <int LP, int STAGE, int TZ>
__global__ void __launch_bounds__(NT, 3)      // three CTAs per SM (shared memory allows three)
stage3d_tma_kernel(const __grid_constant__ CUtensorMap m_in, const __grid_constant__ CUtensorMap m_V,
                   const __grid_constant__ CUtensorMap m_psi, const __grid_constant__ CUtensorMap m_acc,
                   const __grid_constant__ CUtensorMap m_lo, const StageIO<float> io, const Coef<float> c,
                   const int nx, const int ny, const int nz, const int dir) {
    using C = float2;
    constexpr bool CD = LP == 1, MS = LP == 2;
    constexpr int S = Ring3<LP>::S;
    using L = typename Ring3<LP>::L;
    constexpr bool NEED_E = STAGE >= 1;
    constexpr bool NEED_PA = STAGE >= 2;
    constexpr bool NEED_LO = STAGE == 4;
    extern __shared__ unsigned char smem_raw[];
    unsigned char* smem = smem_raw + ((128 - (smem_u32(smem_raw) & 127)) & 127);

    if constexpr (STAGE == 4) {
        if (refused(io.flag)) return;              // before any barrier or copy
    }
    const int t = threadIdx.x;
    const int tx = t % TXP, ty = t / TXP;
    const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY, z0 = blockIdx.z * TZ;
    const int nplanes = min(TZ, nz - z0);
    const int jmax = nplanes + 4;
    const int zbase = dir > 0 ? z0 : z0 + nplanes - 1;   // output plane e is zbase + dir * e
    const uint32_t sbase = smem_u32(smem);
    const uint32_t ibar0 = sbase + L::BAR_OFF, ebar0 = ibar0 + 8 * S;

#ifdef NLSE_BOUNDS_CHECK
    {
        // This thread's window in a plane buffer (k -+ PW -+ 1 .. 2) and its
        // halo slot, its epilogue slots, the tile origin, the TMA x
        // coordinates' 16-byte alignment and the dynamic shared memory given.
        const int kk = (ty + 2) * PW + 2 * tx + 2;
        int hkk = -1;
        if (t < TY) hkk = (t + 2) * PW + 1;
        else if (t < 2 * TY) hkk = (t - TY + 2) * PW + TX + 2;
        else if (t < 2 * TY + TX) hkk = PW + (t - 2 * TY) + 2;
        else if (t < 2 * TY + 2 * TX) hkk = (TY + 2) * PW + (t - 2 * TY - TX) + 2;
        uint32_t dyn;
        asm("mov.u32 %0, %%dynamic_smem_size;" : "=r"(dyn));
        const bool okb = NLSE_IDX(io.flag, kk - PW - 1, PW * PH, kSiteTma3d) &&
                         NLSE_IDX(io.flag, kk + PW + 2, PW * PH, kSiteTma3d) &&
                         (hkk < 0 || (NLSE_IDX(io.flag, hkk - PW, PW * PH, kSiteTma3d) &&
                                      NLSE_IDX(io.flag, hkk + PW, PW * PH, kSiteTma3d))) &&
                         NLSE_IDX(io.flag, ty * TX + 2 * tx + 1, TX * TY, kSiteTma3d) &&
                         NLSE_IDX(io.flag, x0, nx, kSiteTma3d) && NLSE_IDX(io.flag, y0, ny, kSiteTma3d) &&
                         NLSE_IDX(io.flag, z0, nz, kSiteTma3d) &&
                         NLSE_ALIGN16(io.flag, (int64_t)(x0 - 2) * L::CB, kSiteTma3d) &&
                         NLSE_ALIGN16(io.flag, (int64_t)x0 * L::CB, kSiteTma3d) &&
                         NLSE_ALIGN16(io.flag, (int64_t)x0 * 4, kSiteTma3d) &&
                         NLSE_IDX(io.flag, L::TOTAL - 1, dyn, kSiteTma3d);
        if (__syncthreads_or(!okb)) return;
    }
#endif

    if (t == 0) {
        tma_prefetch_desc(&m_in);
        for (int s = 0; s < S + 2; ++s) mbar_init(ibar0 + 8 * s, 1);
        mbar_init_fence();
    }
    __syncthreads();

    auto issue_in = [&](int j) {
        const int s = j % S;
        const uint32_t bar = ibar0 + 8 * s;
        mbar_expect_tx(bar, L::IN_BYTES);
        asm volatile(
            "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];"
            ::"r"(sbase + L::IN_OFF + s * L::IN_SLOT), "l"(reinterpret_cast<uint64_t>(&m_in)), "r"(x0 - 2),
              "r"(y0 - 2), "r"(zbase + dir * (j - 2)), "r"(bar) : "memory");
    };
    auto load_e = [&](uint32_t dst, const CUtensorMap* m, int z, uint32_t bar) {
        asm volatile(
            "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];"
            ::"r"(dst), "l"(reinterpret_cast<uint64_t>(m)), "r"(x0), "r"(y0), "r"(z), "r"(bar) : "memory");
    };
    auto issue_e = [&](int e) {
        const uint32_t dst = sbase + L::E_OFF + (e & 1) * L::E_SLOT;
        const uint32_t bar = ebar0 + 8 * (e & 1);
        const int z = zbase + dir * e;
        uint32_t bytes = L::V_BYTES;
        if (NEED_PA) bytes += 2 * L::T_BYTES;
        if (NEED_LO) bytes += L::T_BYTES;
        mbar_expect_tx(bar, bytes);
        if (io.keep_v) {
            asm volatile(
                "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes.L2::cache_hint "
                "[%0], [%1, {%2, %3, %4}], [%5], %6;"
                ::"r"(dst + L::E_V), "l"(reinterpret_cast<uint64_t>(&m_V)), "r"(x0), "r"(y0), "r"(z), "r"(bar),
                  "l"(l2_evict_last()) : "memory");
        } else {
            load_e(dst + L::E_V, &m_V, z, bar);
        }
        if (NEED_PA) {
            load_e(dst + L::E_PSI, &m_psi, z, bar);
            load_e(dst + L::E_ACC, &m_acc, z, bar);
        }
        if (NEED_LO) load_e(dst + L::E_LO, &m_lo, z, bar);
    };
    int next = 0, enext = 0;
    if (t == 0) {
        for (; next < S && next < jmax; ++next) issue_in(next);
        if (NEED_E) issue_e(enext++);
    }

    auto iplane = [&](int j) { return reinterpret_cast<const C*>(smem + L::IN_OFF + (j % S) * L::IN_SLOT); };
    C* dring = reinterpret_cast<C*>(smem + L::D_OFF);

    bool ok = true;
    auto wait_in = [&](int j) {
        if (ok) ok = mbar_wait(ibar0 + 8 * (j % S), (uint32_t)((j / S) & 1), kWaitNs);
    };
    auto wait_e = [&](int e) {
        if (ok) ok = mbar_wait(ebar0 + 8 * (e & 1), (uint32_t)((e >> 1) & 1), kWaitNs);
    };

    const C m6 = pair<C>(-6.f, -6.f), m12 = pair<C>(-1.f / 12.f, -1.f / 12.f), c10 = pair<C>(10.f / 12.f, 10.f / 12.f);
    const C m12c = pair<C>(-12.f, -12.f);
    const C m2 = pair<C>(-2.f, -2.f), c76 = pair<C>(7.f / 6.f, 7.f / 6.f);
    const C ih2 = pair<C>(c.inv_h2, c.inv_h2), i6h2 = pair<C>(c.inv_6h2, c.inv_6h2);
    const C a2 = pair<C>(c.a, c.a);
    const C ca2 = pair<C>(-io.c_acc, io.c_acc), cy2 = pair<C>(-io.c_y, io.c_y);

    // D at (x, y, z) from its seven stencil values; the caller passes whether
    // the point is outside the grid or on its boundary (Eq. dbc_lap).
    [[maybe_unused]] const int64_t npts = (int64_t)nx * ny * nz;
    auto vat = [&](int64_t gp) -> float { return NLSE_IDX(io.flag, gp, npts, kSiteTma3d) ? io.V[gp] : 0.f; };
    auto dval = [&](bool out, bool bnd, int64_t gp, C ctr, C s6) -> C {
        if (out) return czero<C>();
        if (bnd) return dirichlet_D(c, ctr, vat(gp));
        return mul2(fma2(m6, ctr, s6), ih2);
    };
    // Multi-storage step 1 at one point, (D^x, D^y, D^z), from the centre and
    // the neighbour sums along x, y, z; the Dirichlet split at points on the
    // boundary of one axis; 0 outside the grid and where two or more axes are
    // on the boundary (never used by an interior Laplacian).
    struct D3 { C x, y, z; };
    auto ms_val = [&](bool out, bool bx, bool by, bool bz, int64_t gp, C ctr, C xs, C ys, C zs) -> D3 {
        if (out) return {czero<C>(), czero<C>(), czero<C>()};
        D3 d{mul2(fma2(m2, ctr, xs), ih2), mul2(fma2(m2, ctr, ys), ih2), mul2(fma2(m2, ctr, zs), ih2)};
        const int nb = (int)bx + (int)by + (int)bz;
        if (nb) {
            const C lb = dirichlet_D(c, ctr, vat(gp));
            if (nb > 1) d = {czero<C>(), czero<C>(), czero<C>()};
            else if (bx) d.x = sub2(sub2(lb, d.y), d.z);
            else if (by) d.y = sub2(sub2(lb, d.x), d.z);
            else d.z = sub2(sub2(lb, d.x), d.y);
        }
        return d;
    };
    auto xout = [&](int x) { return x < 0 || x >= nx; };
    auto yout = [&](int y) { return y < 0 || y >= ny; };
    auto zout = [&](int z) { return z < 0 || z >= nz; };
    auto xbnd = [&](int x) { return x == 0 || x == nx - 1; };
    auto ybnd = [&](int y) { return y == 0 || y == ny - 1; };
    auto zbnd = [&](int z) { return z == 0 || z == nz - 1; };

    const int xa = x0 + 2 * tx, y = y0 + ty;
    const int k = (ty + 2) * PW + 2 * tx + 2;    // this thread's pair in a plane buffer
    const bool oa = xout(xa) || yout(y), ob = xout(xa + 1) || yout(y);
    const bool ba = xbnd(xa) || ybnd(y), bb = xbnd(xa + 1) || ybnd(y);
    const bool pin = !oa;                        // nx is even: then xa + 1 < nx too

    // This thread's D-halo point (warps 0-2): buffer index, grid x, y.
    int hk = -1, hx = 0, hy = 0;
    if (t < TY) { hy = y0 + t; hx = x0 - 1; hk = (t + 2) * PW + 1; }
    else if (t < 2 * TY) { hy = y0 + t - TY; hx = x0 + TX; hk = (t - TY + 2) * PW + TX + 2; }
    else if (t < 2 * TY + TX) { hx = x0 + t - 2 * TY; hy = y0 - 1; hk = PW + (t - 2 * TY) + 2; }
    else if (t < 2 * TY + 2 * TX) { hx = x0 + t - 2 * TY - TX; hy = y0 + TY; hk = (TY + 2) * PW + (t - 2 * TY - TX) + 2; }
    const bool hout = xout(hx) || yout(hy), hbnd = xbnd(hx) || ybnd(hy);
    auto halo_d = [&](int j, int z) -> C {
        const C* pc = iplane(j);
        const bool o = hout || zout(z), b = hbnd || zbnd(z);
        const C s6 = add2(add2(add2(pc[hk - 1], pc[hk + 1]), add2(pc[hk - PW], pc[hk + PW])),
                          add2(iplane(j - 1)[hk], iplane(j + 1)[hk]));
        return dval(o, b, ((int64_t)z * ny + hy) * nx + hx, pc[hk], s6);
    };
    auto halo_ms = [&](int j, int z) -> D3 {
        const C* pc = iplane(j);
        return ms_val(hout || zout(z), xbnd(hx), ybnd(hy), zbnd(z), ((int64_t)z * ny + hy) * nx + hx, pc[hk],
                      add2(pc[hk - 1], pc[hk + 1]), add2(pc[hk - PW], pc[hk + PW]),
                      add2(iplane(j - 1)[hk], iplane(j + 1)[hk]));
    };
    // In-plane axial neighbours of this thread's pair in input plane j.
    struct Nbr { Two up, dn; C l, r; };
    auto nbrs = [&](int j) -> Nbr {
        const C* pc = iplane(j);
        return {ld2(pc + k - PW), ld2(pc + k + PW), pc[k - 1], pc[k + 2]};
    };
    // D of this thread's pair at input plane j (grid plane z), centre values
    // cc, vertical neighbours cm / cp, in-plane neighbours nb.  Also returns q,
    // the sum of the four in-plane axial neighbours: the x and y edge terms
    // that plane z contributes to the Laplacian of planes z -+ 1.
    auto pair_d = [&](const Nbr& nb, int z, Two cm, Two cc, Two cp, Two& q) -> Two {
        const Two up = nb.up, dn = nb.dn;
        const C l = nb.l, r = nb.r;
        const bool zo = zout(z), zb = zbnd(z);
        const int64_t gp = ((int64_t)z * ny + y) * nx + xa;
        q.a = add2(add2(l, cc.b), add2(up.a, dn.a));
        q.b = add2(add2(cc.a, r), add2(up.b, dn.b));
        Two d;
        d.a = dval(oa || zo, ba || zb, gp, cc.a, add2(q.a, add2(cm.a, cp.a)));
        d.b = dval(ob || zo, bb || zb, gp + 1, cc.b, add2(q.b, add2(cm.b, cp.b)));
        return d;
    };

    // Multi-storage step 1 of this thread's pair at input plane j (grid plane
    // z): D^x and D^y out, D^z returned.
    const bool bxa = xbnd(xa), bxb = xbnd(xa + 1), byy = ybnd(y);
    auto pair_ms = [&](const Nbr& nb, int z, Two cm, Two cc, Two cp, Two& dx, Two& dy) -> Two {
        const bool zo = zout(z), zb = zbnd(z);
        const int64_t gp = ((int64_t)z * ny + y) * nx + xa;
        const D3 pa = ms_val(oa || zo, bxa, byy, zb, gp, cc.a, add2(nb.l, cc.b), add2(nb.up.a, nb.dn.a),
                             add2(cm.a, cp.a));
        const D3 pb = ms_val(ob || zo, bxb, byy, zb, gp + 1, cc.b, add2(cc.a, nb.r), add2(nb.up.b, nb.dn.b),
                             add2(cm.b, cp.b));
        dx = Two{pa.x, pb.x};
        dy = Two{pa.y, pb.y};
        return Two{pa.z, pb.z};
    };
    // Multi storage: D^x ring (2 planes, x halo) then D^y ring (2 planes, y halo).
    C* dxring = dring;
    C* dyring = dring + 2 * (PW * PH);

    // Prologue: input planes 0 .. 3 (z0-2 .. z0+1 in walk order).
    wait_in(0); wait_in(1); wait_in(2); wait_in(3);
    bool alive = __syncthreads_and(ok);
    Two cm, c0, c1, dm, d0, qm, q0;
    Two dx0, dy0;                                 // multi storage: D^x, D^y at plane z (D^z in dm, d0, d1)
    if (alive && MS) {
        const Two cmm = ld2(iplane(0) + k);
        cm = ld2(iplane(1) + k); c0 = ld2(iplane(2) + k); c1 = ld2(iplane(3) + k);
        Two ux, uy;
        dm = pair_ms(nbrs(1), zbase - dir, cmm, cm, c0, ux, uy);
        d0 = pair_ms(nbrs(2), zbase, cm, c0, c1, dx0, dy0);
        st2(dxring + k, dx0);
        st2(dyring + k, dy0);
        if (hk >= 0) {
            const D3 hd = halo_ms(2, zbase);
            if (t < 2 * TY) dxring[hk] = hd.x;
            else dyring[hk] = hd.y;
        }
    } else if (alive) {
        const Two cmm = ld2(iplane(0) + k);
        cm = ld2(iplane(1) + k); c0 = ld2(iplane(2) + k); c1 = ld2(iplane(3) + k);
        dm = pair_d(nbrs(1), zbase - dir, cmm, cm, c0, qm);
        d0 = pair_d(nbrs(2), zbase, cm, c0, c1, q0);
        st2(dring + k, d0);                       // input plane 2 -> D ring plane 0
        if (hk >= 0) dring[hk] = halo_d(2, zbase);
    }
    __syncthreads();
    // With a 4-slot ring, input plane 4 reuses plane 0's slot, free only now.
    if (S == 4 && t == 0 && next < jmax) issue_in(next++);

    bool bad = false;
#pragma unroll 3
    for (int i = 0; i < TZ; ++i) {
        if (!alive || i >= nplanes) break;
        const int j = i + 2;
        const int z = zbase + dir * i, za = z + dir;
        wait_in(j + 2);
        if (!__syncthreads_and(ok)) { alive = false; break; }
        if (t == 0) {
            if (next < jmax) issue_in(next++);
            if (NEED_E && enext < nplanes) issue_e(enext++);
        }
        // D of the plane ahead (za).
        const Two c2 = ld2(iplane(j + 2) + k);
        Two q1;                                  // also the z+1 edge terms of Lap(z)
        Two dx1, dy1;
        Two d1;
        if constexpr (MS) {
            d1 = pair_ms(nbrs(j + 1), za, c0, c1, c2, dx1, dy1);
            C* dxn = dxring + ((j + 1) & 1) * (PW * PH);
            C* dyn = dyring + ((j + 1) & 1) * (PW * PH);
            st2(dxn + k, dx1);
            st2(dyn + k, dy1);
            if (hk >= 0) {
                const D3 hd = halo_ms(j + 1, za);
                if (t < 2 * TY) dxn[hk] = hd.x;
                else dyn[hk] = hd.y;
            }
        } else {
            d1 = pair_d(nbrs(j + 1), za, c0, c1, c2, q1);
            C* dn = dring + ((j + 1) & 1) * (PW * PH);
            st2(dn + k, d1);
            if (hk >= 0) dn[hk] = halo_d(j + 1, za);
        }
        // No barrier here: the step below reads the D ring slot written in the
        // previous iteration and this thread's own registers, both ordered by
        // the barrier at the top of the loop, and a thread whose wait gave up
        // carries ok = false to that barrier, where the CTA stops together.
        if (NEED_E) wait_e(i);

        if (pin && NLSE_IDX(io.flag, ((int64_t)z * ny + y) * nx + xa + 1, npts, kSiteTma3d)) {
            const C* pz = iplane(j);
            const C* dz = dring + (j & 1) * (PW * PH);
            const bool zb = zbnd(z);
            const bool bA = ba || zb, bB = bb || zb;
            Two lap = d0;
            if constexpr (MS) {
                // D^x of the x neighbours, D^y of the y neighbours, D^z of the z neighbours
                const C* dxz = dxring + (j & 1) * (PW * PH);
                const C* dyz = dyring + (j & 1) * (PW * PH);
                const Two dyu = ld2(dyz + k - PW), dyd = ld2(dyz + k + PW);
                const C sa = add2(add2(add2(dxz[k - 1], dx0.b), add2(dyu.a, dyd.a)), add2(dm.a, d1.a));
                const C sb = add2(add2(add2(dx0.a, dxz[k + 2]), add2(dyu.b, dyd.b)), add2(dm.b, d1.b));
                lap.a = fma2(c76, add2(add2(dx0.a, dy0.a), d0.a), mul2(m12, sa));
                lap.b = fma2(c76, add2(add2(dx0.b, dy0.b), d0.b), mul2(m12, sb));
                if (STAGE == 0) {
                    const int64_t pg = ((int64_t)z * ny + y) * nx + xa;
                    if (bA) lap.a = dirichlet_D(c, c0.a, vat(pg));
                    if (bB) lap.b = dirichlet_D(c, c0.b, vat(pg + 1));
                }
            } else if (!CD) {
                // six axial D
                const Two dup = ld2(dz + k - PW), ddn = ld2(dz + k + PW);
                const C dsa = add2(add2(add2(dz[k - 1], d0.b), add2(dup.a, ddn.a)), add2(dm.a, d1.a));
                const C dsb = add2(add2(add2(d0.a, dz[k + 2]), add2(dup.b, ddn.b)), add2(dm.b, d1.b));
                // twelve edge neighbours of Psi: xy corners in plane z, xz and yz edges in
                // z -+ 1 (the in-plane axial sums q of those planes)
                const Two pu = ld2(pz + k - PW), pd = ld2(pz + k + PW);
                const C pul = pz[k - PW - 1], pur = pz[k - PW + 2], pdl = pz[k + PW - 1], pdr = pz[k + PW + 2];
                const C ea = add2(add2(add2(pul, pu.b), add2(pdl, pd.b)), add2(qm.a, q1.a));
                const C eb = add2(add2(add2(pu.a, pur), add2(pd.a, pdr)), add2(qm.b, q1.b));
                if (!bA) lap.a = fma2(i6h2, fma2(m12c, c0.a, ea), fma2(m12, dsa, mul2(c10, d0.a)));
                if (!bB) lap.b = fma2(i6h2, fma2(m12c, c0.b, eb), fma2(m12, dsb, mul2(c10, d0.b)));
            }
            const int64_t p = ((int64_t)z * ny + y) * nx + xa;
            if constexpr (STAGE == 0) {
                st2(io.lap + p, lap);
            } else {
                const unsigned char* es = smem + L::E_OFF + (i & 1) * L::E_SLOT;
                const int ke = ty * TX + 2 * tx;
                const float* vv = reinterpret_cast<const float*>(es + L::E_V) + ke;
                auto swapped_w = [&](C y_, C lap_, float v_, bool b_) -> C {
                    if (b_) return czero<C>();
                    const float N = nonlin(c.s, y_, v_);
                    const C w = fma2(pair<C>(N, N), y_, mul2(a2, lap_));
                    return pair<C>(w.y, w.x);
                };
                const C swa = swapped_w(c0.a, lap.a, vv[0], bA);
                const C swb = swapped_w(c0.b, lap.b, vv[1], bB);
                if constexpr (STAGE == 1) {
                    st2(io.acc + p, Two{mul2(ca2, swa), mul2(ca2, swb)});
                    st2(io.yout + p, Two{fma2(cy2, swa, c0.a), fma2(cy2, swb, c0.b)});
                } else {
                    const Two pn = ld2(reinterpret_cast<const C*>(es + L::E_PSI) + ke);
                    const Two ac = ld2(reinterpret_cast<const C*>(es + L::E_ACC) + ke);
                    if constexpr (STAGE == 2 || STAGE == 3) {
                        st2(io.acc + p, Two{fma2(ca2, swa, ac.a), fma2(ca2, swb, ac.b)});
                        st2(io.yout + p, Two{fma2(cy2, swa, pn.a), fma2(cy2, swb, pn.b)});
                    } else {
                        const C da = fma2(ca2, swa, ac.a), db = fma2(ca2, swb, ac.b);
                        Two out = pn;
                        Two lo = ld2(reinterpret_cast<const C*>(es + L::E_LO) + ke);
                        kahan_add(out.a.x, lo.a.x, da.x);
                        kahan_add(out.a.y, lo.a.y, da.y);
                        kahan_add(out.b.x, lo.b.x, db.x);
                        kahan_add(out.b.y, lo.b.y, db.y);
                        st2(io.lo + p, lo);
                        st2(io.psi_out + p, out);
                        bad |= !(isfinite(out.a.x) && isfinite(out.a.y) && isfinite(out.b.x) && isfinite(out.b.y));
                    }
                }
            }
        }
        cm = c0; c0 = c1; c1 = c2;
        dm = d0; d0 = d1;
        if constexpr (MS) {
            dx0 = dx1; dy0 = dy1;
        } else {
            qm = q0; q0 = q1;
        }
    }

    if (!alive) {
        if (t == 0) {
            atomicOr(io.flag, 2);
            for (int j = next > S ? next - S : 0; j < next; ++j)
                mbar_wait(ibar0 + 8 * (j % S), (uint32_t)((j / S) & 1), kDrainNs);
            for (int e = enext > 2 ? enext - 2 : 0; e < enext; ++e)
                mbar_wait(ebar0 + 8 * (e & 1), (uint32_t)((e >> 1) & 1), kDrainNs);
        }
        return;
    }
    if constexpr (STAGE == 4) {
        if (__syncthreads_or(bad) && t == 0) atomicOr(io.flag, 1);
    }
}

// 3D boxes over a complex64 (8-byte elements) or float grid.
inline bool map3(CUtensorMap* m, CUtensorMapDataType type, size_t esize, const void* base, int nx, int ny, int nz,
          int bx, int by) {
    cuuint64_t dims[3] = {(cuuint64_t)nx, (cuuint64_t)ny, (cuuint64_t)nz};
    cuuint64_t strides[2] = {(cuuint64_t)nx * esize, (cuuint64_t)nx * ny * esize};
    cuuint32_t box[3] = {(cuuint32_t)bx, (cuuint32_t)by, 1};
    return encode(m, type, 3, base, dims, strides, box);
}

template <int LP, int STAGE, int TZ>
cudaError_t launch_t(const StageLaunch& L, cudaStream_t st) {
    const int nx = (int)L.n[0], ny = (int)L.n[1], nz = (int)L.n[2];
    const CUtensorMapDataType CX = CU_TENSOR_MAP_DATA_TYPE_UINT64, RF = CU_TENSOR_MAP_DATA_TYPE_FLOAT32;
    CUtensorMap m_in, m_V, m_psi, m_acc, m_lo;
    if (!map3(&m_in, CX, 8, L.yin, nx, ny, nz, PW, PH)) return cudaErrorInvalidValue;
    m_V = m_psi = m_acc = m_lo = m_in;
    if (STAGE >= 1 && !map3(&m_V, RF, 4, L.V, nx, ny, nz, TX, TY)) return cudaErrorInvalidValue;
    if (STAGE >= 2 && (!map3(&m_psi, CX, 8, L.psi, nx, ny, nz, TX, TY) ||
                       !map3(&m_acc, CX, 8, L.acc, nx, ny, nz, TX, TY)))
        return cudaErrorInvalidValue;
    if (STAGE == 4 && !map3(&m_lo, CX, 8, L.lo, nx, ny, nz, TX, TY)) return cudaErrorInvalidValue;
    auto kern = stage3d_tma_kernel<LP, STAGE, TZ>;
    const int smem = Ring3<LP>::L::TOTAL;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    // Consecutive stages walk z in opposite directions.
    const int dir = (STAGE % 2 == 0 && STAGE != 0) ? -1 : 1;
    dim3 grid((nx + TX - 1) / TX, (ny + TY - 1) / TY, (nz + TZ - 1) / TZ);
    kern<<<grid, NT, smem, st>>>(m_in, m_V, m_psi, m_acc, m_lo, make_io<float>(L), make_coef<float>(L.h, L.a, L.s),
                                 nx, ny, nz, dir);
    return cudaGetLastError();
}

template <int LP, int TZ>
cudaError_t launch_stage(const StageLaunch& L, cudaStream_t st) {
    switch (L.stage) {
        case 0: return launch_t<LP, 0, TZ>(L, st);
        case 1: return launch_t<LP, 1, TZ>(L, st);
        case 2: return launch_t<LP, 2, TZ>(L, st);
        case 3: return launch_t<LP, 3, TZ>(L, st);
        case 4: return launch_t<LP, 4, TZ>(L, st);
    }
    return cudaErrorInvalidValue;
}

template <int TZ>
cudaError_t launch_planes(const StageLaunch& L, cudaStream_t st) {
    switch (L.lap) {
        case 0: return launch_stage<0, TZ>(L, st);
        case 1: return launch_stage<1, TZ>(L, st);
        case 2: return launch_stage<2, TZ>(L, st);
    }
    return cudaErrorInvalidValue;
}

}  // namespace tma3d
}  // namespace nlse
