// adjoint2d.cuh -- the per-point arithmetic of one reversed RK4 stage of the
// 2D Dirichlet adjoint (the operator is derived in adjoint2d.cu), shared by
// the shared-memory tile kernel (adjoint2d.cu) and the TMA-fed row walk
// (adjoint2d_tma.cu).  Every operation is an explicitly rounded instruction
// (packed f32x2 or __d*_rn), so the compiler can neither contract nor
// reassociate it and both kernels give the same bits for every launch shape.
#pragma once

#include "nlse_device.cuh"
#include "tma.cuh"

namespace nlse {
namespace adj {

template <typename C> __device__ __forceinline__ C two(decltype(C::x) a, decltype(C::x) b) {
    C z; z.x = a; z.y = b; return z;
}

__device__ __forceinline__ float rmul(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double rmul(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ float rfma(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double rfma(double a, double b, double c) { return __fma_rn(a, b, c); }

// Scalars of one reversed stage.
template <typename R>
struct Coef {
    R a;            // coefficient of the Laplacian
    R s;            // nonlinearity
    R inv_a;        // 1 / a
    R ms_inv_a;     // -s / a
    R two_s;        // 2 s
    R inv_h2;       // 1 / h^2
    R inv_6h2;      // 1 / (6 h^2)
    R sw;           // the stored cotangent is w / sw: w = sw * stored
    R cw, cy;       // w_next = cw lam' + cy Ybar
};

template <typename R>
Coef<R> make_coef(double h, double a, double s, double sw, double cw, double cy) {
    Coef<R> c;
    c.a = (R)a; c.s = (R)s; c.inv_a = (R)(1.0 / a); c.ms_inv_a = (R)(-s / a); c.two_s = (R)(2.0 * s);
    c.inv_h2 = (R)(1.0 / (h * h)); c.inv_6h2 = (R)(1.0 / (6.0 * h * h));
    c.sw = (R)sw; c.cw = (R)cw; c.cy = (R)cy;
    return c;
}

// The scaled cotangent w = sw * stored at a point.
template <typename R>
__device__ __forceinline__ cplx<R> wscale(const Coef<R>& c, cplx<R> stored) {
    return mul2(two<cplx<R>>(c.sw, c.sw), stored);
}

// u = -i a w at an interior point, 0 elsewhere (transpose of "i a Lap").
template <typename R>
__device__ __forceinline__ cplx<R> u_of(const Coef<R>& c, cplx<R> stored, bool inner) {
    const cplx<R> w = wscale(c, stored);
    return inner ? mul2(two<cplx<R>>(c.a, -c.a), two<cplx<R>>(w.y, w.x)) : czero<cplx<R>>();
}

// E = u - (1/12)(sum of the four axial u): the transpose of step 2 in D
// (Eq. 2d2shocs2); the CD Laplacian has E = u.  ue, uw: x +- 1; us, un: y +- 1.
template <bool CD, typename C>
__device__ __forceinline__ C e_of(C uc, C ue, C uw, C us, C un) {
    if constexpr (CD) return uc;
    using R = decltype(C::x);
    return fma2(two<C>(R(-1.0 / 12.0), R(-1.0 / 12.0)), add2(add2(ue, uw), add2(us, un)), uc);
}

// The stencil part of Ybar at a point: the transpose of step 1 (Eq.
// 2d2shocs1) applied to E, and for 2SHOC the corner terms of step 2.  ec and
// the four axial E are 0 where their point is not interior; uc is u at the
// point; the corners are paired by row: (y+1: x+1, x-1), (y-1: x+1, x-1).
template <bool CD, typename R>
__device__ __forceinline__ cplx<R> ybar_stencil(const Coef<R>& c, cplx<R> ec, cplx<R> ee, cplx<R> ew, cplx<R> es,
                                                cplx<R> en, cplx<R> uc, cplx<R> c1e, cplx<R> c1w, cplx<R> c2e,
                                                cplx<R> c2w) {
    using C = cplx<R>;
    const C m4 = two<C>(R(-4), R(-4));
    C y = mul2(two<C>(c.inv_h2, c.inv_h2), fma2(m4, ec, add2(add2(ee, ew), add2(es, en))));
    if constexpr (!CD)
        y = fma2(two<C>(c.inv_6h2, c.inv_6h2), fma2(m4, uc, add2(add2(c1e, c1w), add2(c2e, c2w))), y);
    return y;
}

// Adds the pointwise part of Ybar (the transpose of the nonlinear term of F,
// and on the boundary the transpose of D_b of Eq. dbc_lap) and returns the
// point's contribution to dL/dV:
//   interior: Ybar += -i g w + i s Y^2 conj(w),  g = 2 s |Y|^2 - V;  dL/dV += Im(conj(w) Y)
//   boundary: Ybar += -(g / a) E - (s / a) Y^2 conj(E);              dL/dV += Re(conj(E) Y) / a
// w is the scaled cotangent at the point, E its raw E.
template <typename R>
__device__ __forceinline__ R pointwise(const Coef<R>& c, bool inner, cplx<R> w, cplx<R> E, cplx<R> Y, R v,
                                       cplx<R>& ybar) {
    using C = cplx<R>;
    const R yy = rmul(Y.y, Y.y);
    const R rho = rfma(Y.x, Y.x, yy);
    const R y2x = rfma(Y.x, Y.x, -yy);                  // Y^2 = (y2x, y2y)
    const R y2y = rmul(Y.x + Y.x, Y.y);
    const R g = rfma(c.two_s, rho, -v);
    C inc;
    R gv;
    if (inner) {
        const R sx = rfma(y2x, w.x, rmul(y2y, w.y));    // Y^2 conj(w)
        const R sy = rfma(y2y, w.x, -rmul(y2x, w.y));
        inc = two<C>(rfma(g, w.y, -rmul(c.s, sy)), rfma(c.s, sx, -rmul(g, w.x)));
        gv = rfma(w.x, Y.y, -rmul(w.y, Y.x));
    } else {
        const R alpha = rmul(-g, c.inv_a);
        const R ex = rfma(y2x, E.x, rmul(y2y, E.y));    // Y^2 conj(E)
        const R ey = rfma(y2y, E.x, -rmul(y2x, E.y));
        inc = two<C>(rfma(alpha, E.x, rmul(c.ms_inv_a, ex)), rfma(alpha, E.y, rmul(c.ms_inv_a, ey)));
        gv = rmul(rfma(E.x, Y.x, rmul(E.y, Y.y)), c.inv_a);
    }
    ybar = add2(ybar, inc);
    return gv;
}

// The cotangent of the previous stage's K: cw lam' + cy Ybar.
template <typename R>
__device__ __forceinline__ cplx<R> w_next(const Coef<R>& c, cplx<R> lamp, cplx<R> ybar) {
    using C = cplx<R>;
    return fma2(two<C>(c.cy, c.cy), ybar, mul2(two<C>(c.cw, c.cw), lamp));
}

// The running dL/dV of a reverse sweep, 8 bytes per point: FP64 in FP64 runs;
// in FP32 runs a double-float (hi, lo), hi + lo the value with |lo| at most
// half an ulp of hi, updated by error-free transformations (Knuth's TwoSum,
// twice) in FP32 arithmetic, about 48 significant bits.  FP64 instructions
// run at 1/64 of the FP32 rate on this GPU; four of them per point and step
// would bound the last reversed stage.  The sweep ends with one conversion
// to FP64 (gv_double).
template <typename R> struct GAccOf;
template <> struct GAccOf<float> { using type = float2; };
template <> struct GAccOf<double> { using type = double; };
template <typename R> using gacc = typename GAccOf<R>::type;

// (s, e) with s = fl(a + b) and s + e = a + b exactly.
__device__ __forceinline__ float2 two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    const float bv = __fsub_rn(s, a);
    const float av = __fsub_rn(s, bv);
    return make_float2(s, __fadd_rn(__fsub_rn(a, av), __fsub_rn(b, bv)));
}

// (hi, lo) + x, renormalised.
__device__ __forceinline__ float2 df_add(float2 acc, float x) {
    const float2 se = two_sum(acc.x, x);
    return two_sum(se.x, __fadd_rn(se.y, acc.y));
}

// dL/dV after the four reversed stages of a step, added in the order 4, 3, 2, 1.
__device__ __forceinline__ float2 gv_total(float2 acc, float g4, float g3, float g2, float g1) {
    return df_add(df_add(df_add(df_add(acc, g4), g3), g2), g1);
}
__device__ __forceinline__ double gv_total(double acc, double g4, double g3, double g2, double g1) {
    return __dadd_rn(__dadd_rn(__dadd_rn(__dadd_rn(acc, g4), g3), g2), g1);
}

__device__ __forceinline__ double gv_double(float2 acc) { return __dadd_rn((double)acc.x, (double)acc.y); }

}  // namespace adj
}  // namespace nlse
