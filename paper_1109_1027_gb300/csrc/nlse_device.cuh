// nlse_device.cuh -- device-side building blocks shared by the stage kernels:
// complex arithmetic on float2 / double2, the step-1 boundary rule of
// Sec. 3.2 and the RK4 stage epilogue of Eq. (RK4).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "nlse_internal.h"

namespace nlse {

template <typename R> struct CplxOf;
template <> struct CplxOf<float> { using type = float2; };
template <> struct CplxOf<double> { using type = double2; };
template <typename R> using cplx = typename CplxOf<R>::type;

template <typename C> __device__ __forceinline__ C cmake(decltype(C::x) re, decltype(C::x) im) {
    C z; z.x = re; z.y = im; return z;
}
template <typename C> __device__ __forceinline__ C czero() { return cmake<C>(0, 0); }
template <typename C> __device__ __forceinline__ C cadd(C a, C b) { return cmake<C>(a.x + b.x, a.y + b.y); }
template <typename C> __device__ __forceinline__ C csub(C a, C b) { return cmake<C>(a.x - b.x, a.y - b.y); }
template <typename C, typename R> __device__ __forceinline__ C cscale(R r, C a) {
    return cmake<C>(r * a.x, r * a.y);
}
// a + r * b
template <typename C, typename R> __device__ __forceinline__ C caxpy(C a, R r, C b) {
    return cmake<C>(a.x + r * b.x, a.y + r * b.y);
}
template <typename C> __device__ __forceinline__ decltype(C::x) cabs2(C a) { return a.x * a.x + a.y * a.y; }
// i * a
template <typename C> __device__ __forceinline__ C ctimesi(C a) { return cmake<C>(-a.y, a.x); }

// Whether nlse_run's entry check refused the steps now being run (a refusal
// bit in the context's status block, set on the device before the steps were
// enqueued behind it and cleared only by nlse_check): the stage-4 kernels then
// leave the state as it is.  Read once per CTA; no kernel of a step changes
// these bits.
__device__ __forceinline__ bool refused(const int* flag) {
    return (*(const volatile int*)flag & kStatusRefused) != 0;
}

// Bounds-check build (compiled with -DNLSE_BOUNDS_CHECK): the kernels test
// their shared-memory and global indices (and the 16-byte alignment of their
// TMA coordinates) before the access.  An index outside its array sets
// kStatusBounds in the status word and records the smallest failing site
// (file id * 100000 + source line), and the access is skipped: nothing traps.
// nlse_check then returns NLSE_EBOUNDS.  In the normal build every check is
// the constant true and compiles away.
#ifdef NLSE_BOUNDS_CHECK
static __device__ __noinline__ bool bounds_fail(int* flag, int site) {
    atomicOr(flag, kStatusBounds);
    atomicMin(flag + 2, site);              // StatusBlock::site
    return false;
}
__device__ __forceinline__ bool idx_ok(int* flag, int64_t i, int64_t n, int site) {
    return (i >= 0 && i < n) ? true : bounds_fail(flag, site);
}
#define NLSE_IDX(flag, i, n, file) ::nlse::idx_ok((flag), (int64_t)(i), (int64_t)(n), (file) * 100000 + __LINE__)
#define NLSE_ALIGN16(flag, bytes, file) \
    ::nlse::idx_ok((flag), ((int64_t)(bytes)) % 16 == 0 ? 0 : -1, 1, (file) * 100000 + __LINE__)
#else
#define NLSE_IDX(flag, i, n, file) true
#define NLSE_ALIGN16(flag, bytes, file) true
#endif
// File ids of the check sites.
constexpr int kSiteTile2d = 1, kSiteTma3d = 2, kSiteStage1d = 3, kSiteStage2d = 4, kSiteStage3d = 5,
              kSiteFused = 6, kSiteResident1d = 7, kSitePlain = 8, kSiteCheck = 9, kSiteAdj2d = 10;

// Row within its stacked instance of grid row r >= 0 (instances of rows1 rows;
// without a stack rows1 is the grid's row count and r is returned undivided).
__device__ __forceinline__ int inst_row(int r, int rows1) { return r < rows1 ? r : r % rows1; }

// Scalars of one problem, in the stage arithmetic R.
template <typename R>
struct Coef {
    R inv_h2;     // 1 / h^2
    R inv_6h2;    // 1 / (6 h^2)
    R a, s, inv_a;
};

template <typename R>
Coef<R> make_coef(double h, double a, double s) {
    Coef<R> c;
    c.inv_h2 = (R)(1.0 / (h * h));
    c.inv_6h2 = (R)(1.0 / (6.0 * h * h));
    c.a = (R)a; c.s = (R)s; c.inv_a = (R)(1.0 / a);
    return c;
}

// Pointers and coefficients of one RK4 stage (see StageLaunch).
template <typename R>
struct StageIO {
    const cplx<R>* yin;
    const cplx<R>* psi;
    cplx<R>* psi_out;
    cplx<R>* lo;
    cplx<R>* acc;
    cplx<R>* yout;
    cplx<R>* lap;
    const R* V;
    int* flag;
    R c_acc;      // weight of F in the accumulated increment: k/6, k/3, k/3, k/6
    R c_y;        // weight of F in the next stage input: k/2, k/2, k
    int keep_v;   // TMA kernels: load V with an L2 evict-last hint
    int rows1;    // 2D: rows per stacked instance (the Dirichlet rows are 0 and rows1-1 of
                  // each; V has rows1 rows, shared)
};

template <typename R>
StageIO<R> make_io(const StageLaunch& L) {
    StageIO<R> io;
    io.yin = (const cplx<R>*)L.yin;
    io.psi = (const cplx<R>*)L.psi;
    io.psi_out = (cplx<R>*)L.psi_out;
    io.lo = (cplx<R>*)L.lo;
    io.acc = (cplx<R>*)L.acc;
    io.yout = (cplx<R>*)L.yout;
    io.lap = (cplx<R>*)L.lap_out;
    io.V = (const R*)L.V;
    io.flag = L.flag;
    io.keep_v = L.keep_v;
    io.rows1 = (int)(L.rows1 ? L.rows1 : L.n[1]);
    const double k = L.dt;
    const double wa[5] = {0.0, k / 6.0, k / 3.0, k / 3.0, k / 6.0};
    const double wy[5] = {0.0, k / 2.0, k / 2.0, k, 0.0};
    io.c_acc = (R)wa[L.stage];
    io.c_y = (R)wy[L.stage];
    return io;
}

// N = s|y|^2 - V (Eq. nbnb1) with explicitly rounded fused multiply-adds, so
// that every kernel and every launch shape evaluates it with the same
// roundings: fma(s, fma(y.x, y.x, y.y * y.y), -V).
__device__ __forceinline__ float nonlin(float s, float2 y, float v) {
    return __fmaf_rn(s, __fmaf_rn(y.x, y.x, __fmul_rn(y.y, y.y)), -v);
}
__device__ __forceinline__ double nonlin(double s, double2 y, double v) {
    return __fma_rn(s, __fma_rn(y.x, y.x, __dmul_rn(y.y, y.y)), -v);
}

// Dirichlet step-1 boundary value, Eq. (dbc_lap): D_b = -(s|psi_b|^2 - V_b) psi_b / a.
template <typename R>
__device__ __forceinline__ cplx<R> dirichlet_D(const Coef<R>& c, cplx<R> pb, R Vb) {
    R Nb = nonlin(c.s, pb, Vb);
    return cscale(-Nb * c.inv_a, pb);
}

// MSD step-1 boundary value, Eq. (msdbc_lap) with N of Eq. (nbnb1) and
// Im(i z) = Re(z):  D_b = [ Re(D_q / psi_q) + (N_q - N_b) / a ] psi_b,
// q the closest interior point.
template <typename R>
__device__ __forceinline__ cplx<R> msd_D(const Coef<R>& c, cplx<R> pb, R Vb, cplx<R> pq, R Vq,
                                         cplx<R> Dq) {
    R Nb = nonlin(c.s, pb, Vb);
    R Nq = nonlin(c.s, pq, Vq);
    R re_ratio = (Dq.x * pq.x + Dq.y * pq.y) / cabs2(pq);
    return cscale(re_ratio + (Nq - Nb) * c.inv_a, pb);
}

// MSD boundary time derivative, Eq. (msdbc_ut): F_b = i Im(F_q / psi_q) psi_b.
template <typename C>
__device__ __forceinline__ C msd_F(C pb, C pq, C Fq) {
    auto im_ratio = (Fq.y * pq.x - Fq.x * pq.y) / cabs2(pq);
    return ctimesi(cscale(im_ratio, pb));
}

// F = i [ a Lap + (s|y|^2 - V) y ] at an interior point (Sec. 3.1).
template <typename R>
__device__ __forceinline__ cplx<R> rhs_point(const Coef<R>& c, cplx<R> y, cplx<R> lap, R v) {
    R N = nonlin(c.s, y, v);
    return ctimesi(cmake<cplx<R>>(c.a * lap.x + N * y.x, c.a * lap.y + N * y.y));
}

// Compensated addition of a small increment d to the FP32 state (hi, lo)
// (Kahan summation with lo holding the running error).  The adds are
// explicit round-to-nearest intrinsics so that the compiler can neither
// contract nor reassociate them.
__device__ __forceinline__ void kahan_add(float& hi, float& lo, float d) {
    float y = __fadd_rn(d, lo);
    float t = __fadd_rn(hi, y);
    lo = __fsub_rn(y, __fsub_rn(t, hi));
    hi = t;
}

// RK4 stage epilogue at point p (Eq. RK4, with the three work arrays of
// Sec. 3.1 replaced by an accumulated increment acc = k/6 (K1 + 2K2 + 2K3)):
//   stage 1: acc  = k/6 F;          y_next = psi + k/2 F    (y is psi itself)
//   stage 2: acc += k/3 F;          y_next = psi + k/2 F
//   stage 3: acc += k/3 F;          y_next = psi + k F
//   stage 4: psi  = psi + (acc + k/6 F)   (compensated in FP32)
// Returns true when stage 4 produced a non-finite value.
template <int STAGE, typename R>
__device__ __forceinline__ bool stage_epilogue(const StageIO<R>& io, int64_t p, cplx<R> y,
                                               cplx<R> F) {
    using C = cplx<R>;
    if constexpr (STAGE == 1) {
        io.acc[p] = cscale(io.c_acc, F);
        io.yout[p] = caxpy(y, io.c_y, F);
        return false;
    } else if constexpr (STAGE == 2 || STAGE == 3) {
        C pn = io.psi[p];
        C ac = io.acc[p];
        io.acc[p] = caxpy(ac, io.c_acc, F);
        io.yout[p] = caxpy(pn, io.c_y, F);
        return false;
    } else {
        C pn = io.psi[p];
        C d = caxpy(io.acc[p], io.c_acc, F);
        if constexpr (sizeof(R) == 4) {
            C lo = io.lo[p];
            kahan_add(pn.x, lo.x, d.x);
            kahan_add(pn.y, lo.y, d.y);
            io.lo[p] = lo;
            io.psi_out[p] = pn;
        } else {
            pn = cadd(pn, d);
            io.psi_out[p] = pn;
        }
        return !(isfinite(pn.x) && isfinite(pn.y));
    }
}

}  // namespace nlse
