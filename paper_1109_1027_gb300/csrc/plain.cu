// plain.cu -- the paper's own, unfused schedule of one RK4+2SHOC step, kept
// as the per-instance baseline the fused kernels are measured against.
//
// Storage and order follow Sec. 3.1 literally: the step-1 field D, and the
// RK4 work arrays K_tot, K_tmp and Psi_tmp, are full grids in device memory;
// every F(Psi) is two launches (D, then step 2 + F), and each axpy line of
// Eq. (RK4) is its own launch -- fourteen launches per step.  One thread per
// grid point, no shared memory.  Dirichlet boundaries only.
#include "nlse_device.cuh"

namespace nlse {
namespace {

constexpr int NT = 256;

struct Grid3 {
    int n[3];
    int dim;
    int64_t stride[3];
    int64_t npts;
};

__device__ __forceinline__ bool decompose(const Grid3& g, int64_t p, int* c) {
    int64_t r = p;
    c[0] = (int)(r % g.n[0]); r /= g.n[0];
    c[1] = (int)(r % g.n[1]); r /= g.n[1];
    c[2] = (int)r;
    for (int ax = 0; ax < g.dim; ++ax)
        if (c[ax] == 0 || c[ax] == g.n[ax] - 1) return true;
    return false;
}

// Step 1 everywhere: interior D (Eqs. 2shoc1d, 2d2shocs1, 3d2shocs) and the
// Dirichlet boundary value D_b of Eq. (dbc_lap).
template <typename R>
__global__ void __launch_bounds__(NT) plain_d(const cplx<R>* psi, const R* V, cplx<R>* D, Grid3 g,
                                              Coef<R> c) {
    using C = cplx<R>;
    int64_t p = blockIdx.x * (int64_t)NT + threadIdx.x;
    if (p >= g.npts) return;
    int x[3];
    C ctr = psi[p];
    if (decompose(g, p, x)) {
        D[p] = dirichlet_D(c, ctr, V[p]);
        return;
    }
    C sum = czero<C>();
    for (int ax = 0; ax < g.dim; ++ax) sum = cadd(sum, cadd(psi[p + g.stride[ax]], psi[p - g.stride[ax]]));
    D[p] = cscale(c.inv_h2, csub(sum, cscale((R)(2 * g.dim), ctr)));
}

// Step 2 (or CD) and F (Sec. 3.1) into K; F_b = 0 (Eq. dbc_ut).
template <typename R, bool CD>
__global__ void __launch_bounds__(NT) plain_f(const cplx<R>* psi, const cplx<R>* D, const R* V,
                                              cplx<R>* K, Grid3 g, Coef<R> c) {
    using C = cplx<R>;
    int64_t p = blockIdx.x * (int64_t)NT + threadIdx.x;
    if (p >= g.npts) return;
    int x[3];
    if (decompose(g, p, x)) {
        K[p] = czero<C>();
        return;
    }
    C lap = D[p];
    C y = psi[p];
    if (!CD) {
        const int d = g.dim;
        C dsum = czero<C>();
        for (int ax = 0; ax < d; ++ax) dsum = cadd(dsum, cadd(D[p + g.stride[ax]], D[p - g.stride[ax]]));
        C edges = czero<C>();
        for (int a1 = 0; a1 < d; ++a1)
            for (int a2 = a1 + 1; a2 < d; ++a2) {
                int64_t s1 = g.stride[a1], s2 = g.stride[a2];
                edges = cadd(edges, cadd(cadd(psi[p + s1 + s2], psi[p + s1 - s2]),
                                         cadd(psi[p - s1 + s2], psi[p - s1 - s2])));
            }
        // ((16 - 2d)/12) D_c - (1/12) sum_axial D + (1/(6h^2)) (edges - 2d(d-1) psi_c)
        C dpart = csub(cscale((R)((16.0 - 2.0 * d) / 12.0), lap), cscale((R)(1.0 / 12.0), dsum));
        C ppart = cscale(c.inv_6h2, csub(edges, cscale((R)(2 * d * (d - 1)), y)));
        lap = cadd(dpart, ppart);
    }
    K[p] = rhs_point(c, y, lap, V[p]);
}

// out = a + w b   (lines 2, 5, 8 of Eq. RK4)
template <typename R>
__global__ void __launch_bounds__(NT) plain_axpy(cplx<R>* out, const cplx<R>* a, R w, const cplx<R>* b,
                                                 int64_t n) {
    int64_t p = blockIdx.x * (int64_t)NT + threadIdx.x;
    if (p < n) out[p] = caxpy(a[p], w, b[p]);
}

// acc += w b      (lines 4, 7)
template <typename R>
__global__ void __launch_bounds__(NT) plain_acc(cplx<R>* acc, R w, const cplx<R>* b, int64_t n) {
    int64_t p = blockIdx.x * (int64_t)NT + threadIdx.x;
    if (p < n) acc[p] = caxpy(acc[p], w, b[p]);
}

// psi += w (a + b)  (line 10)
template <typename R>
__global__ void __launch_bounds__(NT) plain_final(cplx<R>* psi, R w, const cplx<R>* a, const cplx<R>* b,
                                                  int64_t n, int* flag) {
    int64_t p = blockIdx.x * (int64_t)NT + threadIdx.x;
    if (p >= n) return;
    cplx<R> v = caxpy(psi[p], w, cadd(a[p], b[p]));
    psi[p] = v;
    if (!(isfinite(v.x) && isfinite(v.y))) atomicOr(flag, 1);
}

template <typename R>
cudaError_t step_r(const PlainLaunch& L, cudaStream_t st) {
    using C = cplx<R>;
    Grid3 g;
    g.dim = L.dim;
    for (int ax = 0; ax < 3; ++ax) g.n[ax] = ax < L.dim ? (int)L.n[ax] : 1;
    g.stride[0] = 1;
    g.stride[1] = g.n[0];
    g.stride[2] = (int64_t)g.n[0] * g.n[1];
    g.npts = (int64_t)g.n[0] * g.n[1] * g.n[2];
    Coef<R> c = make_coef<R>(L.h, L.a, L.s);
    C* psi = (C*)L.psi;
    C* D = (C*)L.D;
    C* Ktot = (C*)L.Ktot;
    C* Ktmp = (C*)L.Ktmp;
    C* ptmp = (C*)L.ptmp;
    const R* V = (const R*)L.V;
    const int64_t n = g.npts;
    const unsigned blocks = (unsigned)((n + NT - 1) / NT);
    const R k = (R)L.dt;
    auto F = [&](const C* in, C* out) {
        plain_d<R><<<blocks, NT, 0, st>>>(in, V, D, g, c);
        if (L.lap == 1) plain_f<R, true><<<blocks, NT, 0, st>>>(in, D, V, out, g, c);
        else plain_f<R, false><<<blocks, NT, 0, st>>>(in, D, V, out, g, c);
    };
    F(psi, Ktot);                                                          // 1
    plain_axpy<R><<<blocks, NT, 0, st>>>(ptmp, psi, k / 2, Ktot, n);      // 2
    F(ptmp, Ktmp);                                                         // 3
    plain_acc<R><<<blocks, NT, 0, st>>>(Ktot, (R)2, Ktmp, n);             // 4
    plain_axpy<R><<<blocks, NT, 0, st>>>(ptmp, psi, k / 2, Ktmp, n);      // 5
    F(ptmp, Ktmp);                                                         // 6
    plain_acc<R><<<blocks, NT, 0, st>>>(Ktot, (R)2, Ktmp, n);             // 7
    plain_axpy<R><<<blocks, NT, 0, st>>>(ptmp, psi, k, Ktmp, n);          // 8
    F(ptmp, Ktmp);                                                         // 9
    plain_final<R><<<blocks, NT, 0, st>>>(psi, k / 6, Ktot, Ktmp, n, L.flag);  // 10
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_plain_step(const PlainLaunch& L, cudaStream_t st) {
    return L.prec == 0 ? step_r<float>(L, st) : step_r<double>(L, st);
}

}  // namespace nlse
