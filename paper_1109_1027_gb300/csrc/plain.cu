// plain.cu -- an unfused RK4+2SHOC step, one launch per operation over the
// whole grid: the per-instance baseline the fused kernels are measured
// against, with the storage plan of an unfused CPU-style code (Sec. 3.1): the
// step-1 field D and the RK4 work fields are full grids in device memory.
//
// The step is classic four-stage RK4 written from its Butcher tableau
// (nodes 0, 1/2, 1/2, 1; weights 1/6, 1/3, 1/3, 1/6): for stage j the stage
// input Y = Psi + c_j k K_{j-1} (Y = Psi for j = 1) is one launch, its slope
// K_j = F(Y) two (D, then step 2 + F), and the increment acc = sum b_j k K_j
// one; the state update Psi += acc closes the step -- sixteen launches per
// step.  One thread per grid point, no shared memory.
//
// The same kernels carry the MSD boundary rule in every dimension (the fused
// 2D and 3D kernels are Dirichlet only): with the D and F fields in global
// memory, the paper's sweep order -- interior D, then D_b from the interior
// D at the inward point (Eq. msdbc_lap), interior F, then F_b from the
// interior F at the inward point (Eq. msdbc_ut) -- is one more launch per
// field.  The inward point of a boundary point has every coordinate clamped
// into [1, n-2] (the normal neighbour on a face, the diagonal one on an edge
// or corner).  They also carry the two further conditions Sec. 3.2 names:
// periodic (no boundary points, neighbour indices wrap) and Laplacian-zero
// (D_b = 0 and F_b = i (s|Psi_b|^2 - V_b) Psi_b, the equation with a zero
// Laplacian).  In FP32 the state update adds the increment with the
// compensated (Kahan) sum of the fused path.
#include "nlse_device.cuh"

namespace nlse {
namespace {

constexpr int NT = 256;

struct Grid3 {
    int n[3];
    int dim;
    int bc;                 // 0 Dirichlet, 1 MSD, 2 periodic, 3 Laplacian-zero
    int64_t stride[3];
    int64_t npts;
    int* flag;              // status word (bounds-check build: out-of-range neighbour indices)
};

__device__ __forceinline__ bool decompose(const Grid3& g, int64_t p, int* c) {
    int64_t r = p;
    c[0] = (int)(r % g.n[0]); r /= g.n[0];
    c[1] = (int)(r % g.n[1]); r /= g.n[1];
    c[2] = (int)r;
    if (g.bc == 2) return false;                     // periodic: no boundary points
    for (int ax = 0; ax < g.dim; ++ax)
        if (c[ax] == 0 || c[ax] == g.n[ax] - 1) return true;
    return false;
}

// Index of the neighbour of point p (coordinates x) at offset d along axis
// ax; on a periodic grid the coordinate wraps.
__device__ __forceinline__ int64_t nbr(const Grid3& g, const int* x, int64_t p, int ax, int d) {
    int64_t q;
    if (g.bc != 2) {
        q = p + d * g.stride[ax];
    } else {
        int c = x[ax] + d;
        c = c < 0 ? c + g.n[ax] : (c >= g.n[ax] ? c - g.n[ax] : c);
        q = p + (int64_t)(c - x[ax]) * g.stride[ax];
    }
    return NLSE_IDX(g.flag, q, g.npts, kSitePlain) ? q : p;    // (out of range: recorded, the point itself read)
}

__device__ __forceinline__ int64_t inward(const Grid3& g, const int* x) {
    int64_t q = 0;
    for (int ax = 0; ax < g.dim; ++ax) q += (int64_t)min(max(x[ax], 1), g.n[ax] - 2) * g.stride[ax];
    return q;
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
        D[p] = g.bc == 3 ? czero<C>() : dirichlet_D(c, ctr, V[p]);   // MSD: corrected by plain_d_msd
        return;
    }
    C sum = czero<C>();
    for (int ax = 0; ax < g.dim; ++ax) sum = cadd(sum, cadd(psi[nbr(g, x, p, ax, 1)], psi[nbr(g, x, p, ax, -1)]));
    D[p] = cscale(c.inv_h2, csub(sum, cscale((R)(2 * g.dim), ctr)));
}

// MSD: the step-1 boundary value D_b of Eq. (msdbc_lap) from the interior D
// at the inward point (overwrites the Dirichlet value plain_d left there).
template <typename R>
__global__ void __launch_bounds__(NT) plain_d_msd(const cplx<R>* psi, const R* V, cplx<R>* D, Grid3 g,
                                                  Coef<R> c) {
    int64_t p = blockIdx.x * (int64_t)NT + threadIdx.x;
    if (p >= g.npts) return;
    int x[3];
    if (!decompose(g, p, x)) return;
    const int64_t q = inward(g, x);
    D[p] = msd_D(c, psi[p], V[p], psi[q], V[q], D[q]);
}

// MSD: F_b = i Im(F_q / psi_q) psi_b, Eq. (msdbc_ut), from the interior F at
// the inward point q.
template <typename R>
__global__ void __launch_bounds__(NT) plain_f_msd(const cplx<R>* psi, cplx<R>* K, Grid3 g) {
    int64_t p = blockIdx.x * (int64_t)NT + threadIdx.x;
    if (p >= g.npts) return;
    int x[3];
    if (!decompose(g, p, x)) return;
    const int64_t q = inward(g, x);
    K[p] = msd_F(psi[p], psi[q], K[q]);
}

// Step 2 (or CD) and F (Sec. 3.1) into K; F_b = 0 (Eq. dbc_ut).  With LAP
// the Laplacian itself goes to K instead (boundary points: D_b).
template <typename R, bool CD, bool LAP = false>
__global__ void __launch_bounds__(NT) plain_f(const cplx<R>* psi, const cplx<R>* D, const R* V,
                                              cplx<R>* K, Grid3 g, Coef<R> c) {
    using C = cplx<R>;
    int64_t p = blockIdx.x * (int64_t)NT + threadIdx.x;
    if (p >= g.npts) return;
    int x[3];
    if (decompose(g, p, x)) {
        // Dirichlet F_b = 0 (MSD: replaced by plain_f_msd); Laplacian-zero: the
        // equation with Lap_b = 0.
        K[p] = LAP ? D[p] : (g.bc == 3 ? rhs_point(c, psi[p], czero<C>(), V[p]) : czero<C>());
        return;
    }
    C lap = D[p];
    C y = psi[p];
    if (!CD) {
        const int d = g.dim;
        C dsum = czero<C>();
        for (int ax = 0; ax < d; ++ax) dsum = cadd(dsum, cadd(D[nbr(g, x, p, ax, 1)], D[nbr(g, x, p, ax, -1)]));
        C edges = czero<C>();
        for (int a1 = 0; a1 < d; ++a1)
            for (int a2 = a1 + 1; a2 < d; ++a2) {
                const int64_t pp = nbr(g, x, p, a1, 1), pm = nbr(g, x, p, a1, -1);
                edges = cadd(edges, cadd(cadd(psi[nbr(g, x, pp, a2, 1)], psi[nbr(g, x, pp, a2, -1)]),
                                         cadd(psi[nbr(g, x, pm, a2, 1)], psi[nbr(g, x, pm, a2, -1)])));
            }
        // ((16 - 2d)/12) D_c - (1/12) sum_axial D + (1/(6h^2)) (edges - 2d(d-1) psi_c)
        C dpart = csub(cscale((R)((16.0 - 2.0 * d) / 12.0), lap), cscale((R)(1.0 / 12.0), dsum));
        C ppart = cscale(c.inv_6h2, csub(edges, cscale((R)(2 * d * (d - 1)), y)));
        lap = cadd(dpart, ppart);
    }
    K[p] = LAP ? lap : rhs_point(c, y, lap, V[p]);
}

// out = a + w b: a stage input Y = Psi + c_j k K_{j-1}
template <typename R>
__global__ void __launch_bounds__(NT) plain_axpy(cplx<R>* out, const cplx<R>* a, R w, const cplx<R>* b,
                                                 int64_t n) {
    int64_t p = blockIdx.x * (int64_t)NT + threadIdx.x;
    if (p < n) out[p] = caxpy(a[p], w, b[p]);
}

// acc = w b (first stage) or acc += w b: the increment sum b_j k K_j
template <typename R, bool FIRST>
__global__ void __launch_bounds__(NT) plain_acc(cplx<R>* acc, R w, const cplx<R>* b, int64_t n) {
    int64_t p = blockIdx.x * (int64_t)NT + threadIdx.x;
    if (p < n) acc[p] = FIRST ? cscale(w, b[p]) : caxpy(acc[p], w, b[p]);
}

// psi += acc, compensated in FP32 when lo is given
template <typename R>
__global__ void __launch_bounds__(NT) plain_final(cplx<R>* psi, cplx<R>* lo, const cplx<R>* acc, int64_t n,
                                                  int* flag) {
    int64_t p = blockIdx.x * (int64_t)NT + threadIdx.x;
    if (p >= n || refused(flag)) return;
    cplx<R> v = psi[p];
    const cplx<R> d = acc[p];
    if constexpr (sizeof(R) == 4) {
        if (lo) {
            cplx<R> l = lo[p];
            kahan_add(v.x, l.x, d.x);
            kahan_add(v.y, l.y, d.y);
            lo[p] = l;
        } else {
            v = cadd(v, d);
        }
    } else {
        v = cadd(v, d);
    }
    psi[p] = v;
    if (!(isfinite(v.x) && isfinite(v.y))) atomicOr(flag, 1);
}

Grid3 make_grid(const PlainLaunch& L) {
    Grid3 g;
    g.dim = L.dim;
    g.bc = L.bc;
    for (int ax = 0; ax < 3; ++ax) g.n[ax] = ax < L.dim ? (int)L.n[ax] : 1;
    g.stride[0] = 1;
    g.stride[1] = g.n[0];
    g.stride[2] = (int64_t)g.n[0] * g.n[1];
    g.npts = (int64_t)g.n[0] * g.n[1] * g.n[2];
    g.flag = L.flag;
    return g;
}

template <typename R>
cudaError_t step_r(const PlainLaunch& L, cudaStream_t st) {
    using C = cplx<R>;
    const Grid3 g = make_grid(L);
    Coef<R> c = make_coef<R>(L.h, L.a, L.s);
    C* psi = (C*)L.psi;
    C* D = (C*)L.D;
    C* K = (C*)L.K;
    C* Y = (C*)L.Y;
    C* acc = (C*)L.acc;
    const R* V = (const R*)L.V;
    const int64_t n = g.npts;
    const unsigned blocks = (unsigned)((n + NT - 1) / NT);
    const bool msd = L.bc == 1;
    auto F = [&](const C* in, C* out) {
        plain_d<R><<<blocks, NT, 0, st>>>(in, V, D, g, c);
        if (msd) plain_d_msd<R><<<blocks, NT, 0, st>>>(in, V, D, g, c);
        if (L.lap == 1) plain_f<R, true><<<blocks, NT, 0, st>>>(in, D, V, out, g, c);
        else plain_f<R, false><<<blocks, NT, 0, st>>>(in, D, V, out, g, c);
        if (msd) plain_f_msd<R><<<blocks, NT, 0, st>>>(in, out, g);
    };
    // Butcher tableau of classic RK4: nodes c_j, weights b_j (in units of k).
    const double c_node[4] = {0.0, 0.5, 0.5, 1.0};
    const double b_weight[4] = {1.0 / 6.0, 1.0 / 3.0, 1.0 / 3.0, 1.0 / 6.0};
    for (int j = 0; j < 4; ++j) {
        const C* in = psi;
        if (j > 0) {
            plain_axpy<R><<<blocks, NT, 0, st>>>(Y, psi, (R)(c_node[j] * L.dt), K, n);
            in = Y;
        }
        F(in, K);
        const R w = (R)(b_weight[j] * L.dt);
        if (j == 0) plain_acc<R, true><<<blocks, NT, 0, st>>>(acc, w, K, n);
        else plain_acc<R, false><<<blocks, NT, 0, st>>>(acc, w, K, n);
    }
    plain_final<R><<<blocks, NT, 0, st>>>(psi, (C*)L.lo, acc, n, L.flag);
    return cudaGetLastError();
}

template <typename R>
cudaError_t lap_r(const PlainLaunch& L, void* lap_out, cudaStream_t st) {
    using C = cplx<R>;
    const Grid3 g = make_grid(L);
    const Coef<R> c = make_coef<R>(L.h, L.a, L.s);
    const unsigned blocks = (unsigned)((g.npts + NT - 1) / NT);
    const C* psi = (const C*)L.psi;
    const R* V = (const R*)L.V;
    C* D = (C*)L.D;
    plain_d<R><<<blocks, NT, 0, st>>>(psi, V, D, g, c);
    if (L.bc == 1) plain_d_msd<R><<<blocks, NT, 0, st>>>(psi, V, D, g, c);
    if (L.lap == 1) plain_f<R, true, true><<<blocks, NT, 0, st>>>(psi, D, V, (C*)lap_out, g, c);
    else plain_f<R, false, true><<<blocks, NT, 0, st>>>(psi, D, V, (C*)lap_out, g, c);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_plain_step(const PlainLaunch& L, cudaStream_t st) {
    return L.prec == 0 ? step_r<float>(L, st) : step_r<double>(L, st);
}

cudaError_t launch_plain_laplacian(const PlainLaunch& L, void* lap_out, cudaStream_t st) {
    return L.prec == 0 ? lap_r<float>(L, lap_out, st) : lap_r<double>(L, lap_out, st);
}

}  // namespace nlse
