// invariants.cu -- FP64 reductions behind nlse_invariants: mass, energy, the
// extremes of L_i = (h^2/a)(s|Psi_i|^2 - V_i) and of the MSD boundary term
// |B_b| of Table t:bc2, which together give the time-step bound of
// Eq. (kdfull), and a count of non-finite values.  The stability check before
// a run asks for the extremes only and skips the energy.
//
// Pointwise evaluation straight from global memory (this runs every few
// hundred steps, not every stage): each thread takes grid points in a
// grid-stride loop, forms the 2SHOC Laplacian in FP64 where the energy needs
// it, and the block reduces with warp shuffles.  Every block writes one row
// of partials to scratch; a single-block kernel then reduces the rows in a
// fixed order, so the result is deterministic for a given launch shape.
//
// 2D Dirichlet grids (single, stacked or batched) take the energy from a
// tiled pass instead: a block converts its 36 x 12 window of the state to
// FP64 once into shared memory, forms D on the 34 x 10 ring around its
// 32 x 8 tile there, and the Laplacian and the energy density of its points
// from those; the grid-stride pass then skips the energy.  3D Dirichlet
// grids do the same on a 32 x 8 column walking 16 planes (rings of four
// state planes and three D planes).  Evaluating the
// Laplacian point by point from global memory converted every value to FP64
// some thirty times, at an FP64 rate 1/64 of the FP32 rate.
#include <cfloat>

#include "nlse_device.cuh"

namespace nlse {
namespace {

template <typename R>
struct InvView {
    const cplx<R>* psi;
    const cplx<R>* lo;
    const R* V;
    int dim;
    int n[3];
    int64_t stride[3];
    double h2a;        // h^2 / a
    double inv_h2, inv_6h2, a, s, inv_a;
    int bc, lap;
    int rows1;         // 2D: rows per stacked instance (n[1] when not stacked)
    int64_t vpts;      // points of V (one instance: V is shared by a stack)
};

// V at point p (a stack's instances share V).
template <typename R>
__device__ __forceinline__ double v_at(const InvView<R>& v, int64_t p) { return (double)v.V[p % v.vpts]; }

template <typename R>
__device__ __forceinline__ double2 psi_at(const InvView<R>& v, int64_t p) {
    cplx<R> z = v.psi[p];
    double2 r = make_double2((double)z.x, (double)z.y);
    if (v.lo) {
        cplx<R> l = v.lo[p];
        r.x += (double)l.x;
        r.y += (double)l.y;
    }
    return r;
}

template <typename R>
__device__ __forceinline__ bool on_boundary(const InvView<R>& v, const int* c) {
    if (v.bc == 2) return false;                     // periodic: no boundary points
    if (v.dim == 2 && v.rows1 != v.n[1]) {           // a stack: boundary rows of every instance
        const int yl = c[1] % v.rows1;
        if (yl == 0 || yl == v.rows1 - 1) return true;
        return c[0] == 0 || c[0] == v.n[0] - 1;
    }
    for (int ax = 0; ax < v.dim; ++ax)
        if (c[ax] == 0 || c[ax] == v.n[ax] - 1) return true;
    return false;
}

// Storage index of coordinates c; on a periodic grid they wrap.
template <typename R>
__device__ __forceinline__ int64_t index_of(const InvView<R>& v, const int* c) {
    int64_t p = 0;
    for (int ax = 0; ax < 3; ++ax) {
        int x = c[ax];
        if (v.bc == 2) x = x < 0 ? x + v.n[ax] : (x >= v.n[ax] ? x - v.n[ax] : x);
        p += x * v.stride[ax];
    }
    return p;
}

// Index of the point at offsets (d0, d1, d2) from c.
template <typename R>
__device__ __forceinline__ int64_t index_at(const InvView<R>& v, const int* c, int d0, int d1, int d2) {
    const int q[3] = {c[0] + d0, c[1] + d1, c[2] + d2};
    return index_of(v, q);
}

template <typename R>
__device__ __forceinline__ int64_t axial(const InvView<R>& v, const int* c, int ax, int d) {
    return index_at(v, c, ax == 0 ? d : 0, ax == 1 ? d : 0, ax == 2 ? d : 0);
}

// Step-1 D at an interior point: sum of axial neighbours minus 2d centre, / h^2.
template <typename R>
__device__ double2 d_interior(const InvView<R>& v, const int* c) {
    int64_t p = index_of(v, c);
    double2 ctr = psi_at(v, p);
    double2 sum = make_double2(0.0, 0.0);
    for (int ax = 0; ax < v.dim; ++ax) {
        double2 u = psi_at(v, axial(v, c, ax, 1));
        double2 w = psi_at(v, axial(v, c, ax, -1));
        sum.x += u.x + w.x;
        sum.y += u.y + w.y;
    }
    double k = 2.0 * v.dim;
    return make_double2((sum.x - k * ctr.x) * v.inv_h2, (sum.y - k * ctr.y) * v.inv_h2);
}

// The closest interior point of a boundary point: every coordinate clamped into [1, n-2].
template <typename R>
__device__ __forceinline__ void inward(const InvView<R>& v, const int* c, int* q) {
    for (int ax = 0; ax < 3; ++ax) q[ax] = c[ax];
    for (int ax = 0; ax < v.dim; ++ax) q[ax] = min(max(c[ax], 1), v.n[ax] - 2);
}

// Step-1 D at any point, with the boundary rule of Sec. 3.2.
template <typename R>
__device__ double2 d_any(const InvView<R>& v, const int* c) {
    if (!on_boundary(v, c)) return d_interior(v, c);
    int64_t b = index_of(v, c);
    double2 pb = psi_at(v, b);
    double Nb = v.s * (pb.x * pb.x + pb.y * pb.y) - v_at(v, b);
    if (v.bc == 3) return make_double2(0.0, 0.0);                 // Laplacian-zero
    if (v.bc == 0) return make_double2(-Nb * v.inv_a * pb.x, -Nb * v.inv_a * pb.y);
    int q[3];
    inward(v, c, q);
    int64_t qi = index_of(v, q);
    double2 pq = psi_at(v, qi);
    double2 dq = d_interior(v, q);
    double Nq = v.s * (pq.x * pq.x + pq.y * pq.y) - v_at(v, qi);
    double re_ratio = (dq.x * pq.x + dq.y * pq.y) / (pq.x * pq.x + pq.y * pq.y);
    double f = re_ratio + (Nq - Nb) * v.inv_a;
    return make_double2(f * pb.x, f * pb.y);
}

// Laplacian at an interior point: CD (D itself) or 2SHOC step 2 in the form
// common to Eqs. (2shoc1d2), (2d2shocs2), (3d2shocs2):
//   ((16 - 2d)/12) D_c - (1/12) sum_axial D + (1/(6h^2)) (sum_edges Psi - 2d(d-1) Psi_c).
template <typename R>
__device__ double2 lap_interior(const InvView<R>& v, const int* c) {
    double2 dc = d_interior(v, c);
    if (v.lap == 1) return dc;
    const int d = v.dim;
    double2 dsum = make_double2(0.0, 0.0);
    for (int ax = 0; ax < d; ++ax)
        for (int sg = -1; sg <= 1; sg += 2) {
            int q[3] = {c[0], c[1], c[2]};
            q[ax] += sg;
            double2 t = d_any(v, q);
            dsum.x += t.x;
            dsum.y += t.y;
        }
    double2 edges = make_double2(0.0, 0.0);
    int64_t p = index_of(v, c);
    for (int a1 = 0; a1 < d; ++a1)
        for (int a2 = a1 + 1; a2 < d; ++a2)
            for (int s1 = -1; s1 <= 1; s1 += 2)
                for (int s2 = -1; s2 <= 1; s2 += 2) {
                    int off[3] = {0, 0, 0};
                    off[a1] = s1;
                    off[a2] = s2;
                    double2 t = psi_at(v, index_at(v, c, off[0], off[1], off[2]));
                    edges.x += t.x;
                    edges.y += t.y;
                }
    double2 pc = psi_at(v, p);
    double wc = (16.0 - 2.0 * d) / 12.0, we = 2.0 * d * (d - 1);
    return make_double2(wc * dc.x - dsum.x / 12.0 + (edges.x - we * pc.x) * v.inv_6h2,
                        wc * dc.y - dsum.y / 12.0 + (edges.y - we * pc.y) * v.inv_6h2);
}

struct Acc {
    double mass, energy, lmin, lmax, bmax, nonfinite;
};

__device__ __forceinline__ void acc_combine(Acc& a, const Acc& b) {
    a.mass += b.mass;
    a.energy += b.energy;
    a.lmin = fmin(a.lmin, b.lmin);
    a.lmax = fmax(a.lmax, b.lmax);
    a.bmax = fmax(a.bmax, b.bmax);
    a.nonfinite += b.nonfinite;
}

__device__ __forceinline__ Acc acc_shfl_down(const Acc& a, int off) {
    Acc b;
    b.mass = __shfl_down_sync(0xffffffffu, a.mass, off);
    b.energy = __shfl_down_sync(0xffffffffu, a.energy, off);
    b.lmin = __shfl_down_sync(0xffffffffu, a.lmin, off);
    b.lmax = __shfl_down_sync(0xffffffffu, a.lmax, off);
    b.bmax = __shfl_down_sync(0xffffffffu, a.bmax, off);
    b.nonfinite = __shfl_down_sync(0xffffffffu, a.nonfinite, off);
    return b;
}

__device__ __forceinline__ Acc acc_identity() {
    Acc a;
    a.mass = a.energy = a.nonfinite = 0.0;
    a.lmin = DBL_MAX;
    a.lmax = -DBL_MAX;
    a.bmax = 0.0;
    return a;
}

// Block reduction; thread 0 returns the block total.
__device__ Acc block_reduce(Acc a) {
    __shared__ Acc warp_tot[kInvThreads / 32];
    for (int off = 16; off > 0; off >>= 1) acc_combine(a, acc_shfl_down(a, off));
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (lane == 0) warp_tot[w] = a;
    __syncthreads();
    if (w == 0) {
        a = lane < kInvThreads / 32 ? warp_tot[lane] : acc_identity();
        for (int off = 16; off > 0; off >>= 1) acc_combine(a, acc_shfl_down(a, off));
    }
    return a;
}

// ENERGY = false leaves the energy sum at zero: the time-step bound needs
// only the pointwise extremes (and, for MSD, the boundary term), which read
// each point once, while the energy's FP64 Laplacian is the costly part.
// Accumulates the points first, first + stride, ... of one grid into a.
// Coordinates are formed (three integer divisions) only where they are
// needed: for the energy's Laplacian and the MSD boundary term.
template <typename R, bool ENERGY>
__device__ void accumulate(const InvView<R>& v, int64_t npts, int64_t first, int64_t stride, Acc& a) {
    const bool coords = ENERGY || v.bc == 1;
    const bool shared_v = v.vpts != npts;            // a stack: V indexed within the instance
    for (int64_t p = first; p < npts; p += stride) {
        double2 ps = psi_at(v, p);
        double rho = ps.x * ps.x + ps.y * ps.y;
        double Vp = shared_v ? v_at(v, p) : (double)v.V[p];
        if (!isfinite(rho)) { a.nonfinite += 1.0; continue; }
        a.mass += rho;
        double L = v.h2a * (v.s * rho - Vp);
        a.lmin = fmin(a.lmin, L);
        a.lmax = fmax(a.lmax, L);
        if (!coords) continue;
        int c[3];
        int64_t r = p;
        c[0] = (int)(r % v.n[0]); r /= v.n[0];
        c[1] = (int)(r % v.n[1]); r /= v.n[1];
        c[2] = (int)r;
        if (!on_boundary(v, c)) {
            if (!ENERGY) continue;
            double2 lp = lap_interior(v, c);
            a.energy += -v.a * (ps.x * lp.x + ps.y * lp.y) + Vp * rho - 0.5 * v.s * rho * rho;
        } else if (v.bc == 1) {
            // B_b = (h^2/(i a)) F_q / Psi_q (Table t:bc2); |1/i| = 1.
            int q[3];
            inward(v, c, q);
            int64_t qi = index_of(v, q);
            double2 pq = psi_at(v, qi);
            double2 lq = lap_interior(v, q);
            double Nq = v.s * (pq.x * pq.x + pq.y * pq.y) - v_at(v, qi);
            // F_q / i = a Lap + N Psi; |F_q / Psi_q| = |a Lap + N Psi| / |Psi|.
            double fx = v.a * lq.x + Nq * pq.x, fy = v.a * lq.y + Nq * pq.y;
            double B = v.h2a * sqrt((fx * fx + fy * fy) / (pq.x * pq.x + pq.y * pq.y));
            a.bmax = fmax(a.bmax, B);
        }
    }
}

// ---- the tiled energy pass (2D, Dirichlet) ------------------------------

constexpr int kETX = 32, kETY = 8;                    // a block's tile: one point per thread
constexpr int kEPX = kETX + 4, kEPY = kETY + 4;       // the state with a 2-point halo
constexpr int kEDX = kETX + 2, kEDY = kETY + 2;       // D with a 1-point halo
static_assert(kETX * kETY == kInvThreads, "one point per thread");

template <typename R>
struct EGrid {
    const cplx<R>* psi;
    const cplx<R>* lo;
    const R* V;                 // rows1 rows (shared by a stack's instances)
    int nx, ny, rows1;          // ny: all rows of a stack; the Dirichlet rows are 0 and rows1-1 of each
    int lap;
    double a, s, inv_a, inv_h2, inv_6h2;
};

// Sum over the block of one double per thread, in a fixed order; thread 0
// returns it.
__device__ double block_sum(double x) {
    __shared__ double warp_tot[kInvThreads / 32];
    for (int off = 16; off > 0; off >>= 1) x += __shfl_down_sync(0xffffffffu, x, off);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    __syncthreads();                                   // warp_tot may still be read by a previous call
    if (lane == 0) warp_tot[w] = x;
    __syncthreads();
    if (w == 0) {
        x = lane < kInvThreads / 32 ? warp_tot[lane] : 0.0;
        for (int off = 16; off > 0; off >>= 1) x += __shfl_down_sync(0xffffffffu, x, off);
    }
    return x;
}

// The energy density -a Re(conj(Psi) Lap Psi) + V |Psi|^2 - (s/2) |Psi|^4
// summed over the interior points of the tile at (x0, y0); thread 0 returns
// the block's sum.  D, the Laplacian and the density follow d_interior,
// d_any (Dirichlet) and lap_interior above, term by term.
template <typename R>
__device__ double energy_tile(const EGrid<R>& g, int x0, int y0) {
    __shared__ double2 sP[kEPY * kEPX];
    __shared__ double2 sD[kEDY * kEDX];
    const int t = threadIdx.x;
    auto vat = [&](int y, int x) { return (double)g.V[(int64_t)(y % g.rows1) * g.nx + x]; };
    for (int i = t; i < kEPY * kEPX; i += kInvThreads) {
        const int ly = i / kEPX, lx = i - ly * kEPX;
        const int x = x0 - 2 + lx, y = y0 - 2 + ly;
        double2 v = make_double2(0.0, 0.0);
        if (x >= 0 && x < g.nx && y >= 0 && y < g.ny) {
            const int64_t p = (int64_t)y * g.nx + x;
            const cplx<R> z = g.psi[p];
            v = make_double2((double)z.x, (double)z.y);
            if (g.lo) {
                const cplx<R> l = g.lo[p];
                v.x += (double)l.x;
                v.y += (double)l.y;
            }
        }
        sP[i] = v;
    }
    __syncthreads();
    for (int i = t; i < kEDY * kEDX; i += kInvThreads) {
        const int ly = i / kEDX, lx = i - ly * kEDX;
        const int x = x0 - 1 + lx, y = y0 - 1 + ly;
        const double2* c = sP + (ly + 1) * kEPX + (lx + 1);
        double2 d = make_double2(0.0, 0.0);
        if (x >= 0 && x < g.nx && y >= 0 && y < g.ny) {
            const int yl = y % g.rows1;
            if (x == 0 || x == g.nx - 1 || yl == 0 || yl == g.rows1 - 1) {
                const double Nb = g.s * (c[0].x * c[0].x + c[0].y * c[0].y) - vat(y, x);
                d = make_double2(-Nb * g.inv_a * c[0].x, -Nb * g.inv_a * c[0].y);
            } else {
                double2 sum = make_double2(0.0, 0.0);
                sum.x += c[1].x + c[-1].x;
                sum.y += c[1].y + c[-1].y;
                sum.x += c[kEPX].x + c[-kEPX].x;
                sum.y += c[kEPX].y + c[-kEPX].y;
                d = make_double2((sum.x - 4.0 * c[0].x) * g.inv_h2, (sum.y - 4.0 * c[0].y) * g.inv_h2);
            }
        }
        sD[i] = d;
    }
    __syncthreads();
    double e = 0.0;
    const int lx = t % kETX, ly = t / kETX;
    const int x = x0 + lx, y = y0 + ly;
    if (x > 0 && x < g.nx - 1 && y < g.ny) {
        const int yl = y % g.rows1;
        if (yl > 0 && yl < g.rows1 - 1) {
            const double2* c = sP + (ly + 2) * kEPX + (lx + 2);
            const double2* dd = sD + (ly + 1) * kEDX + (lx + 1);
            double2 lp = dd[0];
            if (g.lap != 1) {
                double2 dsum = make_double2(0.0, 0.0);
                const double2 dn[4] = {dd[-1], dd[1], dd[-kEDX], dd[kEDX]};
                for (int q = 0; q < 4; ++q) {
                    dsum.x += dn[q].x;
                    dsum.y += dn[q].y;
                }
                double2 edges = make_double2(0.0, 0.0);
                const double2 en[4] = {c[-kEPX - 1], c[kEPX - 1], c[-kEPX + 1], c[kEPX + 1]};
                for (int q = 0; q < 4; ++q) {
                    edges.x += en[q].x;
                    edges.y += en[q].y;
                }
                lp = make_double2(1.0 * dd[0].x - dsum.x / 12.0 + (edges.x - 4.0 * c[0].x) * g.inv_6h2,
                                  1.0 * dd[0].y - dsum.y / 12.0 + (edges.y - 4.0 * c[0].y) * g.inv_6h2);
            }
            const double rho = c[0].x * c[0].x + c[0].y * c[0].y;
            e = -g.a * (c[0].x * lp.x + c[0].y * lp.y) + vat(y, x) * rho - 0.5 * g.s * rho * rho;
        }
    }
    return block_sum(e);
}

template <typename R>
__global__ void __launch_bounds__(kInvThreads) energy2d_partial(EGrid<R> g, double* epartials) {
    const int ntx = (g.nx + kETX - 1) / kETX;
    const int b = blockIdx.x;
    const double e = energy_tile(g, (b % ntx) * kETX, (b / ntx) * kETY);
    if (threadIdx.x == 0) epartials[b] = e;
}

// A batch: block b belongs to instance emap[b], whose tiles are numbered as
// in a launch for that instance alone, so the rows equal those of one launch
// per instance.
template <typename R>
__global__ void __launch_bounds__(kInvThreads) energy2d_batch_partial(const InvBatchEntry* __restrict__ tab,
                                                                      const int* __restrict__ emap,
                                                                      const cplx<R>* psi, const cplx<R>* lo,
                                                                      const R* V, int lap, double* epartials) {
    const int b = blockIdx.x;
    const InvBatchEntry e = tab[emap[b]];
    EGrid<R> g;
    g.psi = psi + e.off;
    g.lo = lo ? lo + e.off : nullptr;
    g.V = V + e.off;
    g.nx = e.nx; g.ny = e.ny; g.rows1 = e.ny;
    g.lap = lap;
    g.a = e.a; g.s = e.s; g.inv_a = 1.0 / e.a;
    g.inv_h2 = 1.0 / (e.h * e.h); g.inv_6h2 = 1.0 / (6.0 * e.h * e.h);
    const int ntx = (e.nx + kETX - 1) / kETX, tl = b - e.erow0;
    const double s = energy_tile(g, (tl % ntx) * kETX, (tl / ntx) * kETY);
    if (threadIdx.x == 0) epartials[b] = s;
}

// ---- 3D: a 32 x 8 column walking kEZ planes ------------------------------

constexpr int kEZ = 16;
constexpr int kEP3 = kEPX * kEPY;                     // a state plane with a 2-point xy halo
constexpr int kED3 = kEDX * kEDY;                     // a D plane with a 1-point xy halo

template <typename R>
struct EGrid3 {
    const cplx<R>* psi;
    const cplx<R>* lo;
    const R* V;
    int nx, ny, nz;
    int lap;
    double a, s, inv_a, inv_h2, inv_6h2;
};

template <typename R>
__global__ void __launch_bounds__(kInvThreads) energy3d_partial(EGrid3<R> g, double* epartials) {
    extern __shared__ __align__(16) unsigned char esm[];
    double2* sP = reinterpret_cast<double2*>(esm);    // [4][kEPY][kEPX], plane z in slot z & 3
    double2* sD = sP + 4 * kEP3;                       // [3][kEDY][kEDX], plane z in slot (z + 3) % 3
    const int ntx = (g.nx + kETX - 1) / kETX, nty = (g.ny + kETY - 1) / kETY;
    const int b = blockIdx.x;
    const int x0 = (b % ntx) * kETX, y0 = ((b / ntx) % nty) * kETY, z0 = (b / (ntx * nty)) * kEZ;
    const int z1 = min(z0 + kEZ, g.nz);
    const int t = threadIdx.x;
    const int64_t plane = (int64_t)g.nx * g.ny;
    auto pslot = [](int z) { return (z + 4) & 3; };
    auto dslot = [](int z) { return (z + 3) % 3; };
    auto load = [&](int z) {
        double2* dst = sP + pslot(z) * kEP3;
        for (int i = t; i < kEP3; i += kInvThreads) {
            const int ly = i / kEPX, lx = i - ly * kEPX;
            const int x = x0 - 2 + lx, y = y0 - 2 + ly;
            double2 v = make_double2(0.0, 0.0);
            if (x >= 0 && x < g.nx && y >= 0 && y < g.ny && z >= 0 && z < g.nz) {
                const int64_t p = z * plane + (int64_t)y * g.nx + x;
                const cplx<R> q = g.psi[p];
                v = make_double2((double)q.x, (double)q.y);
                if (g.lo) {
                    const cplx<R> l = g.lo[p];
                    v.x += (double)l.x;
                    v.y += (double)l.y;
                }
            }
            dst[i] = v;
        }
    };
    auto dplane = [&](int z) {
        double2* dst = sD + dslot(z) * kED3;
        const double2* pm = sP + pslot(z - 1) * kEP3;
        const double2* pc = sP + pslot(z) * kEP3;
        const double2* pp = sP + pslot(z + 1) * kEP3;
        for (int i = t; i < kED3; i += kInvThreads) {
            const int ly = i / kEDX, lx = i - ly * kEDX;
            const int x = x0 - 1 + lx, y = y0 - 1 + ly;
            const int k = (ly + 1) * kEPX + (lx + 1);
            double2 d = make_double2(0.0, 0.0);
            if (x >= 0 && x < g.nx && y >= 0 && y < g.ny && z >= 0 && z < g.nz) {
                const double2 c = pc[k];
                if (x == 0 || x == g.nx - 1 || y == 0 || y == g.ny - 1 || z == 0 || z == g.nz - 1) {
                    const double Nb = g.s * (c.x * c.x + c.y * c.y) - (double)g.V[z * plane + (int64_t)y * g.nx + x];
                    d = make_double2(-Nb * g.inv_a * c.x, -Nb * g.inv_a * c.y);
                } else {
                    double2 sum = make_double2(0.0, 0.0);
                    sum.x += pc[k + 1].x + pc[k - 1].x;
                    sum.y += pc[k + 1].y + pc[k - 1].y;
                    sum.x += pc[k + kEPX].x + pc[k - kEPX].x;
                    sum.y += pc[k + kEPX].y + pc[k - kEPX].y;
                    sum.x += pp[k].x + pm[k].x;
                    sum.y += pp[k].y + pm[k].y;
                    d = make_double2((sum.x - 6.0 * c.x) * g.inv_h2, (sum.y - 6.0 * c.y) * g.inv_h2);
                }
            }
            dst[i] = d;
        }
    };
    for (int z = z0 - 2; z <= z0 + 1; ++z) load(z);
    __syncthreads();
    dplane(z0 - 1);
    dplane(z0);
    __syncthreads();
    double e = 0.0;
    const int lx = t % kETX, ly = t / kETX;
    const int x = x0 + lx, y = y0 + ly;
    const bool inxy = x > 0 && x < g.nx - 1 && y > 0 && y < g.ny - 1;
    for (int z = z0; z < z1; ++z) {
        load(z + 2);                                   // into the slot of plane z - 2
        __syncthreads();
        dplane(z + 1);
        __syncthreads();
        if (inxy && z > 0 && z < g.nz - 1) {
            const int k = (ly + 2) * kEPX + (lx + 2), kd = (ly + 1) * kEDX + (lx + 1);
            const double2* pm = sP + pslot(z - 1) * kEP3;
            const double2* pc = sP + pslot(z) * kEP3;
            const double2* pp = sP + pslot(z + 1) * kEP3;
            const double2* dm = sD + dslot(z - 1) * kED3;
            const double2* dc = sD + dslot(z) * kED3;
            const double2* dp = sD + dslot(z + 1) * kED3;
            double2 lp = dc[kd];
            if (g.lap != 1) {
                // axial D in the order x -+ 1, y -+ 1, z -+ 1; edges in the order of the
                // axis pairs (x, y), (x, z), (y, z), each at (-,-), (-,+), (+,-), (+,+)
                const double2 dn[6] = {dc[kd - 1], dc[kd + 1], dc[kd - kEDX], dc[kd + kEDX], dm[kd], dp[kd]};
                double2 dsum = make_double2(0.0, 0.0);
                for (int q = 0; q < 6; ++q) {
                    dsum.x += dn[q].x;
                    dsum.y += dn[q].y;
                }
                const double2 en[12] = {pc[k - kEPX - 1], pc[k + kEPX - 1], pc[k - kEPX + 1], pc[k + kEPX + 1],
                                        pm[k - 1], pp[k - 1], pm[k + 1], pp[k + 1],
                                        pm[k - kEPX], pp[k - kEPX], pm[k + kEPX], pp[k + kEPX]};
                double2 edges = make_double2(0.0, 0.0);
                for (int q = 0; q < 12; ++q) {
                    edges.x += en[q].x;
                    edges.y += en[q].y;
                }
                const double2 c = pc[k];
                lp = make_double2((10.0 / 12.0) * dc[kd].x - dsum.x / 12.0 + (edges.x - 12.0 * c.x) * g.inv_6h2,
                                  (10.0 / 12.0) * dc[kd].y - dsum.y / 12.0 + (edges.y - 12.0 * c.y) * g.inv_6h2);
            }
            const double2 c = pc[k];
            const double rho = c.x * c.x + c.y * c.y;
            const double v = (double)g.V[z * plane + (int64_t)y * g.nx + x];
            e += -g.a * (c.x * lp.x + c.y * lp.y) + v * rho - 0.5 * g.s * rho * rho;
        }
        __syncthreads();
    }
    e = block_sum(e);
    if (t == 0) epartials[b] = e;
}

// The rows [0, n) in a fixed order into *out (the energy slot of a result row).
__global__ void __launch_bounds__(kInvThreads) energy_final(const double* __restrict__ rows, int n, double* out) {
    double x = 0.0;
    for (int i = threadIdx.x; i < n; i += kInvThreads) x += rows[i];
    x = block_sum(x);
    if (threadIdx.x == 0) *out = x;
}

__global__ void __launch_bounds__(kInvThreads) energy_batch_final(const InvBatchEntry* __restrict__ tab,
                                                                  const double* __restrict__ rows, double* out) {
    const InvBatchEntry e = tab[blockIdx.x];
    double x = 0.0;
    for (int i = e.erow0 + threadIdx.x; i < e.erow1; i += kInvThreads) x += rows[i];
    x = block_sum(x);
    if (threadIdx.x == 0) out[(int64_t)blockIdx.x * kPartialWidth + 1] = x;
}

__device__ __forceinline__ void write_row(double* row, const Acc& a) {
    row[0] = a.mass; row[1] = a.energy; row[2] = a.lmin;
    row[3] = a.lmax; row[4] = a.bmax; row[5] = a.nonfinite;
}

template <typename R, bool ENERGY>
__global__ void __launch_bounds__(kInvThreads) invariants_partial(InvView<R> v, int64_t npts,
                                                                  double* partials) {
    Acc a = acc_identity();
    accumulate<R, ENERGY>(v, npts, blockIdx.x * (int64_t)blockDim.x + threadIdx.x, (int64_t)gridDim.x * blockDim.x,
                          a);
    a = block_reduce(a);
    if (threadIdx.x == 0) write_row(partials + (int64_t)blockIdx.x * kPartialWidth, a);
}

// A batch of 2D instances in one launch: block b belongs to the instance whose
// rows [row0, row1) of partials contain b and covers the points that block
// b - row0 of a single-instance launch of row1 - row0 blocks would, so the
// partial rows are those of one launch per instance, bit for bit.
template <typename R, bool ENERGY>
__global__ void __launch_bounds__(kInvThreads) invariants_batch_partial(const InvBatchEntry* tab, int count,
                                                                        const cplx<R>* psi, const cplx<R>* lo,
                                                                        const R* V, int bc, int lap,
                                                                        double* partials) {
    const int b = blockIdx.x;
    int lo_i = 0, hi_i = count - 1;                 // last instance with row0 <= b
    while (lo_i < hi_i) {
        const int mid = (lo_i + hi_i + 1) / 2;
        if (tab[mid].row0 <= b) lo_i = mid;
        else hi_i = mid - 1;
    }
    const InvBatchEntry e = tab[lo_i];
    InvView<R> v;
    v.psi = psi + e.off;
    v.lo = lo ? lo + e.off : nullptr;
    v.V = V + e.off;
    v.dim = 2;
    v.n[0] = e.nx; v.n[1] = e.ny; v.n[2] = 1;
    v.stride[0] = 1; v.stride[1] = e.nx; v.stride[2] = (int64_t)e.nx * e.ny;
    v.h2a = e.h * e.h / e.a;
    v.inv_h2 = 1.0 / (e.h * e.h);
    v.inv_6h2 = 1.0 / (6.0 * e.h * e.h);
    v.a = e.a; v.s = e.s; v.inv_a = 1.0 / e.a;
    v.bc = bc; v.lap = lap;
    v.rows1 = e.ny;
    v.vpts = (int64_t)e.nx * e.ny;
    const int nblk = e.row1 - e.row0;
    Acc a = acc_identity();
    accumulate<R, ENERGY>(v, (int64_t)e.nx * e.ny, (b - e.row0) * (int64_t)blockDim.x + threadIdx.x,
                          (int64_t)nblk * blockDim.x, a);
    a = block_reduce(a);
    if (threadIdx.x == 0) write_row(partials + (int64_t)b * kPartialWidth, a);
}

__device__ void reduce_rows(const double* partials, int nrows, double* out);

__global__ void __launch_bounds__(kInvThreads) invariants_final(const double* partials, int nrows,
                                                                double* out) {
    reduce_rows(partials, nrows, out);
}

// One block per instance: its rows [row0, row1) into its result row.
__global__ void __launch_bounds__(kInvThreads) invariants_batch_final(const InvBatchEntry* tab,
                                                                      const double* partials, double* out) {
    const InvBatchEntry e = tab[blockIdx.x];
    reduce_rows(partials + (int64_t)e.row0 * kPartialWidth, e.row1 - e.row0,
                out + (int64_t)blockIdx.x * kPartialWidth);
}

__device__ void reduce_rows(const double* partials, int nrows, double* out) {
    Acc a = acc_identity();
    for (int i = threadIdx.x; i < nrows; i += blockDim.x) {
        const double* row = partials + (int64_t)i * kPartialWidth;
        Acc b;
        b.mass = row[0]; b.energy = row[1]; b.lmin = row[2];
        b.lmax = row[3]; b.bmax = row[4]; b.nonfinite = row[5];
        acc_combine(a, b);
    }
    a = block_reduce(a);
    if (threadIdx.x == 0) {
        out[0] = a.mass; out[1] = a.energy; out[2] = a.lmin;
        out[3] = a.lmax; out[4] = a.bmax; out[5] = a.nonfinite;
    }
}

template <typename R>
cudaError_t launch_r(const InvLaunch& L, double* partials, int nblocks, double* out,
                     cudaStream_t st) {
    InvView<R> v;
    v.psi = (const cplx<R>*)L.psi;
    v.lo = (const cplx<R>*)L.lo;
    v.V = (const R*)L.V;
    v.dim = L.dim;
    for (int ax = 0; ax < 3; ++ax) v.n[ax] = ax < L.dim ? (int)L.n[ax] : 1;
    v.stride[0] = 1;
    v.stride[1] = v.n[0];
    v.stride[2] = (int64_t)v.n[0] * v.n[1];
    v.h2a = L.h * L.h / L.a;
    v.inv_h2 = 1.0 / (L.h * L.h);
    v.inv_6h2 = 1.0 / (6.0 * L.h * L.h);
    v.a = L.a; v.s = L.s; v.inv_a = 1.0 / L.a;
    v.bc = L.bc; v.lap = L.lap;
    int64_t npts = (int64_t)v.n[0] * v.n[1] * v.n[2];
    v.rows1 = (int)(L.rows1 ? L.rows1 : v.n[1]);
    v.vpts = (int64_t)v.n[0] * v.rows1 * v.n[2];
    const bool tiled = L.energy && (L.dim == 2 || L.dim == 3) && L.bc == 0 && L.epartials;
    if (L.energy && !tiled) invariants_partial<R, true><<<nblocks, kInvThreads, 0, st>>>(v, npts, partials);
    else invariants_partial<R, false><<<nblocks, kInvThreads, 0, st>>>(v, npts, partials);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    invariants_final<<<1, kInvThreads, 0, st>>>(partials, nblocks, out);
    if ((e = cudaGetLastError()) != cudaSuccess || !tiled) return e;
    int ntiles;
    if (L.dim == 3) {
        EGrid3<R> g;
        g.psi = v.psi; g.lo = v.lo; g.V = v.V;
        g.nx = v.n[0]; g.ny = v.n[1]; g.nz = v.n[2];
        g.lap = L.lap;
        g.a = v.a; g.s = v.s; g.inv_a = v.inv_a; g.inv_h2 = v.inv_h2; g.inv_6h2 = v.inv_6h2;
        ntiles = energy3d_tiles(v.n[0], v.n[1], v.n[2]);
        const size_t smem = sizeof(double2) * (4 * kEP3 + 3 * kED3);
        energy3d_partial<R><<<ntiles, kInvThreads, smem, st>>>(g, L.epartials);
    } else {
        EGrid<R> g;
        g.psi = v.psi; g.lo = v.lo; g.V = v.V;
        g.nx = v.n[0]; g.ny = v.n[1]; g.rows1 = v.rows1;
        g.lap = L.lap;
        g.a = v.a; g.s = v.s; g.inv_a = v.inv_a; g.inv_h2 = v.inv_h2; g.inv_6h2 = v.inv_6h2;
        ntiles = energy2d_tiles(v.n[0], v.n[1]);
        energy2d_partial<R><<<ntiles, kInvThreads, 0, st>>>(g, L.epartials);
    }
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    energy_final<<<1, kInvThreads, 0, st>>>(L.epartials, ntiles, out + 1);
    return cudaGetLastError();
}

}  // namespace

int energy2d_tiles(int64_t nx, int64_t ny) {
    return (int)(((nx + kETX - 1) / kETX) * ((ny + kETY - 1) / kETY));
}

int energy3d_tiles(int64_t nx, int64_t ny, int64_t nz) {
    return (int)(((nx + kETX - 1) / kETX) * ((ny + kETY - 1) / kETY) * ((nz + kEZ - 1) / kEZ));
}

int inv_num_blocks(const InvLaunch& L, int num_sms) {
    int64_t npts = 1;
    for (int ax = 0; ax < L.dim; ++ax) npts *= L.n[ax];
    int64_t want = (npts + kInvThreads - 1) / kInvThreads;
    int64_t cap = (int64_t)num_sms * 4;
    return (int)(want < cap ? want : cap);
}

cudaError_t launch_invariants(const InvLaunch& L, double* partials, int nblocks, double* out,
                              cudaStream_t st) {
    return L.prec == 0 ? launch_r<float>(L, partials, nblocks, out, st)
                       : launch_r<double>(L, partials, nblocks, out, st);
}

namespace {
template <typename R>
cudaError_t launch_batch_r(const InvBatchLaunch& B, cudaStream_t st) {
    const cplx<R>* psi = (const cplx<R>*)B.psi;
    const cplx<R>* lo = (const cplx<R>*)B.lo;
    const R* V = (const R*)B.V;
    const bool tiled = B.energy && B.bc == 0 && B.emap;
    if (B.energy && !tiled)
        invariants_batch_partial<R, true><<<B.nrows, kInvThreads, 0, st>>>(B.table, B.count, psi, lo, V, B.bc, B.lap,
                                                                           B.partials);
    else
        invariants_batch_partial<R, false><<<B.nrows, kInvThreads, 0, st>>>(B.table, B.count, psi, lo, V, B.bc, B.lap,
                                                                            B.partials);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    invariants_batch_final<<<B.count, kInvThreads, 0, st>>>(B.table, B.partials, B.out);
    if ((e = cudaGetLastError()) != cudaSuccess || !tiled) return e;
    energy2d_batch_partial<R><<<B.etiles, kInvThreads, 0, st>>>(B.table, B.emap, psi, lo, V, B.lap, B.epartials);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    energy_batch_final<<<B.count, kInvThreads, 0, st>>>(B.table, B.epartials, B.out);
    return cudaGetLastError();
}
}  // namespace

cudaError_t launch_invariants_batch(const InvBatchLaunch& B, cudaStream_t st) {
    return B.prec == 0 ? launch_batch_r<float>(B, st) : launch_batch_r<double>(B, st);
}

}  // namespace nlse
