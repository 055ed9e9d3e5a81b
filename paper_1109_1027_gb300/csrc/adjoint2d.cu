// adjoint2d.cu -- reverse-mode (adjoint) kernels for the gradient of a
// final-time loss through RK4 + 2SHOC on a 2D grid with Dirichlet boundaries.
//
// One forward RK4 step (Eq. RK4) reads, with stage inputs Y1 = Psi,
// Y2 = Psi + k/2 K1, Y3 = Psi + k/2 K2, Y4 = Psi + k K3 and K_j = F(Y_j):
//     Psi' = Psi + k/6 (K1 + 2 K2 + 2 K3 + K4).
// Given lam' = dL/dPsi', its reverse visits the stages 4, 3, 2, 1 with
// cotangents w4 = k/6 lam', w3 = k/3 lam' + k Ybar4, w2 = k/3 lam' + k/2 Ybar3,
// w1 = k/6 lam' + k/2 Ybar2, where Ybar_j = J_F(Y_j)^T w_j, and returns
// lam = lam' + Ybar4 + Ybar3 + Ybar2 + Ybar1; dL/dV gathers dF/dV(Y_j)^T w_j.
//
// J_F^T in the real-pair convention (a complex cotangent stores d/dRe + i d/dIm;
// the transpose of z -> alpha z + beta conj(z) is w -> conj(alpha) w + beta conj(w)),
// with F_p = i a Lap_p + i (s|Y_p|^2 - V_p) Y_p at interior p, F_b = 0 (Eq. dbc_ut):
//   u = -i a w on interior points (0 elsewhere)      transpose of "i a Lap"
//   E = u - (1/12) sum of the four axial u           transpose of step 2 in D (Eq. 2d2shocs2)
//   Ybar = (sum of axial interior E - 4 E_interior) / h^2      transpose of step 1 (Eq. 2d2shocs1)
//        + (sum of the four corner u - 4 u) / (6 h^2)           corner terms of step 2
//        + boundary: alpha E + beta conj(E), alpha = -(2s|Y|^2 - V)/a, beta = -s Y^2/a   (Eq. dbc_lap)
//        + interior: -i (2s|Y|^2 - V) w + i s Y^2 conj(w)
//   dL/dV += interior: Im(conj(w) Y);  boundary: Re(conj(E) Y) / a.
// (With the CD Laplacian: E = u and no corner terms.)  The stage kernels
// accumulate dL/dV in FP64.
#include <cfloat>

#include "nlse_device.cuh"

namespace nlse {
namespace {

constexpr int TX = 64, TY = 16, NT = 256;
constexpr int PX = TX + 4, PY = TY + 4;   // u with a 2-point halo
constexpr int DX = TX + 2, DY = TY + 2;   // E with a 1-point halo

template <typename R>
struct AdjIO {
    const cplx<R>* w;      // cotangent of this stage's K (scaled by scale_w)
    R scale_w;
    const cplx<R>* Y;      // this stage's input Y_j
    const R* V;
    const cplx<R>* lamp;   // lam' = dL/dPsi_{n+1}
    cplx<R>* lam;          // running dL/dPsi_n
    cplx<R>* w_next;       // cotangent of the previous stage's K
    double* gV;            // dL/dV, accumulated in FP64
    R cw, cy;              // w_next = cw lam' + cy Ybar
};

template <typename R, bool CD, int J>
__global__ void __launch_bounds__(NT) adj2d_kernel(AdjIO<R> io, Coef<R> c, int nx, int ny, int rows1) {
    using C = cplx<R>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* sU = reinterpret_cast<C*>(smem_raw);   // [PY][PX]
    C* sE = sU + PX * PY;                     // [DY][DX]
    const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY, tid = threadIdx.x;
    // Interior of its stacked instance (rows1 rows each; one instance when rows1 = ny).
    auto interior = [&](int x, int y) {
        if (x <= 0 || x >= nx - 1 || y < 0 || y >= ny) return false;
        const int yl = inst_row(y, rows1);
        return yl > 0 && yl < rows1 - 1;
    };

    for (int i = tid; i < PX * PY; i += NT) {
        const int ly = i / PX, lx = i - ly * PX;
        const int gx = x0 - 2 + lx, gy = y0 - 2 + ly;
        C u = czero<C>();
        if (gx >= 0 && gx < nx && gy >= 0 && gy < ny && interior(gx, gy)) {
            const C w = cscale(io.scale_w, io.w[(int64_t)gy * nx + gx]);
            u = cmake<C>(c.a * w.y, -c.a * w.x);                    // -i a w
        }
        sU[i] = u;
    }
    __syncthreads();
    for (int i = tid; i < DX * DY; i += NT) {
        const int ly = i / DX, lx = i - ly * DX;
        const C* q = sU + (ly + 1) * PX + (lx + 1);
        C e = q[0];
        if (!CD) e = csub(e, cscale((R)(1.0 / 12.0), cadd(cadd(q[1], q[-1]), cadd(q[PX], q[-PX]))));
        sE[i] = e;
    }
    __syncthreads();

    for (int i = tid; i < TX * TY; i += NT) {
        const int ly = i / TX, lx = i - ly * TX;
        const int gx = x0 + lx, gy = y0 + ly;
        if (gx >= nx || gy >= ny) continue;
        const int64_t p = (int64_t)gy * nx + gx;
        const C* e = sE + (ly + 1) * DX + (lx + 1);
        const C* u = sU + (ly + 2) * PX + (lx + 2);
        auto ein = [&](int dx, int dy) {
            return interior(gx + dx, gy + dy) ? e[dy * DX + dx] : czero<C>();
        };
        const bool inner = interior(gx, gy);
        const C esum = cadd(cadd(ein(1, 0), ein(-1, 0)), cadd(ein(0, 1), ein(0, -1)));
        C ybar = cscale(c.inv_h2, csub(esum, cscale((R)4, inner ? e[0] : czero<C>())));
        if (!CD) {
            const C corners = cadd(cadd(u[PX + 1], u[PX - 1]), cadd(u[-PX + 1], u[-PX - 1]));
            ybar = cadd(ybar, cscale(c.inv_6h2, csub(corners, cscale((R)4, u[0]))));
        }
        const C Y = io.Y[p];
        const R v = io.V[(int64_t)inst_row(gy, rows1) * nx + gx];     // V is shared by stacked instances
        const R rho = Y.x * Y.x + Y.y * Y.y;
        const C Y2 = cmake<C>(Y.x * Y.x - Y.y * Y.y, 2 * Y.x * Y.y);   // Y^2
        R gv;
        if (inner) {
            const C w = cscale(io.scale_w, io.w[p]);
            const R g = 2 * c.s * rho - v;
            // -i g w + i s Y^2 conj(w)
            const C sy = cmake<C>(Y2.x * w.x + Y2.y * w.y, Y2.y * w.x - Y2.x * w.y);   // Y^2 conj(w)
            ybar = cadd(ybar, cmake<C>(g * w.y - c.s * sy.y, -g * w.x + c.s * sy.x));
            gv = w.x * Y.y - w.y * Y.x;                                             // Im(conj(w) Y)
        } else {
            const C E = e[0];
            const R alpha = -(2 * c.s * rho - v) * c.inv_a;
            const C ce = cmake<C>(Y2.x * E.x + Y2.y * E.y, Y2.y * E.x - Y2.x * E.y); // Y^2 conj(E)
            ybar = cadd(ybar, cadd(cscale(alpha, E), cscale(-c.s * c.inv_a, ce)));
            gv = (E.x * Y.x + E.y * Y.y) * c.inv_a;                                 // Re(conj(E) Y) / a
        }
        io.gV[p] += (double)gv;
        const C lp = io.lamp[p];
        if constexpr (J == 4) io.lam[p] = cadd(lp, ybar);
        else io.lam[p] = cadd(io.lam[p], ybar);
        if constexpr (J > 1) io.w_next[p] = cadd(cscale(io.cw, lp), cscale(io.cy, ybar));
    }
}

template <typename R, bool CD, int J>
cudaError_t launch_j(const AdjLaunch& L, cudaStream_t st) {
    AdjIO<R> io;
    io.w = (const cplx<R>*)L.w;
    io.scale_w = (R)L.scale_w;
    io.Y = (const cplx<R>*)L.Y;
    io.V = (const R*)L.V;
    io.lamp = (const cplx<R>*)L.lamp;
    io.lam = (cplx<R>*)L.lam;
    io.w_next = (cplx<R>*)L.w_next;
    io.gV = L.gV;
    io.cw = (R)L.cw;
    io.cy = (R)L.cy;
    const int nx = (int)L.nx, ny = (int)L.ny;
    dim3 grid((nx + TX - 1) / TX, (ny + TY - 1) / TY);
    const size_t smem = sizeof(cplx<R>) * (PX * PY + DX * DY);
    auto kern = adj2d_kernel<R, CD, J>;
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    kern<<<grid, NT, smem, st>>>(io, make_coef<R>(L.h, L.a, L.s), nx, ny, (int)(L.rows1 ? L.rows1 : L.ny));
    return cudaGetLastError();
}

template <typename R, bool CD>
cudaError_t launch_r(const AdjLaunch& L, cudaStream_t st) {
    switch (L.j) {
        case 4: return launch_j<R, CD, 4>(L, st);
        case 3: return launch_j<R, CD, 3>(L, st);
        case 2: return launch_j<R, CD, 2>(L, st);
        case 1: return launch_j<R, CD, 1>(L, st);
    }
    return cudaErrorInvalidValue;
}

// L = sum |psi - target|^2 (FP64 partial sums per block) and lam = 2 (psi - target).
template <typename R>
__global__ void __launch_bounds__(256) loss_kernel(const cplx<R>* psi, const cplx<R>* target, cplx<R>* lam,
                                                   double* partials, int64_t n) {
    __shared__ double warp_sum[8];
    double acc = 0.0;
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n; p += (int64_t)gridDim.x * blockDim.x) {
        const cplx<R> a = psi[p], b = target[p];
        const double dx = (double)a.x - (double)b.x, dy = (double)a.y - (double)b.y;
        acc += dx * dx + dy * dy;
        lam[p] = cmake<cplx<R>>((R)(2 * dx), (R)(2 * dy));
    }
    for (int off = 16; off > 0; off >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, off);
    if ((threadIdx.x & 31) == 0) warp_sum[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int w = 0; w < 8; ++w) s += warp_sum[w];
        partials[blockIdx.x] = s;
    }
}

__global__ void sum_kernel(const double* partials, int n, double* out) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        double s = 0.0;
        for (int i = 0; i < n; ++i) s += partials[i];
        *out = s;
    }
}

__global__ void stack_sum_kernel(const double* src, int count, int64_t n, double* dst) {
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < n; q += (int64_t)gridDim.x * blockDim.x) {
        double s = 0.0;
        for (int i = 0; i < count; ++i) s += src[(int64_t)i * n + q];
        dst[q] = s;
    }
}

template <typename R>
__global__ void __launch_bounds__(256) scale_kernel(cplx<R>* z, R f, int64_t n) {
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n; p += (int64_t)gridDim.x * blockDim.x)
        z[p] = cscale(f, z[p]);
}

}  // namespace

cudaError_t launch_scale(int prec, void* z, double f, int64_t n, cudaStream_t st) {
    const int64_t b = (n + 255) / 256;
    const unsigned blocks = (unsigned)(b < 4096 ? (b < 1 ? 1 : b) : 4096);
    if (prec == 0) scale_kernel<float><<<blocks, 256, 0, st>>>((float2*)z, (float)f, n);
    else scale_kernel<double><<<blocks, 256, 0, st>>>((double2*)z, f, n);
    return cudaGetLastError();
}

cudaError_t launch_adjoint_stage_2d(const AdjLaunch& L, cudaStream_t st) {
    const bool cd = L.lap == 1;
    if (L.prec == 0) return cd ? launch_r<float, true>(L, st) : launch_r<float, false>(L, st);
    return cd ? launch_r<double, true>(L, st) : launch_r<double, false>(L, st);
}

cudaError_t launch_stack_sum(const double* src, int count, int64_t n, double* dst, cudaStream_t st) {
    const int64_t b = (n + 255) / 256;
    stack_sum_kernel<<<(unsigned)(b < 4096 ? (b < 1 ? 1 : b) : 4096), 256, 0, st>>>(src, count, n, dst);
    return cudaGetLastError();
}

int loss_num_blocks(int64_t n) {
    int64_t b = (n + 255) / 256;
    return (int)(b < 1024 ? (b < 1 ? 1 : b) : 1024);
}

cudaError_t launch_loss(int prec, const void* psi, const void* target, void* lam, int64_t n, double* partials,
                        int nblocks, double* out, cudaStream_t st) {
    if (prec == 0)
        loss_kernel<float><<<nblocks, 256, 0, st>>>((const float2*)psi, (const float2*)target, (float2*)lam,
                                                    partials, n);
    else
        loss_kernel<double><<<nblocks, 256, 0, st>>>((const double2*)psi, (const double2*)target, (double2*)lam,
                                                     partials, n);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    sum_kernel<<<1, 32, 0, st>>>(partials, nblocks, out);
    return cudaGetLastError();
}

}  // namespace nlse
