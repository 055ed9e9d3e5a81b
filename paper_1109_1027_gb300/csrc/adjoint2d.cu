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
// (With the CD Laplacian: E = u and no corner terms.)  Stages 4, 3, 2 store
// their dL/dV contribution; stage 1 adds the four to the running dL/dV in the
// order 4, 3, 2, 1 (one read-modify-write per step; FP64, or in FP32 runs a
// double-float converted to FP64 when the sweep ends).  The
// per-point arithmetic is in adjoint2d.cuh, shared with the TMA row walk of
// adjoint2d_tma.cuh, which runs the stage wherever its rows are 16-byte
// aligned; the shared-memory tile kernel below serves the rest.
#include <cfloat>

#include "adjoint2d.cuh"
#include "tmap.cuh"

namespace nlse {
namespace {

constexpr int TX = 64, TY = 16, NT = 256;
constexpr int PX = TX + 4, PY = TY + 4;   // u with a 2-point halo
constexpr int DX = TX + 2, DY = TY + 2;   // E with a 1-point halo

template <typename R>
struct AdjIO {
    const cplx<R>* w;      // stored cotangent of this stage's K (w = scale * stored)
    const cplx<R>* Y;      // this stage's input Y_j
    const R* V;
    const cplx<R>* lamp;   // lam' = dL/dPsi_{n+1}
    cplx<R>* lam;          // running dL/dPsi_n
    cplx<R>* w_next;       // cotangent of the previous stage's K
    R* g_out;              // stages 4..2: this stage's dL/dV contribution
    const R* g4;           // stage 1: the contributions of stages 4, 3, 2
    const R* g3;
    const R* g2;
    adj::gacc<R>* gV;      // stage 1: the running dL/dV
};

template <typename R, bool CD, int J>
__global__ void __launch_bounds__(NT) adj2d_kernel(AdjIO<R> io, adj::Coef<R> c, int nx, int ny, int rows1) {
    using C = cplx<R>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* sU = reinterpret_cast<C*>(smem_raw);   // [PY][PX]
    C* sE = sU + PX * PY;                     // [DY][DX]
    __shared__ bool rin[PY];                  // grid rows y0-2 .. y0+TY+1: interior of their instance
    const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY, tid = threadIdx.x;
    if (tid < PY) {
        const int gy = y0 - 2 + tid;
        const int yl = gy >= 0 ? inst_row(gy, rows1) : -1;
        rin[tid] = gy >= 0 && gy < ny && yl > 0 && yl < rows1 - 1;
    }
    __syncthreads();
    // Interior of its stacked instance, by row offset ly from y0 - 2.
    auto interior = [&](int x, int ly) { return x > 0 && x < nx - 1 && rin[ly]; };

    for (int i = tid; i < PX * PY; i += NT) {
        const int ly = i / PX, lx = i - ly * PX;
        const int gx = x0 - 2 + lx, gy = y0 - 2 + ly;
        C u = czero<C>();
        if (gx >= 0 && gx < nx && gy >= 0 && gy < ny) u = adj::u_of(c, io.w[(int64_t)gy * nx + gx], interior(gx, ly));
        sU[i] = u;
    }
    __syncthreads();
    for (int i = tid; i < DX * DY; i += NT) {
        const int ly = i / DX, lx = i - ly * DX;
        const C* q = sU + (ly + 1) * PX + (lx + 1);
        sE[i] = adj::e_of<CD>(q[0], q[1], q[-1], q[PX], q[-PX]);
    }
    __syncthreads();

    for (int i = tid; i < TX * TY; i += NT) {
        const int ly = i / TX, lx = i - ly * TX;
        const int gx = x0 + lx, gy = y0 + ly;
        if (gx >= nx || gy >= ny) continue;
        const int64_t p = (int64_t)gy * nx + gx;
        const C* e = sE + (ly + 1) * DX + (lx + 1);
        const C* u = sU + (ly + 2) * PX + (lx + 2);
        auto ein = [&](int dx, int dy) { return interior(gx + dx, ly + 2 + dy) ? e[dy * DX + dx] : czero<C>(); };
        const bool inner = interior(gx, ly + 2);
        C ybar = adj::ybar_stencil<CD>(c, inner ? e[0] : czero<C>(), ein(1, 0), ein(-1, 0), ein(0, 1), ein(0, -1),
                                       u[0], u[PX + 1], u[PX - 1], u[-PX + 1], u[-PX - 1]);
        const R v = io.V[(int64_t)inst_row(gy, rows1) * nx + gx];     // V is shared by stacked instances
        const R gv = adj::pointwise(c, inner, adj::wscale(c, io.w[p]), e[0], io.Y[p], v, ybar);
        if constexpr (J == 1) {
            io.lam[p] = add2(io.lam[p], ybar);
            io.gV[p] = adj::gv_total(io.gV[p], io.g4[p], io.g3[p], io.g2[p], gv);
        } else {
            const C lp = io.lamp[p];
            io.lam[p] = add2(J == 4 ? lp : io.lam[p], ybar);
            io.w_next[p] = adj::w_next(c, lp, ybar);
            io.g_out[p] = gv;
        }
    }
}

template <typename R, bool CD, int J>
cudaError_t launch_j(const AdjLaunch& L, cudaStream_t st) {
    AdjIO<R> io;
    io.w = (const cplx<R>*)L.w;
    io.Y = (const cplx<R>*)L.Y;
    io.V = (const R*)L.V;
    io.lamp = (const cplx<R>*)L.lamp;
    io.lam = (cplx<R>*)L.lam;
    io.w_next = (cplx<R>*)L.w_next;
    io.g_out = (R*)L.g_out;
    io.g4 = (const R*)L.g_in[0];
    io.g3 = (const R*)L.g_in[1];
    io.g2 = (const R*)L.g_in[2];
    io.gV = (adj::gacc<R>*)L.gV;
    const int nx = (int)L.nx, ny = (int)L.ny;
    dim3 grid((nx + TX - 1) / TX, (ny + TY - 1) / TY);
    const size_t smem = sizeof(cplx<R>) * (PX * PY + DX * DY);
    auto kern = adj2d_kernel<R, CD, J>;
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    kern<<<grid, NT, smem, st>>>(io, adj::make_coef<R>(L.h, L.a, L.s, L.scale_w, L.cw, L.cy), nx, ny,
                                 (int)(L.rows1 ? L.rows1 : L.ny));
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

__global__ void __launch_bounds__(256) gv_double_kernel(const float2* acc, double* out, int64_t n) {
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n; p += (int64_t)gridDim.x * blockDim.x)
        out[p] = adj::gv_double(acc[p]);
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

bool adjoint_2d_tma_eligible(const AdjLaunch& L) {
    if (L.nx % (L.prec == 0 ? 4 : 2) != 0) return false;
    const void* ptrs[10] = {L.w, L.Y, L.V, L.lamp, L.lam, L.w_next, L.g_out, L.g_in[0], L.g_in[1], L.gV};
    for (const void* p : ptrs)
        if ((uintptr_t)p % 16) return false;
    return (uintptr_t)L.g_in[2] % 16 == 0 && encoder() != nullptr;
}

cudaError_t launch_adjoint_stage_2d(const AdjLaunch& L, cudaStream_t st) {
    if (L.walk_rows && adjoint_2d_tma_eligible(L)) {
        switch (L.walk_rows) {
            case 8: return launch_adjoint_2d_tma_rows8(L, st);
            case 32: return launch_adjoint_2d_tma_rows32(L, st);
            default: return launch_adjoint_2d_tma_rows16(L, st);
        }
    }
    const bool cd = L.lap == 1;
    if (L.prec == 0) return cd ? launch_r<float, true>(L, st) : launch_r<float, false>(L, st);
    return cd ? launch_r<double, true>(L, st) : launch_r<double, false>(L, st);
}

cudaError_t launch_gv_double(const void* acc, double* out, int64_t n, cudaStream_t st) {
    const int64_t b = (n + 255) / 256;
    gv_double_kernel<<<(unsigned)(b < 4096 ? (b < 1 ? 1 : b) : 4096), 256, 0, st>>>((const float2*)acc, out, n);
    return cudaGetLastError();
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
