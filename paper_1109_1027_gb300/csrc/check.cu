// check.cu -- the entry check of nlse_run on the device: the time-step bound
// of Eq. (kdfull) of every instance is evaluated from its state and compared
// with its dt, and the verdict is left in the context's status block, so that
// nlse_run never waits for the host.  When the check refuses (dt above the
// bound, or a NaN or Inf in the state), the status block carries the refusal
// and every RK4 stage-4 kernel leaves the state as it is until nlse_check
// reads and clears it.
//
// Only the extremes of u_i = s|Psi_i|^2 - V_i are needed (L_i = (h^2/a) u_i,
// and rounding is monotone, so max_i fl(h^2/a u_i) = fl(h^2/a max_i u_i)); the
// boundary term B of Table t:bc2 is 0 for the boundary rules this check
// serves (Dirichlet, periodic, Laplacian-zero; MSD contexts take the full
// invariants path).  The extremes are FP64 values.  For a complex64 state
// (hi + compensated lo) the FP64 evaluation of every point would make this an
// FP64-rate-bound pass on a GPU whose FP64 rate is 1/64 of its FP32 rate, so
// each point is first evaluated in FP32 together with a rigorous bound E_i on
// |u32_i - u64_i|.  A warp takes 128 points at a time (4 per lane, each load
// instruction covering 32 consecutive points), bounds their FP32 values,
// reduces max(u32 - E) and min(u32 + E) over the warp with shuffles, and keeps
// only the points that can still be an extreme of the 128 (u32_i + E_i >=
// max_j(u32_j - E_j), and the mirror rule for the minimum): on smooth fields a
// few points per tile.  The warp collects those candidates in a shared buffer
// and forms their FP64 values 32 at a time, every lane busy: an FP64
// instruction issued for a warp with one useful lane costs as much as one
// with 32, and at 1/64 of the FP32 rate per-tile evaluation made the check
// FP64-bound.  The result is the exact FP64 extreme, at the cost of one
// memory pass.
#include <cfloat>
#include <climits>

#include "nlse_device.cuh"
#include "stability.cuh"

namespace nlse {
namespace {

constexpr int kThreads = 256;

struct Ext {
    double umin, umax, bad;
};

__device__ __forceinline__ Ext ext_identity() { return {DBL_MAX, -DBL_MAX, 0.0}; }

__device__ __forceinline__ void ext_combine(Ext& a, const Ext& b) {
    a.umin = fmin(a.umin, b.umin);
    a.umax = fmax(a.umax, b.umax);
    a.bad += b.bad;
}

__device__ Ext ext_block_reduce(Ext a) {
    __shared__ Ext warp_tot[kThreads / 32];
    for (int off = 16; off > 0; off >>= 1) {
        Ext b{__shfl_down_sync(0xffffffffu, a.umin, off), __shfl_down_sync(0xffffffffu, a.umax, off),
              __shfl_down_sync(0xffffffffu, a.bad, off)};
        ext_combine(a, b);
    }
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (lane == 0) warp_tot[w] = a;
    __syncthreads();
    if (w == 0) {
        a = lane < kThreads / 32 ? warp_tot[lane] : ext_identity();
        for (int off = 16; off > 0; off >>= 1) {
            Ext b{__shfl_down_sync(0xffffffffu, a.umin, off), __shfl_down_sync(0xffffffffu, a.umax, off),
                  __shfl_down_sync(0xffffffffu, a.bad, off)};
            ext_combine(a, b);
        }
    }
    return a;
}

// u = s|Psi|^2 - V of one complex64 point (hi + lo) in FP64, with explicit
// roundings (the same expression nlse_invariants evaluates pointwise).
__device__ __forceinline__ double u_fp64(float2 h, float2 l, float v, double s) {
    const double x = __dadd_rn((double)h.x, (double)l.x), y = __dadd_rn((double)h.y, (double)l.y);
    return __fma_rn(s, __fma_rn(x, x, __dmul_rn(y, y)), -(double)v);
}

// FP32 value u32 of u at one complex64 point and a bound E on |u32 - u64|
// (with rho_hi = hi.x^2 + hi.y^2): the compensated part changes rho by
// |2 hi.x lo.x + lo.x^2 + 2 hi.y lo.y + lo.y^2| <= t = (2|hi.x| + |lo.x|)|lo.x|
// + (2|hi.y| + |lo.y|)|lo.y|; the two FP32 roundings of rho32 add 2^-23 rho,
// the FMA of u32 2^-24 |u32|, and s rounded to FP32 2^-24 |s| rho.
// E = 2^-18 (|u32| + |s| rho32) + 2 |s| t + (|s| + 1) 2^-120 covers these
// with a margin of at least 2 and absorbs FP32 underflow; an overflowed u32
// (or an infinite E) makes the point a candidate for both extremes.
__device__ __forceinline__ void u_fp32(float2 h, float2 l, float v, float s32, float abs_s, float& u, float& E) {
    const float rho = __fmaf_rn(h.x, h.x, __fmul_rn(h.y, h.y));
    u = __fmaf_rn(s32, rho, -v);
    const float ax = fabsf(l.x), ay = fabsf(l.y);
    const float t = __fmaf_rn(__fmaf_rn(2.0f, fabsf(h.x), ax), ax, __fmul_rn(__fmaf_rn(2.0f, fabsf(h.y), ay), ay));
    E = __fmaf_rn(2.0f * abs_s, t, __fmaf_rn(ldexpf(1.0f, -18), fabsf(u) + abs_s * rho, (abs_s + 1.0f) * 7.52316385e-37f));
}

constexpr int kWarpPts = 4;                 // points per lane in one warp tile (128 points; 64
                                            // registers, four blocks per SM)
constexpr int kCand = 64;                   // a warp's candidate buffer: one batch of 32 and an overflow

// The candidates of one warp waiting for their FP64 value: the point's
// inputs and which extreme it may be (bit 0: maximum, bit 1: minimum).
struct CandBuf {
    float2 h[kCand], l[kCand];
    float v[kCand];
    int f[kCand];
};

// The points [p0, p1) of one instance (complex64 state + compensated part),
// by the block's warps in tiles of 256 points.  A non-finite input point
// counts as bad (its FP64 value would be non-finite too) and is no candidate.
__device__ __forceinline__ Ext extremes32(const float2* __restrict__ ps, const float2* __restrict__ ls,
                                          const float* __restrict__ vs, int64_t p0, int64_t p1, double s,
                                          CandBuf* cb) {
    Ext e = ext_identity();
    const float s32 = (float)s, abs_s = fabsf(s32);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    int nc = 0;                                 // buffered candidates (the same in every lane)
    // FP64 values of the buffered candidates [0, n), n <= 32, one per lane.
    auto flush = [&](int n) {
        __syncwarp();
        if (lane < n) {
            const double u64 = u_fp64(cb->h[lane], cb->l[lane], cb->v[lane], s);
            if (cb->f[lane] & 1) e.umax = fmax(e.umax, u64);
            if (cb->f[lane] & 2) e.umin = fmin(e.umin, u64);
        }
        __syncwarp();
    };
    for (int64_t tb = p0 + (int64_t)warp * 32 * kWarpPts; tb < p1; tb += (int64_t)nwarps * 32 * kWarpPts) {
        float2 h[kWarpPts], l[kWarpPts];
        float v[kWarpPts], u[kWarpPts], E[kWarpPts];
        bool use[kWarpPts];
#pragma unroll
        for (int k = 0; k < kWarpPts; ++k) {
            const int64_t p = tb + k * 32 + lane;
            use[k] = p < p1;
            h[k] = use[k] ? ps[p] : make_float2(0.f, 0.f);
            l[k] = (use[k] && ls) ? ls[p] : make_float2(0.f, 0.f);
            v[k] = use[k] ? vs[p] : 0.f;
        }
        float lb = -FLT_MAX, ub = FLT_MAX;   // the tile's max(u32 - E), min(u32 + E)
#pragma unroll
        for (int k = 0; k < kWarpPts; ++k) {
            if (use[k] && !(isfinite(h[k].x) && isfinite(h[k].y) && isfinite(l[k].x) && isfinite(l[k].y))) {
                e.bad += 1.0;
                use[k] = false;
            }
            u_fp32(h[k], l[k], v[k], s32, abs_s, u[k], E[k]);
            if (use[k]) {
                lb = fmaxf(lb, u[k] - E[k]);     // a NaN (inf - inf) is ignored by fmaxf / fminf
                ub = fminf(ub, u[k] + E[k]);
            }
        }
        for (int off = 16; off > 0; off >>= 1) {
            lb = fmaxf(lb, __shfl_xor_sync(0xffffffffu, lb, off));
            ub = fminf(ub, __shfl_xor_sync(0xffffffffu, ub, off));
        }
#pragma unroll
        for (int k = 0; k < kWarpPts; ++k) {
            const bool cmax = use[k] && !(u[k] + E[k] < lb);   // true for an infinite or NaN u32
            const bool cmin = use[k] && !(u[k] - E[k] > ub);
            const unsigned m = __ballot_sync(0xffffffffu, cmax || cmin);
            if (cmax || cmin) {
                const int q = nc + __popc(m & ((1u << lane) - 1u));
                cb->h[q] = h[k]; cb->l[q] = l[k]; cb->v[q] = v[k];
                cb->f[q] = (cmax ? 1 : 0) | (cmin ? 2 : 0);
            }
            nc += __popc(m);
            if (nc >= 32) {                     // one full batch; the rest moves to the front
                flush(32);
                if (lane < nc - 32) {
                    cb->h[lane] = cb->h[32 + lane]; cb->l[lane] = cb->l[32 + lane];
                    cb->v[lane] = cb->v[32 + lane]; cb->f[lane] = cb->f[32 + lane];
                }
                __syncwarp();
                nc -= 32;
            }
        }
    }
    if (nc) flush(nc);
    return e;
}

// One complex128 point: FP64 throughout.
__device__ __forceinline__ void point64(Ext& e, double2 p, double v, double s) {
    const double rho = __fma_rn(p.x, p.x, __dmul_rn(p.y, p.y));
    if (!isfinite(rho)) {
        e.bad += 1.0;
        return;
    }
    const double u = __fma_rn(s, rho, -v);
    e.umin = fmin(e.umin, u);
    e.umax = fmax(e.umax, u);
}

// Block b covers one contiguous chunk of the points of one entry (the entry
// whose rows [row0, row1) contain b, row_entry[b]) and writes one row of
// partials.
template <typename R>
__global__ void __launch_bounds__(kThreads) check_partial(const CheckEntry* __restrict__ tab,
                                                           const int* __restrict__ row_entry,
                                                           const cplx<R>* __restrict__ psi,
                                                           const cplx<R>* __restrict__ lo, const R* __restrict__ V,
                                                           double* __restrict__ partials, int row_base) {
    const int b = row_base + blockIdx.x;
    const CheckEntry e = tab[row_entry[b]];
    const int64_t nblk = e.row1 - e.row0;
    const int64_t per = (e.npts + nblk - 1) / nblk;
    const int64_t p0 = (b - e.row0) * per, p1 = min(e.npts, p0 + per);
    const cplx<R>* ps = psi + e.psi_off;
    const cplx<R>* ls = lo ? lo + e.psi_off : nullptr;
    const R* vs = V + e.v_off;
    Ext acc = ext_identity();
    if constexpr (sizeof(R) == 4) {
        __shared__ CandBuf cand[kThreads / 32];
        acc = extremes32(ps, ls, vs, p0, p1, e.s, &cand[threadIdx.x >> 5]);
    } else {
        for (int64_t p = p0 + threadIdx.x; p < p1; p += kThreads) point64(acc, ps[p], vs[p], e.s);
    }
    acc = ext_block_reduce(acc);
    if (threadIdx.x == 0) {
        double* row = partials + (int64_t)b * 3;
        row[0] = acc.umin; row[1] = acc.umax; row[2] = acc.bad;
    }
}

// One block per entry: its rows in a fixed order, then the bound of
// Eq. (kdfull) against the entry's dt.  A refusal sets its status bit; the
// smallest refused entry index is kept for the message, and every entry's
// bound is written to bounds[].
__global__ void __launch_bounds__(kThreads) check_final(const CheckEntry* __restrict__ tab,
                                                         const double* __restrict__ partials,
                                                         double* __restrict__ bounds, StatusBlock* status,
                                                         int inst_base) {
    const int inst = inst_base + (int)blockIdx.x;
    const CheckEntry e = tab[inst];
    Ext a = ext_identity();
    for (int r = e.row0 + threadIdx.x; r < e.row1; r += kThreads) {
        const double* row = partials + (int64_t)r * 3;
        ext_combine(a, Ext{row[0], row[1], row[2]});
    }
    a = ext_block_reduce(a);
    if (threadIdx.x != 0) return;
    const double bound = dt_bound(e.dim, e.h, e.a, e.h2a * a.umin, e.h2a * a.umax, 0.0);
    bounds[inst] = bound;
    int bit = 0;
    if (a.bad != 0.0) bit = kStatusEntryNonFinite;
    else if (!(e.dt <= bound)) bit = kStatusUnstable;
    if (bit) {
        atomicOr(&status->bits, bit);
        atomicMin(&status->inst, inst);
    }
}

// The same verdict from the reduced row of the full invariants reduction
// (mass, energy, min L, max L, max |B|, non-finite count), for MSD contexts.
__global__ void invariants_gate(const double* __restrict__ r, int dim, double h, double a, double dt,
                                double* __restrict__ bound_out, StatusBlock* status) {
    const double bound = dt_bound(dim, h, a, r[2], r[3], r[4]);
    *bound_out = bound;
    int bit = 0;
    if (r[5] != 0.0 || !isfinite(r[0])) bit = kStatusEntryNonFinite;
    else if (!(dt <= bound)) bit = kStatusUnstable;
    if (bit) {
        atomicOr(&status->bits, bit);
        atomicMin(&status->inst, 0);
    }
}

}  // namespace

cudaError_t launch_invariants_gate(const double* reduced, int dim, double h, double a, double dt, double* bound_out,
                                   StatusBlock* status, cudaStream_t st) {
    invariants_gate<<<1, 1, 0, st>>>(reduced, dim, h, a, dt, bound_out, status);
    return cudaGetLastError();
}

int check_rows(int64_t npts) {
    const int64_t want = (npts + kPointsPerCheckRow - 1) / kPointsPerCheckRow;
    return (int)(want < 1 ? 1 : (want > kMaxCheckRowsPerEntry ? kMaxCheckRowsPerEntry : want));
}

cudaError_t launch_entry_check(const CheckLaunch& C, cudaStream_t st) {
    // The entries [inst_base, inst_base + count) and their rows [row_base, row_base + nrows).
    if (C.prec == 0)
        check_partial<float><<<C.nrows, kThreads, 0, st>>>(C.table, C.row_entry, (const float2*)C.psi,
                                                           (const float2*)C.lo, (const float*)C.V, C.partials,
                                                           C.row_base);
    else
        check_partial<double><<<C.nrows, kThreads, 0, st>>>(C.table, C.row_entry, (const double2*)C.psi,
                                                            (const double2*)C.lo, (const double*)C.V, C.partials,
                                                            C.row_base);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    check_final<<<C.count, kThreads, 0, st>>>(C.table, C.partials, C.bounds, C.status, C.inst_base);
    return cudaGetLastError();
}

}  // namespace nlse
