/*
 * nlse.h -- C ABI of libnlse, a GB300 (sm_103a) CUDA library that integrates
 * the nonlinear Schroedinger / Gross-Pitaevskii equation
 *
 *     i Psi_t + a Lap(Psi) - V Psi + s |Psi|^2 Psi = 0,      a > 0   (Eq. NLSE, Sec. 1)
 *
 * on 1D/2D/3D grids with the explicit classic RK4 integrator (Eq. RK4, Sec. 3.1)
 * and the two-step high-order compact (2SHOC) Laplacian of Caplan and
 * Carretero-Gonzalez, arXiv 1109.1027 (Secs. 2.1-2.3, single-storage form).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  - Grid: n[0] (x, fastest), n[1] (y), n[2] (z) points per axis, boundary
 *    points included, one spacing h for every axis (Secs. 2.1-2.3); the first
 *    and last index on every active axis are boundary points.  Storage is
 *    row-major with x contiguous: p = x + n[0] * (y + n[1] * z).
 *  - Psi is interleaved complex: complex64 (float re, float im) when
 *    prec == NLSE_FP32, complex128 when prec == NLSE_FP64.  V is real, float
 *    or double to match.  All pointers named *_dev are device pointers; the
 *    caller owns them.  Device pointers must be 16-byte aligned.
 *  - Streams are cudaStream_t passed as void* (NULL = legacy default stream).
 *    Calls enqueue work on the stream and return without synchronising, except
 *    where stated (nlse_invariants, nlse_invariants_batch, nlse_check,
 *    nlse_run_host, nlse_adjoint).  Failures found on the device (a NaN or
 *    Inf written by a step, a refusal of nlse_run's entry check, a timed-out
 *    wait) are kept in the context's status and returned by the next
 *    nlse_check, which reads and clears them.
 *  - Every call returns an nlse_status.  Nothing aborts, throws or traps on
 *    the device.  nlse_last_error() describes the last failure of the calling
 *    thread.
 *  - A context may be used by one host thread at a time.
 */
#ifndef NLSE_H
#define NLSE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    NLSE_OK = 0,
    NLSE_EINVAL = 1,        /* invalid argument or parameter                         */
    NLSE_ENOMEM = 2,        /* device or host allocation failed                      */
    NLSE_ECUDA = 3,         /* a CUDA runtime call failed (message in nlse_last_error) */
    NLSE_EUNSTABLE = 4,     /* dt exceeds the stability bound of Eq. (kdfull)        */
    NLSE_ENONFINITE = 5,    /* a NaN or Inf appeared in the state                    */
    NLSE_ETIMEOUT = 6,      /* a bounded device-side wait gave up                    */
    NLSE_EUNSUPPORTED = 7,  /* valid request that this build does not implement      */
    NLSE_EBOUNDS = 8        /* bounds-check build (-DNLSE_BOUNDS_CHECK): a kernel met an
                               index outside its array and skipped the access        */
} nlse_status;

/* Boundary conditions of Sec. 3.2. */
typedef enum {
    NLSE_BC_DIRICHLET = 0,  /* Eqs. (dbc_lap), (dbc_ut): Psi_t = 0 on the boundary   */
    NLSE_BC_MSD = 1,        /* Eqs. (msdbc_ut), (msdbc_lap): |Psi|^2 held constant;
                               "b-1" is the inward point with every coordinate
                               clamped into [1, n-2].  1D: fused kernels; 2D and
                               3D: the unfused kernels (interior D, then D_b,
                               interior F, then F_b, each field in device memory).
                               Not with NLSE_LAP_2SHOC_MS in 2D/3D, nor batches.   */
    NLSE_BC_PERIODIC = 2,   /* named in Sec. 3.2, not defined there: n points per
                               axis with spacing h and x_n = x_0 (no duplicated end
                               point); every point interior, indices wrap          */
    NLSE_BC_LAPZERO = 3     /* named in Sec. 3.2: Laplacian-zero, D_b = 0 and the
                               boundary follows the equation with Lap_b = 0,
                               F_b = i (s|Psi_b|^2 - V_b) Psi_b.  Periodic and
                               Laplacian-zero run on the unfused kernels in every
                               dimension; not with NLSE_LAP_2SHOC_MS in 2D/3D,
                               nor batches or nlse_adjoint                         */
} nlse_bc;

/* Arithmetic of the state and the stencil. */
typedef enum {
    NLSE_FP32 = 0,          /* complex64 state with a compensated (Kahan) low part;
                               mass, energy and the stability bound in FP64           */
    NLSE_FP64 = 1           /* complex128 throughout                                  */
} nlse_prec;

/* Laplacian inside F (Sec. 3.1 names 2SHOC and CD). */
typedef enum {
    NLSE_LAP_2SHOC = 0,     /* fourth-order 2SHOC, Secs. 2.1-2.3 (single storage)    */
    NLSE_LAP_CD = 1,        /* second-order central difference, Eq. (dx2)            */
    NLSE_LAP_2SHOC_MS = 2   /* 2SHOC in its multi-storage form, Eqs. (2d2shocMs1-2),
                               (3d2shocMs1-2): one second difference per axis kept
                               apart, then (7/6) sum_a D^a - (1/12) sum_a (D^a at
                               the two neighbours along a); the same operator as
                               NLSE_LAP_2SHOC (results equal up to rounding) with
                               fewer operations.  Dirichlet only in 2D/3D; at a
                               point on the boundary of axis a only, D^a_b is D_b
                               of Eq. (dbc_lap) minus the other axes' second
                               differences (the paper gives no split).  In 1D it
                               is NLSE_LAP_2SHOC.                                  */
} nlse_lap;

/* nlse_params.flags */
#define NLSE_FLAG_NO_STABILITY_CHECK 1u  /* nlse_run skips the entry check of dt  */
#define NLSE_FLAG_STACK 4u               /* dim = 2 only: the state holds n[2] >= 1
                                            instances of the n[0] x n[1] grid, instance
                                            i in rows i n[1] .. (i+1) n[1] - 1 of an
                                            n[0] x (n[1] n[2]) array; all share h, dt,
                                            a, s and V (n[0] x n[1]); each has its own
                                            Dirichlet boundary.  One launch per stage
                                            covers the stack; results per instance
                                            equal a single-grid run bit for bit.
                                            nlse_invariants gives totals over the stack
                                            (dt_max: the smallest bound); nlse_adjoint
                                            the summed loss, dL/dpsi0 per instance and
                                            dL/dV summed over the instances.  Dirichlet
                                            and the fused schedule only.           */
#define NLSE_FLAG_PLAIN_SCHEDULE 2u      /* step unfused, with the storage plan of
                                            Sec. 3.1: the step-1 field D and the RK4
                                            work fields (stage input, slope,
                                            increment) as full device arrays, one
                                            launch per operation (16 per step);
                                            no compensation.  Dirichlet only.  A
                                            baseline.                            */

typedef struct {
    int dim;                /* 1, 2 or 3                                              */
    int64_t n[3];           /* points per axis incl. boundary; n[d] >= 3 for d < dim  */
    double h;               /* grid spacing, > 0                                      */
    double dt;              /* RK4 time step k, > 0                                   */
    double a;               /* dispersion coefficient, > 0                            */
    double s;               /* nonlinearity coefficient (any sign)                    */
    int bc;                 /* nlse_bc                                                */
    int prec;               /* nlse_prec                                              */
    int lap;                /* nlse_lap                                               */
    unsigned flags;         /* NLSE_FLAG_*                                            */
} nlse_params;

typedef struct nlse_ctx nlse_ctx;

/* Creates a solver context for one grid on the current CUDA device: the
 * problem of Eq. (NLSE) (Sec. 1) on the grid of Sec. 2.1, stepped by the RK4
 * of Sec. 3.1 with the boundary rule of Sec. 3.2.
 * V_dev: the potential V (float for FP32, double for FP64), borrowed: it must
 * stay valid and unchanged while the context is used.  The context allocates
 * its own device work space: two stage buffers, the RK4 accumulator, the
 * compensated low part of the FP32 state (zeroed here) and the reduction
 * buffers.  Returns NLSE_EINVAL for dim outside 1..3, n < 3 on an active axis,
 * h, dt or a not positive and finite, or an unknown bc / prec / lap. */
int nlse_create(const nlse_params* p, const void* V_dev, nlse_ctx** out);

/* Creates one context for `count` independent 2D instances of uneven sizes
 * and parameters, advanced together (one launch per RK4 stage covers every
 * instance): each is the problem of Eq. (NLSE) on its own grid (Sec. 2.1)
 * with the Dirichlet rule of Sec. 3.2; the batching has no counterpart in the
 * paper.  p[i] gives instance i's grid, h, dt, a and s; prec, lap, bc
 * and flags must be the same for all, bc Dirichlet, and n[0] a multiple of 4
 * (FP32) or 2 (FP64).  Psi, V and every work array are single flat device
 * buffers: instance i occupies n[0](i) * n[1](i) points starting at element
 * offset sum_{j<i} n[0](j) * n[1](j).  V_dev is that flat potential
 * (borrowed).  nlse_rk4_step, nlse_run, nlse_lap2shoc, nlse_check and
 * nlse_reset_compensation then take the flat Psi; nlse_run's stability check
 * refuses when any instance's dt exceeds its own bound. */
int nlse_create_batch(int count, const nlse_params* p, const void* V_dev, nlse_ctx** out);

/* Number of instances of a batch context (0 for a single-grid context).  No
 * counterpart in the paper, which treats one grid at a time. */
int nlse_batch_count(const nlse_ctx* ctx);

/* Per-instance mass, energy and dt_max (Eq. kdfull) (arrays of
 * nlse_batch_count entries, any may be NULL) of a batch context, as
 * nlse_invariants computes them for one grid.  Synchronises the stream.  Returns NLSE_ENONFINITE if any
 * instance holds a NaN or Inf. */
int nlse_invariants_batch(nlse_ctx* ctx, const void* psi_dev, double* mass, double* energy, double* dt_max,
                          void* stream);

/* Releases the context and its device memory (synchronises the device).  No
 * counterpart in the paper. */
void nlse_destroy(nlse_ctx* ctx);

/* 2SHOC Laplacian (or CD, per params.lap) of psi into lap_dev (same layout).
 * Step 1 is the second-order D (Eqs. 2shoc1d, 2d2shocs1, 3d2shocs), step 2
 * re-differences it (Eqs. 2shoc1d2, 2d2shocs2, 3d2shocs2).  Boundary points
 * receive the step-1 boundary value D_b of Sec. 3.2 (Eq. dbc_lap, or Eq.
 * msdbc_lap for MSD), which the paper states also serves as the boundary of
 * the whole Laplacian.  psi_dev and lap_dev must not overlap. */
int nlse_lap2shoc(nlse_ctx* ctx, const void* psi_dev, void* lap_dev, void* stream);

/* One classic RK4 step of size params.dt (Eq. RK4), in place on psi_dev, with
 * F(Psi) = i[a Lap Psi + (s|Psi|^2 - V) Psi] (Sec. 3.1) and the boundary rule
 * of Sec. 3.2 for F at boundary points.  Four fused stage kernels.  In FP32
 * the state is psi_dev plus the context's compensated low part, which is reset
 * to zero whenever psi_dev differs from the previous call's pointer or
 * nlse_reset_compensation() is called.  No entry check; the state is left
 * unchanged while a refusal of an earlier nlse_run is pending (see nlse_run). */
int nlse_rk4_step(nlse_ctx* ctx, void* psi_dev, void* stream);

/* nsteps RK4 steps in place (same arithmetic as nsteps calls of
 * nlse_rk4_step), stream-ordered: no host synchronisation.  The steps are
 * replays of CUDA graphs of 32, 16, 8, 4, 2 and 1 steps captured on first use
 * for this psi_dev (n = 32 q + r: q replays of the 32-step graph and one of
 * each graph whose bit is set in r).  When the stream is being captured by the
 * caller, the kernels are enqueued directly instead and become part of the
 * caller's graph; the binding of a new psi_dev (FP32: zeroing the compensated
 * part; batches: encoding the tensor maps, which synchronises) then belongs
 * in a call before the capture, e.g. nlse_run(ctx, psi_dev, 0, stream).  Unless NLSE_FLAG_NO_STABILITY_CHECK is set, the steps are
 * preceded on the stream by an entry check on the device: the bound of
 * Eq. (kdfull) of every instance, evaluated in FP64 from the current state,
 * against its dt.  If dt exceeds a bound (or the state holds a NaN or Inf),
 * the check records the refusal in the context's status; the state is then
 * left unchanged by these steps and by every later step until nlse_check,
 * which returns NLSE_EUNSTABLE (or NLSE_ENONFINITE) and clears the refusal.
 * Returns a host-side error (invalid argument, launch failure) directly. */
int nlse_run(nlse_ctx* ctx, void* psi_dev, int64_t nsteps, void* stream);

/* nlse_run (Eq. RK4, Sec. 3.1) on a state in host memory, for callers that
 * keep Psi on the host (no counterpart in the paper):
 * copies psi_host (cbytes of the context's grid or batch; page-locked memory
 * makes the copies asynchronous DMA) into a device buffer the context owns
 * (allocated on first use), runs nsteps steps there, copies the result back
 * into psi_host and synchronises the stream.  A host state has no FP32
 * compensated part: each call starts from psi_host with it zero.  As it
 * synchronises anyway, it returns the context's status as nlse_check does
 * (and clears it): a refusal of the entry check (psi_host unchanged), a
 * non-finite value produced by the steps (psi_host holds the result).
 * A batch context moves the state in up to 16 chunks of consecutive instances
 * of about equal size, on three internal streams ordered after the caller's:
 * a chunk's copy in, its steps and its copy out overlap the neighbouring
 * chunks' (the results are the bits of nlse_run).  Its entry check then runs
 * per chunk: a refusal leaves the refused chunk's instances unchanged, the
 * other chunks are stepped, and the refusal (naming the first refused
 * instance) is returned. */
int nlse_run_host(nlse_ctx* ctx, void* psi_host, int64_t nsteps, void* stream);

/* Mass M = h^d sum |Psi|^2, energy
 * E = h^d sum_interior [ -a Re(conj(Psi) Lap Psi) + V |Psi|^2 - (s/2)|Psi|^4 ]
 * (the paper defines neither; this is the discrete Hamiltonian of Eq. NLSE)
 * and the time-step bound of Eq. (kdfull),
 *   dt_max = sqrt(8) h^2 / (a max{ ||B||_inf, max_{i, g in G} |L_i - g| }),
 *   L_i = (h^2/a)(s|Psi_i|^2 - V_i), G from the Table of Sec. 3.3 (t:sumresults),
 *   B from Table t:bc2 (0 for Dirichlet),
 * all accumulated in FP64 on the device from the state (plus the FP32
 * compensated part when psi_dev is the context's current state).  Synchronises
 * the stream and writes the three host doubles (any may be NULL; with energy
 * NULL the energy sum, the costly FP64 Laplacian, is skipped).  Returns
 * NLSE_ENONFINITE when the state holds a NaN or Inf. */
int nlse_invariants(nlse_ctx* ctx, const void* psi_dev, double* mass, double* energy,
                    double* dt_max, void* stream);   /* single-grid contexts only */

/* Zeroes the FP32 compensated low part (call after writing psi externally).
 * No counterpart in the paper, which computes in FP64 throughout (Sec. 4). */
int nlse_reset_compensation(nlse_ctx* ctx, void* stream);

/* No counterpart in the paper.
 * Synchronises the stream, reads the context's device status and clears it.
 * Returns, in this order of precedence: NLSE_EBOUNDS (bounds-check build
 * only) if a kernel met an index outside its array; NLSE_ETIMEOUT if a kernel gave up a
 * bounded wait for its own data transfers; NLSE_EUNSTABLE if an entry check
 * of nlse_run found dt above the bound of Eq. (kdfull) (the message names the
 * instance, its dt and its bound); NLSE_ENONFINITE if an entry check found a
 * NaN or Inf in the state or an RK4 step since the last check produced one. */
int nlse_check(nlse_ctx* ctx, void* stream);

/* nlse_invariants without a context and without allocating anything.  The
 * paper has no counterpart: this exists for callers that cannot allocate
 * device memory -- code inside a framework that owns all device memory
 * through its own pool or budget, or a latency-critical path that cannot
 * take the device synchronisation a cudaMalloc may cause -- and so cannot
 * create an nlse_ctx.  Same reductions as nlse_invariants for a single grid
 * (p->dt is not used; a stack, NLSE_FLAG_STACK, is refused with
 * NLSE_EUNSUPPORTED; an FP32 state is taken as psi_dev alone, without a
 * compensated part), with the block partials in a static device array of
 * 786,480 bytes that the library holds on every GPU that loads it, for the
 * life of the process.  Grids above 67,108,864 points are rejected with
 * NLSE_EINVAL.  The first call on a device looks the array's address up
 * (cudaGetSymbolAddress) with that device current; make that first call
 * before any stream capture.  All calls share the array: calls that overlap
 * on the GPU (unordered streams) race and must not be issued.  Synchronises
 * the stream; writes the three host doubles (any may be NULL). */
int nlse_invariants_noalloc(const nlse_params* p, const void* psi_dev, const void* V_dev,
                            double* mass, double* energy, double* dt_max, void* stream);

/* Gradient of the final-time loss L = sum_points |Psi_T - target|^2, where
 * Psi_T is the state after nsteps RK4 steps from psi0 (as nlse_run computes
 * it), with respect to psi0 and V: the discrete adjoint of Eq. (RK4) with F
 * of Sec. 3.1, the 2SHOC Laplacian (Secs. 2.2) and the Dirichlet rule
 * (Eqs. dbc_lap, dbc_ut), checkpointed every ckpt_every steps (the reverse
 * sweep recomputes each segment from its checkpoint).  Single-grid 2D
 * Dirichlet contexts.  psi0_dev and target_dev are complex fields of the
 * context's precision (not modified); dpsi0_dev (same type) receives
 * dL/dRe(psi0) + i dL/dIm(psi0); dV_dev receives dL/dV as FP64 (double;
 * accumulated in FP64, or for FP32 contexts as an FP32 double-float of about
 * 48 significant bits); *loss the FP64 loss.  The context allocates its work
 * space on first use: (5 + 4 ckpt_every + c nsteps/ckpt_every) fields of the
 * state's size (c = 2 in FP32, 1 in FP64), as the reverse sweep keeps the four
 * stage inputs of every step of a segment.  Uses the context's compensated
 * part, which then no longer belongs to any caller state.  Synchronises the
 * stream; a refusal of an earlier nlse_run still pending in the context's
 * status (which keeps the state from stepping) is returned and cleared, as
 * nlse_check would. */
int nlse_adjoint(nlse_ctx* ctx, const void* psi0_dev, const void* target_dev, int64_t nsteps,
                 int64_t ckpt_every, void* dpsi0_dev, void* dV_dev, double* loss, void* stream);

/* nlse_adjoint in two halves, for callers that need the loss before they know
 * whether (or with what weight) they want its gradient -- an automatic-
 * differentiation framework's forward and backward calls.  The forward half
 * runs the nsteps RK4 steps of Eq. (RK4) from psi0 with a checkpoint every
 * ckpt_every steps, keeps the checkpoints and dL/dPsi_T in the context's
 * adjoint work space, writes the FP64 loss L = sum |Psi_T - target|^2 to
 * *loss and synchronises the stream.  Arguments and support as nlse_adjoint.
 * The paper has no counterpart (it computes no gradients). */
int nlse_adjoint_forward(nlse_ctx* ctx, const void* psi0_dev, const void* target_dev, int64_t nsteps,
                         int64_t ckpt_every, double* loss, void* stream);

/* The reverse half: the gradients of dloss * L, dL/dpsi0 into dpsi0_dev and
 * dL/dV (FP64) into dV_dev, as nlse_adjoint gives them, from the forward pass
 * the context holds (the segments are recomputed from its checkpoints).  Each
 * forward pass admits one reverse sweep: NLSE_EINVAL without a pending forward
 * pass of nlse_adjoint_forward on this context (nlse_adjoint consumes its own).
 * Other calls on the context in between are allowed.  Synchronises the
 * stream.  The paper has no counterpart. */
int nlse_adjoint_backward(nlse_ctx* ctx, double dloss, void* dpsi0_dev, void* dV_dev, void* stream);

/* Tiling of the streaming kernels (the paper has no counterpart: these are
 * launch-shape choices that leave the arithmetic unchanged; results are bit
 * for bit the same).  Set per context, typically by an autotuner that times
 * the candidates on the actual problem.  Setting a key drops the context's
 * captured time-loop graph; NLSE_TILE_BATCH_NARROW also rebuilds the batch
 * work list (synchronising the device). */
#define NLSE_TILE_ROWS 1          /* 2D: rows per CTA, 8, 16 (default) or 32            */
#define NLSE_TILE_PLANES 2        /* 3D FP32: z planes per CTA, 32 (default), 64 or 128 */
#define NLSE_TILE_BATCH_NARROW 3  /* batch: instances with n[0] <= value get 64-column
                                     tiles, the others 256-column tiles (default 64)    */
#define NLSE_TILE_1D_RESIDENT 4   /* 1D grids of up to 4096 points: a power of two
                                     c <= 16 runs nlse_run / nlse_rk4_step as one
                                     launch for all steps on a cluster of at most c
                                     CTAs (fewer where the grid is too short); 0 the
                                     four tiled launches per step.  Default 16       */
#define NLSE_TILE_2D_FUSE 5       /* 2D FP32 Dirichlet contexts (single grids and
                                     stacks; 2SHOC or CD; rows 16-byte aligned): 1
                                     runs each RK4 step as two launches of two stages
                                     each (temporal blocking: stages 1+2, then 3+4,
                                     with Y_1 and Y_3 kept on chip; 80 instead of
                                     168 bytes moved per point and step), 0 as four
                                     single-stage launches (default).  Other
                                     contexts accept the key and ignore it.        */
#define NLSE_TILE_ADJ_ROWS 6      /* the adjoint's reversed stages (2D): 8
                                     (default), 16 or 32 rows per CTA of the TMA row
                                     walk, 0 the shared-memory tile kernel (which
                                     also serves rows that are not 16-byte
                                     aligned)                                      */
/* Sets one tiling key of the context (no counterpart in the paper).  Returns
 * NLSE_EINVAL for an unknown key or a value outside its range (the context is
 * then unchanged). */
int nlse_set_tiling(nlse_ctx* ctx, int key, int value);
/* Reads one tiling key into *value (its default if never set); no counterpart
 * in the paper.  NLSE_EINVAL for an unknown key or NULL arguments. */
int nlse_get_tiling(const nlse_ctx* ctx, int key, int* value);

/* Self-test of the failure path of the bounded waits; no counterpart in the
 * paper.  Every mbarrier wait of the TMA-fed kernels gives up after a time
 * limit, records NLSE_ETIMEOUT in the context's status and lets the kernel
 * return, so a transfer that never lands cannot hang the GPU.  This enqueues
 * a one-warp kernel that runs exactly that path: it waits, with the same
 * bounded wait, on an mbarrier that nothing completes, gives up after
 * limit_ms (0 < limit_ms <= 1000) and sets the timeout bit; the next
 * nlse_check returns NLSE_ETIMEOUT and clears it.  No copy is issued and
 * nothing traps; the context stays usable. */
int nlse_selftest_timeout(nlse_ctx* ctx, double limit_ms, void* stream);

/* Measurement helper; no counterpart in the paper.  Times a chain of FP64
 * fused multiply-adds on every SM of the current GPU (CUDA events, best of
 * three launches after a warm-up) and writes the rate in FP64 flops per
 * second (2 per FMA) to *flops_per_s: the denominator of the roofline of the
 * FP64 stage kernels, which FP64 arithmetic bounds on this GPU.  Allocates a
 * small output buffer; synchronises the stream. */
int nlse_measure_fp64_rate(double* flops_per_s, void* stream);

/* Human-readable description of the calling thread's last error ("" if none).
 * No counterpart in the paper; the string belongs to the library. */
const char* nlse_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* NLSE_H */
