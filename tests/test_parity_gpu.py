"""Parity of the CUDA library with the FP64 CPU oracle, through the C ABI.

Every input is seeded and synthetic (paper_1109_1027_gb300.workloads); both
sides receive identical bytes (for FP32 the oracle is fed the FP32-rounded
input).  Tolerances:

* FP64: 1e-12 relative to the field's scale.  The two sides differ only in
  rounding order (and FMA contraction on the GPU), a few ulps per operation.
* FP32, one evaluation of the Laplacian: 2e-6 x max|psi| x (sum of the
  stencil's |coefficients|)/h^2.  The stencil cancels terms of size
  max|psi|/h^2, so the absolute error is a few FP32 ulps (6e-8) of that scale
  times the ~25 operations.
* FP32 state after RK4 steps: 1e-5 relative L2 (the tolerance the FP32 path
  is specified to), and 1e-5 x max|psi| pointwise.
"""
import numpy as np
import pytest
import torch

import oracle
import paper_experiments as pe
from paper_1109_1027_gb300 import nlse
from paper_1109_1027_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

DEV = "cuda:0"


def to_dev(arr, prec):
    if np.iscomplexobj(arr):
        dt = torch.complex64 if prec == "fp32" else torch.complex128
    else:
        dt = torch.float32 if prec == "fp32" else torch.float64
    return torch.from_numpy(np.ascontiguousarray(arr)).to(DEV).to(dt).contiguous()


def rounded(arr, prec):
    """The bytes the GPU sees, as FP64 numpy for the oracle."""
    if prec == "fp64":
        return np.asarray(arr)
    if np.iscomplexobj(arr):
        return np.asarray(arr).astype(np.complex64).astype(np.complex128)
    return np.asarray(arr).astype(np.float32).astype(np.float64)


def lap_scale(psi, h, dim):
    return np.abs(psi).max() * (64.0 / 12.0) * dim / h ** 2 * 2


def rel_l2(a, b):
    return float(np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel()))


SHAPES = {
    1: [(3,), (5,), (1030,), (3001,)],
    # widths divisible by 4 run the TMA-fed streaming kernel (ragged CTA
    # tails in x and y included); the others the generic tile kernel
    2: [(3, 3), (17, 70), (40, 131), (67, 200), (45, 260), (100, 388), (33, 4), (70, 128)],
    # widths divisible by 4 run the TMA-fed FP32 kernel (ragged tiles in x, y
    # and z, z spanning two 64-plane chunks); the others the generic kernel
    3: [(3, 3, 3), (9, 20, 37), (35, 18, 40), (70, 33, 19), (70, 40, 100), (5, 17, 64)],
}
LAPS = ("2shoc", "cd", "2shoc_ms")
OLAP = {"2shoc": oracle.LAP_2SHOC, "cd": oracle.LAP_CD, "2shoc_ms": oracle.LAP_2SHOC_MS}
CASES = [(shape, prec, lap) for d in (1, 2, 3) for shape in SHAPES[d]
         for prec in ("fp64", "fp32") for lap in LAPS]


def _msd_field(shape, seed):
    """A smooth field of nearly constant modulus (a plane wave times a mild
    bump, plus 1e-3 noise), the kind of state the MSD rule is made for.  On
    white-noise fields the MSD boundary in 2D/3D is unstable even at half the
    bound of Eq. (kdfull) -- in the oracle as on the GPU -- because that bound
    linearises the boundary rule."""
    rng = np.random.Generator(np.random.PCG64(seed))
    xs = wl.mesh(shape, -1.0, 1.0)
    kvec = rng.uniform(-1.5, 1.5, len(shape))
    c0 = rng.uniform(-0.3, 0.3, len(shape))
    phase = sum(k * x for k, x in zip(kvec, xs))
    r2 = sum((x - c) ** 2 for x, c in zip(xs, c0))
    return 2.5 * np.exp(1j * phase) * (1 + 0.2 * np.exp(-r2 / 0.2)) + 1e-3 * wl.random_field(shape, seed=seed + 7)


def _problem(shape, seed):
    psi = wl.random_field(shape, seed=seed)
    V = wl.random_potential(shape, seed=seed + 1, scale=2.0)
    return psi, V


@pytest.mark.parametrize("shape,prec,lap", CASES)
def test_laplacian_matches_oracle(shape, prec, lap):
    h, a, s = 0.37, 0.8, -1.3
    psi, V = _problem(shape, 100 + len(shape))
    psi_r, V_r = rounded(psi, prec), rounded(V, prec)
    ref = oracle.laplacian(oracle.Problem(shape, h, a, s, lap=OLAP[lap]), psi_r, V_r)
    solver = nlse.Solver(to_dev(V, prec), h, 1e-3, a, s, prec=prec, lap=lap)
    got = solver.lap2shoc(to_dev(psi, prec)).cpu().numpy()
    tol = (1e-12 if prec == "fp64" else 2e-6) * lap_scale(psi_r, h, len(shape))
    assert np.abs(got - ref).max() <= tol


@pytest.mark.parametrize("shape", [(3, 3), (17, 70), (40, 131), (3, 3, 3), (9, 20, 37), (35, 18, 40)])
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_laplacian_msd_multi_d_matches_oracle(shape, prec):
    """MSD step-1 boundary values in 2D/3D, Eq. (msdbc_lap) at the inward
    point (faces: normal neighbour; edges and corners: the diagonal one)."""
    psi, V = _problem(shape, 8)
    psi = psi + 3.0
    h, a, s = 0.21, 1.1, 0.7
    psi_r, V_r = rounded(psi, prec), rounded(V, prec)
    ref = oracle.laplacian(oracle.Problem(shape, h, a, s, bc=oracle.BC_MSD), psi_r, V_r)
    solver = nlse.Solver(to_dev(V, prec), h, 1e-3, a, s, bc="msd", prec=prec)
    got = solver.lap2shoc(to_dev(psi, prec)).cpu().numpy()
    tol = (1e-12 if prec == "fp64" else 4e-6) * lap_scale(psi_r, h, len(shape))
    assert np.abs(got - ref).max() <= tol


OBC = {"periodic": oracle.BC_PERIODIC, "lapzero": oracle.BC_LAPZERO}
MORE_BC = [(shape, prec, bc, lap) for shape in [(3,), (40,), (3, 3), (17, 70), (3, 3, 3), (9, 20, 37)]
           for prec in ("fp64", "fp32") for bc in ("periodic", "lapzero") for lap in ("2shoc", "cd")]


@pytest.mark.parametrize("shape,prec,bc,lap", MORE_BC)
def test_laplacian_periodic_and_lapzero_match_oracle(shape, prec, bc, lap):
    h, a, s = 0.37, 0.8, -1.3
    psi, V = _problem(shape, 120 + len(shape))
    psi_r, V_r = rounded(psi, prec), rounded(V, prec)
    ref = oracle.laplacian(oracle.Problem(shape, h, a, s, bc=OBC[bc], lap=OLAP[lap]), psi_r, V_r)
    solver = nlse.Solver(to_dev(V, prec), h, 1e-3, a, s, bc=bc, prec=prec, lap=lap)
    got = solver.lap2shoc(to_dev(psi, prec)).cpu().numpy()
    tol = (1e-12 if prec == "fp64" else 2e-6) * lap_scale(psi_r, h, len(shape))
    assert np.abs(got - ref).max() <= tol


@pytest.mark.parametrize("shape,prec,bc", [(s_, p_, b_) for s_ in [(1030,), (40, 131), (9, 20, 37)]
                                           for p_ in ("fp64", "fp32") for b_ in ("periodic", "lapzero")])
def test_rk4_steps_periodic_and_lapzero_match_oracle(shape, prec, bc):
    a, s, h = 0.7, -1.1, 0.5
    psi, V = _problem(shape, 330 + sum(shape))
    psi_r, V_r = rounded(psi, prec), rounded(V, prec)
    prob = oracle.Problem(shape, h, a, s, bc=OBC[bc])
    m0, e0, dtmax = oracle.invariants(prob, psi_r, V_r)
    k = 0.5 * dtmax
    ref = oracle.run(prob, psi_r, V_r, k, 5)
    solver = nlse.Solver(to_dev(V, prec), h, k, a, s, bc=bc, prec=prec)
    m, e, d = solver.invariants(to_dev(psi, prec))
    if prec == "fp64":
        assert (m, e, d) == (pytest.approx(m0, rel=1e-12), pytest.approx(e0, rel=1e-11), pytest.approx(dtmax, rel=1e-12))
    x = to_dev(psi, prec)
    solver.run(x, 5)
    solver.check()
    got = x.cpu().numpy()
    scale = np.abs(ref).max()
    if prec == "fp64":
        assert np.abs(got - ref).max() <= 1e-12 * scale
    else:
        assert np.abs(got - ref).max() <= 1e-5 * scale
        assert rel_l2(got, ref) <= 1e-5


def test_laplacian_msd_1d_matches_oracle():
    for n in (3, 4, 1025, 2049):
        for prec in ("fp64", "fp32"):
            psi, V = _problem((n,), 7)
            psi = psi + 3.0           # keep psi away from zero at the boundary neighbours
            h, a, s = 0.21, 1.1, 0.7
            psi_r, V_r = rounded(psi, prec), rounded(V, prec)
            ref = oracle.laplacian(oracle.Problem((n,), h, a, s, bc=oracle.BC_MSD), psi_r, V_r)
            solver = nlse.Solver(to_dev(V, prec), h, 1e-3, a, s, bc="msd", prec=prec)
            got = solver.lap2shoc(to_dev(psi, prec)).cpu().numpy()
            tol = (1e-12 if prec == "fp64" else 4e-6) * lap_scale(psi_r, h, 1)
            assert np.abs(got - ref).max() <= tol, (n, prec)


STEP_CASES = [(shape, prec, lap, "dirichlet") for d in (1, 2, 3) for shape in SHAPES[d][1:]
              for prec in ("fp64", "fp32") for lap in LAPS]
STEP_CASES += [((n,), prec, "2shoc", "msd") for n in (5, 1030, 3001) for prec in ("fp64", "fp32")]
# MSD in 2D and 3D (the unfused kernels carry it), both Laplacians that have it
STEP_CASES += [(shape, prec, lap, "msd") for shape in [(17, 70), (40, 131), (9, 20, 37), (35, 18, 40)]
               for prec in ("fp64", "fp32") for lap in ("2shoc", "cd")]


@pytest.mark.parametrize("shape,prec,lap,bc", STEP_CASES)
def test_rk4_steps_match_oracle(shape, prec, lap, bc):
    a, s = 0.7, -1.1
    h = 0.5
    psi, V = _problem(shape, 300 + sum(shape))
    if bc == "msd" and len(shape) == 1:
        psi = psi + 2.5
    elif bc == "msd":
        psi = _msd_field(shape, 300 + sum(shape))
        h = 2.0 / (min(shape) - 1)
    psi_r, V_r = rounded(psi, prec), rounded(V, prec)
    prob = oracle.Problem(shape, h, a, s, bc=oracle.BC_MSD if bc == "msd" else 0, lap=OLAP[lap])
    _, _, dtmax = oracle.invariants(prob, psi_r, V_r)
    k = 0.5 * dtmax
    nsteps = 5
    ref = oracle.run(prob, psi_r, V_r, k, nsteps)
    solver = nlse.Solver(to_dev(V, prec), h, k, a, s, bc=bc, prec=prec, lap=lap)
    x = to_dev(psi, prec)
    for _ in range(nsteps):
        solver.rk4_step(x)
    solver.check()
    got = x.cpu().numpy()
    scale = np.abs(ref).max()
    if prec == "fp64":
        assert np.abs(got - ref).max() <= 1e-12 * scale
    else:
        assert np.abs(got - ref).max() <= 1e-5 * scale
        assert rel_l2(got, ref) <= 1e-5


@pytest.mark.parametrize("shape", [(1030,), (67, 200), (35, 18, 40)])
@pytest.mark.parametrize("lap", ["2shoc", "cd"])
def test_unfused_schedule_matches_oracle(shape, lap):
    """The paper's own unfused schedule (NLSE_FLAG_PLAIN_SCHEDULE), FP64."""
    a, s, h = 0.7, -1.1, 0.5
    psi, V = _problem(shape, 400 + sum(shape))
    prob = oracle.Problem(shape, h, a, s, lap=oracle.LAP_CD if lap == "cd" else 0)
    _, _, dtmax = oracle.invariants(prob, psi, V)
    k = 0.5 * dtmax
    ref = oracle.run(prob, psi, V, k, 40)
    solver = nlse.Solver(to_dev(V, "fp64"), h, k, a, s, prec="fp64", lap=lap, plain=True)
    x = to_dev(psi, "fp64")
    solver.run(x, 40)
    solver.check()
    assert np.abs(x.cpu().numpy() - ref).max() <= 1e-12 * np.abs(ref).max()


@pytest.mark.parametrize("shape,prec", [((3001,), "fp64"), ((67, 200), "fp32"), ((67, 200), "fp64"),
                                        ((35, 18, 40), "fp32"), ((40, 131), "fp32")])
def test_run_replays_the_same_steps(shape, prec):
    """nlse_run (replays of the cached 32-, 16-, ... 1-step graphs) is
    bit-identical to repeated nlse_rk4_step."""
    psi, V = _problem(shape, 55)
    h, a, s = 0.5, 0.9, 1.0
    prob = oracle.Problem(shape, h, a, s)
    _, _, dtmax = oracle.invariants(prob, rounded(psi, prec), rounded(V, prec))
    Vd = to_dev(V, prec)
    s1 = nlse.Solver(Vd, h, 0.5 * dtmax, a, s, prec=prec)
    s2 = nlse.Solver(Vd, h, 0.5 * dtmax, a, s, prec=prec)
    x1, x2 = to_dev(psi, prec), to_dev(psi, prec)
    s1.run(x1, 70)
    for _ in range(70):
        s2.rk4_step(x2)
    assert torch.equal(x1, x2)


@pytest.mark.parametrize("shape", [(1030,), (67, 200), (35, 18, 40)])
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_invariants_match_oracle(shape, prec):
    psi, V = _problem(shape, 77)
    h, a, s = 0.4, 0.6, -0.9
    psi_r, V_r = rounded(psi, prec), rounded(V, prec)
    m0, e0, d0 = oracle.invariants(oracle.Problem(shape, h, a, s), psi_r, V_r)
    solver = nlse.Solver(to_dev(V, prec), h, 1e-4, a, s, prec=prec)
    m, e, d = solver.invariants(to_dev(psi, prec))
    assert m == pytest.approx(m0, rel=1e-12)
    assert e == pytest.approx(e0, rel=1e-11)
    assert d == pytest.approx(d0, rel=1e-12)


@pytest.mark.parametrize("shape", [(67, 200), (17, 33), (35, 18, 40), (9, 33, 70)])
@pytest.mark.parametrize("lap", ["2shoc", "cd"])
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_tiled_energy_matches_oracle(shape, lap, prec):
    """The tiled energy pass of 2D and 3D Dirichlet grids (32 x 8 tiles; in 3D
    walks of 16 planes), on shapes with ragged tiles in every direction, both
    Laplacian forms, against the oracle's energy."""
    psi, V = _problem(shape, 81)
    h, a, s = 0.45, 0.7, -1.2
    psi_r, V_r = rounded(psi, prec), rounded(V, prec)
    ol = oracle.LAP_CD if lap == "cd" else 0
    m0, e0, d0 = oracle.invariants(oracle.Problem(shape, h, a, s, lap=ol), psi_r, V_r)
    solver = nlse.Solver(to_dev(V, prec), h, 1e-4, a, s, prec=prec, lap=lap)
    m, e, d = solver.invariants(to_dev(psi, prec))
    assert e == pytest.approx(e0, rel=1e-11, abs=1e-12 * abs(m0))
    assert m == pytest.approx(m0, rel=1e-12)
    assert d == pytest.approx(d0, rel=1e-12)


def test_invariants_msd_1d_match_oracle():
    n = 1030
    psi, V = _problem((n,), 78)
    psi = psi + 2.0
    h, a, s = 0.4, 0.6, -0.9
    m0, e0, d0 = oracle.invariants(oracle.Problem((n,), h, a, s, bc=oracle.BC_MSD), psi, V)
    solver = nlse.Solver(to_dev(V, "fp64"), h, 1e-4, a, s, bc="msd", prec="fp64")
    m, e, d = solver.invariants(to_dev(psi, "fp64"))
    assert (m, e, d) == (pytest.approx(m0, rel=1e-12), pytest.approx(e0, rel=1e-11),
                         pytest.approx(d0, rel=1e-12))


def test_invariants_without_energy_give_the_same_mass_and_bound():
    """Skipping the energy sum (the stability check's mode) leaves mass and
    dt_max bit for bit as they are with it, Dirichlet and MSD."""
    for shape, bc, prec in [((130, 77), "dirichlet", "fp32"), ((1030,), "msd", "fp64"), ((20, 18, 33), "dirichlet", "fp64")]:
        psi, V = _problem(shape, 79)
        solver = nlse.Solver(to_dev(V, prec), 0.4, 1e-4, 0.6, -0.9, bc=bc, prec=prec)
        x = to_dev(psi + 2.0, prec)
        m, e, d = solver.invariants(x)
        m2, e2, d2 = solver.invariants(x, energy=False)
        assert (m2, d2) == (m, d) and e2 is None and e != 0.0


def test_dirichlet_boundary_is_bit_exact_over_a_run():
    """Eq. (dbc_ut): F_b = 0, so boundary values never change, in either precision."""
    for prec in ("fp32", "fp64"):
        inst = wl.dark_vortex_2d(n=130, steps=0)
        prob = oracle.Problem(inst.shape, inst.h, inst.a, inst.s)
        _, _, dtmax = oracle.invariants(prob, inst.psi0, inst.V)
        solver = nlse.Solver(to_dev(inst.V, prec), inst.h, 0.5 * dtmax, inst.a, inst.s, prec=prec)
        x = to_dev(inst.psi0, prec)
        x0 = x.clone()
        solver.run(x, 40)
        for sl in [(0, slice(None)), (-1, slice(None)), (slice(None), 0), (slice(None), -1)]:
            assert torch.equal(x[sl], x0[sl])


# -- the workloads at reduced size / steps ------------------------------------

def test_bright_soliton_1d_full_config():
    """1D bright soliton, FP64, n = 2048 on [-40, 40], dt = 0.5 dt_max, 2000
    steps: GPU = oracle to 1e-12 (relative L2), and both follow the exact
    travelling sech soliton to the scheme's accuracy."""
    inst = wl.bright_soliton_1d()
    prob = oracle.Problem(inst.shape, inst.h, inst.a, inst.s)
    _, _, dtmax = oracle.invariants(prob, inst.psi0, inst.V)
    k = 0.5 * dtmax
    ref = oracle.run(prob, inst.psi0, inst.V, k, inst.steps)
    solver = nlse.Solver(to_dev(inst.V, "fp64"), inst.h, k, inst.a, inst.s, prec="fp64")
    x = to_dev(inst.psi0, "fp64")
    solver.run(x, inst.steps)
    got = x.cpu().numpy()
    assert rel_l2(got, ref) <= 1e-12
    x_axis = wl.axis(inst.shape[0], inst.lo, inst.hi)
    exact = pe.bright_soliton(x_axis, inst.steps * k, x0=inst.meta["x0"], c=inst.meta["c"])
    assert rel_l2(got, exact) < 1e-5


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-12), ("fp32", 1e-5)])
def test_dark_vortex_2d_reduced(prec, tol):
    """2D dark vortex on a 256^2 crop of the workload's recipe, 200 steps."""
    inst = wl.dark_vortex_2d(n=256, steps=200)
    prob = oracle.Problem(inst.shape, inst.h, inst.a, inst.s)
    _, _, dtmax = oracle.invariants(prob, inst.psi0, inst.V)
    k = 0.5 * dtmax
    psi_r, V_r = rounded(inst.psi0, prec), rounded(inst.V, prec)
    ref = oracle.run(prob, psi_r, V_r, k, inst.steps)
    solver = nlse.Solver(to_dev(inst.V, prec), inst.h, k, inst.a, inst.s, prec=prec)
    x = to_dev(inst.psi0, prec)
    solver.run(x, inst.steps)
    assert rel_l2(x.cpu().numpy(), ref) <= tol


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-12), ("fp32", 1e-5)])
def test_vortex_ring_3d_reduced(prec, tol):
    """3D vortex ring on a 48^3 grid of the workload's recipe, 60 steps."""
    inst = vr = wl.vortex_ring_3d(n=48, steps=60)
    prob = oracle.Problem(inst.shape, inst.h, inst.a, inst.s)
    _, _, dtmax = oracle.invariants(prob, inst.psi0, inst.V)
    k = 0.5 * dtmax
    psi_r, V_r = rounded(vr.psi0, prec), rounded(vr.V, prec)
    ref = oracle.run(prob, psi_r, V_r, k, inst.steps)
    solver = nlse.Solver(to_dev(inst.V, prec), inst.h, k, inst.a, inst.s, prec=prec)
    x = to_dev(inst.psi0, prec)
    solver.run(x, inst.steps)
    assert rel_l2(x.cpu().numpy(), ref) <= tol


def _crop_one_step(psi, V, inst, k, y, x, r=10):
    """Oracle value of one RK4 step at (y, x): the step's result at a point
    depends only on the state within 8 points (four stages, two points
    each), so it is computed on a window of half-width r >= 9 that keeps
    the grid's real boundary where the window reaches it."""
    ny, nx = psi.shape
    y0, y1 = max(0, y - r), min(ny, y + r + 1)
    x0, x1 = max(0, x - r), min(nx, x + r + 1)
    sub = psi[y0:y1, x0:x1]
    out = oracle.run(oracle.Problem(sub.shape, inst.h, inst.a, inst.s), sub, V[y0:y1, x0:x1], k, 1)
    return out[y - y0, x - x0]


@pytest.mark.parametrize("prec,fuse", [("fp32", 0), ("fp32", 1), ("fp64", 0)])
def test_dark_vortex_2d_full_size_sampled(prec, fuse):
    """The 2048^2 workload in the benchmark's launch configurations (four
    single-stage launches per step, or two stage pairs): one RK4 step through
    nlse_run, checked at sampled points (incl. corners, edges and the vortex
    core) against the oracle on windows."""
    inst = wl.dark_vortex_2d()
    prob_small = oracle.Problem((64, 64), inst.h, inst.a, inst.s)
    psi_r, V_r = rounded(inst.psi0, prec), rounded(inst.V, prec)
    # dt from the oracle's bound on the full state
    _, _, dtmax = oracle.invariants(oracle.Problem(inst.shape, inst.h, inst.a, inst.s), psi_r, V_r)
    k = 0.5 * dtmax
    solver = nlse.Solver(to_dev(inst.V, prec), inst.h, k, inst.a, inst.s, prec=prec,
                         check_stability=False)
    solver.set_tiling(nlse.TILE_2D_FUSE, fuse)
    x = to_dev(inst.psi0, prec)
    solver.run(x, 1)
    got = x.cpu().numpy()
    n = inst.shape[0]
    rng = np.random.Generator(np.random.PCG64(2024))
    pts = [(0, 0), (0, n - 1), (n - 1, 0), (n - 1, n - 1), (1, 1), (n // 2, n // 2), (n // 2 + 1, n // 2),
           (2, n // 3), (n - 2, 700), (63, 64), (64, 63), (1000, 1023)]
    pts += [tuple(int(v) for v in rng.integers(0, n, 2)) for _ in range(36)]
    tol = (1e-12 if prec == "fp64" else 1e-6) * np.abs(psi_r).max()
    del prob_small
    for (yy, xx) in pts:
        ref = _crop_one_step(psi_r, V_r, inst, k, yy, xx)
        assert abs(got[yy, xx] - ref) <= tol, (yy, xx, got[yy, xx], ref)


def _crop_one_step_3d(psi, V, inst, k, z, y, x, r=10):
    """Oracle value of one RK4 step at (z, y, x) from a window of half-width
    r >= 9 (the step's result depends on the state within 8 points)."""
    nz, ny, nx = psi.shape
    sl = tuple(slice(max(0, c - r), min(n, c + r + 1)) for c, n in ((z, nz), (y, ny), (x, nx)))
    sub = psi[sl]
    out = oracle.run(oracle.Problem(sub.shape, inst.h, inst.a, inst.s), sub, V[sl], k, 1)
    return out[z - sl[0].start, y - sl[1].start, x - sl[2].start]


def test_vortex_ring_3d_full_size_sampled():
    """The 512^3 vortex ring in FP32 (the TMA-fed kernel, the benchmark's
    launch configuration): one RK4 step through nlse_run, checked at sampled
    points (corners, faces, the ring core, random points) against the oracle
    on windows."""
    inst = wl.vortex_ring_3d()
    psi_r = inst.psi0.astype(np.complex64).astype(np.complex128)
    V_r = inst.V.astype(np.float32).astype(np.float64)
    Vd = torch.from_numpy(inst.V).to(DEV).float().contiguous()
    x = torch.from_numpy(inst.psi0).to(DEV).to(torch.complex64).contiguous()
    probe = nlse.Solver(Vd, inst.h, 1.0, inst.a, inst.s, prec="fp32", check_stability=False)
    k = 0.5 * probe.invariants(x)[2]
    probe.close()
    solver = nlse.Solver(Vd, inst.h, k, inst.a, inst.s, prec="fp32", check_stability=False)
    solver.run(x, 1)
    n = inst.shape[0]
    cx, cy = inst.meta["centre"]
    ring = int(round((cx + 8.0 + 30.0) / inst.h)), int(round((cy + 30.0) / inst.h))
    pts = [(0, 0, 0), (n - 1, n - 1, n - 1), (0, n // 2, 5), (n // 2, 0, n // 2), (n // 2, n // 2, n - 1),
           (1, 1, 1), (n // 2, ring[1], ring[0]), (n // 2 + 1, ring[1], ring[0] + 1), (63, 64, 31), (64, 63, 32),
           (255, 256, 257)]
    rng = np.random.Generator(np.random.PCG64(303))
    pts += [tuple(int(v) for v in rng.integers(0, n, 3)) for _ in range(20)]
    got = {p: complex(x[p].item()) for p in pts}
    tol = 1e-6 * np.abs(psi_r).max()
    for p in pts:
        ref = _crop_one_step_3d(psi_r, V_r, inst, k, *p)
        assert abs(got[p] - ref) <= tol, (p, got[p], ref)


# -- the paper's accuracy experiments on the GPU -------------------------------

TABLES = pe.read_tables(pe.__file__.replace("paper_experiments.py", "golden/paper_tables.txt"))


def _gpu_runner(name, h, lap):
    st = pe.setup(name, h)
    solver = nlse.Solver(to_dev(st["V"], "fp64"), h, st["k"], st["a"], st["s"],
                         bc="msd" if st["bc"] == 1 else "dirichlet", prec="fp64", lap=lap,
                         check_stability=False)

    def run(p, n):
        x = to_dev(p, "fp64")
        solver.run(x, n)
        return x.cpu().numpy()
    return run


@pytest.mark.parametrize("lap,scheme", [("2shoc", "2SHOC"), ("cd", "CD")])
def test_paper_table_2d_on_gpu(lap, scheme):
    """Fig. f:num2d table (Sec. 4.2), FP64 on the GPU, h = 1 .. 1/8."""
    for i, h in enumerate(pe.E23_H[:4]):
        er, ei = pe.measure("E2", h, _gpu_runner("E2", h, lap))
        assert er == pytest.approx(TABLES[("E2", scheme, "real")][i], rel=2e-4)
        assert ei == pytest.approx(TABLES[("E2", scheme, "imag")][i], rel=2e-4)


def test_paper_table_1d_on_gpu():
    """Fig. f:num1d table (Sec. 4.1), MSD boundaries, FP64 on the GPU: the
    printed orders of the 2SHOC errors to 0.01."""
    got = [pe.measure("E1", h, _gpu_runner("E1", h, "2shoc")) for h in pe.E1_H]
    ref = TABLES[("E1", "2SHOC", "real")]
    for i in range(4):
        o = pe.order(got[i][0], got[i + 1][0], pe.E1_H[i], pe.E1_H[i + 1])
        assert o == pytest.approx(pe.order(ref[i], ref[i + 1], 2, 1), abs=1e-2)


def test_paper_table_3d_on_gpu():
    """Fig. f:num3d table (Sec. 4.3), FP64 on the GPU, h = 1, 1/2, 1/4."""
    for i, h in enumerate(pe.E23_H[:3]):
        er, ei = pe.measure("E3", h, _gpu_runner("E3", h, "2shoc"))
        assert er == pytest.approx(TABLES[("E3", "2SHOC", "real")][i], rel=2e-4)
        assert ei == pytest.approx(TABLES[("E3", "2SHOC", "imag")][i], rel=2e-4)


# -- failure reporting ---------------------------------------------------------

def test_nonfinite_state_is_reported():
    shape = (40, 70)
    psi, V = _problem(shape, 5)
    psi[20, 30] = np.nan
    solver = nlse.Solver(to_dev(V, "fp32"), 0.5, 1e-3, 1.0, 1.0, prec="fp32", check_stability=False)
    x = to_dev(psi, "fp32")
    with pytest.raises(nlse.NLSEError) as ei:
        solver.invariants(x)
    assert ei.value.code == nlse.ENONFINITE
    solver.rk4_step(x)
    with pytest.raises(nlse.NLSEError) as ei:
        solver.check()
    assert ei.value.code == nlse.ENONFINITE
    solver.check()       # the flag was cleared


def test_unstable_time_step_is_refused():
    """The entry check of nlse_run runs on the device: the call itself
    returns, the state is left as it was, and nlse_check reports the refusal
    (then clears it)."""
    shape = (64,)
    psi, V = _problem(shape, 6)
    prob = oracle.Problem(shape, 0.25, 1.0, 0.0)
    _, _, dtmax = oracle.invariants(prob, psi, np.zeros(shape))
    solver = nlse.Solver(to_dev(np.zeros(shape), "fp64"), 0.25, 1.2 * dtmax, 1.0, 0.0, prec="fp64")
    x = to_dev(psi, "fp64")
    x0 = x.clone()
    solver.run(x, 10)
    with pytest.raises(nlse.NLSEError) as ei:
        solver.check()
    assert ei.value.code == nlse.EUNSTABLE
    assert torch.equal(x, x0)
    solver.check()                                  # cleared


def test_bad_tensors_are_rejected():
    solver = nlse.Solver(to_dev(np.zeros((8, 8)), "fp32"), 0.5, 1e-3, 1.0, 1.0)
    with pytest.raises(ValueError):
        solver.rk4_step(torch.zeros((8, 8), dtype=torch.complex128, device=DEV))
    with pytest.raises(ValueError):
        solver.rk4_step(torch.zeros((8, 9), dtype=torch.complex64, device=DEV))
    with pytest.raises(ValueError):
        solver.rk4_step(torch.zeros((8, 8), dtype=torch.complex64))


def test_compensation_resets_when_the_state_changes():
    """The FP32 low part belongs to one state: switching psi buffers resets it,
    so two independent runs from the same start agree bit for bit."""
    inst = wl.dark_vortex_2d(n=96, steps=0)
    prob = oracle.Problem(inst.shape, inst.h, inst.a, inst.s)
    _, _, dtmax = oracle.invariants(prob, inst.psi0, inst.V)
    solver = nlse.Solver(to_dev(inst.V, "fp32"), inst.h, 0.5 * dtmax, inst.a, inst.s)
    a_ = to_dev(inst.psi0, "fp32")
    b_ = to_dev(inst.psi0, "fp32")
    solver.run(a_, 40)
    solver.run(b_, 40)
    assert torch.equal(a_, b_)


# -- tiling choices (launch shape only: results identical bit for bit) ---------

def test_tiling_variants_give_identical_results():
    from paper_1109_1027_gb300 import autotune
    for shape, prec, key, values, lap in [((100, 388), "fp32", nlse.TILE_ROWS, (8, 16, 32), "2shoc"),
                                          ((45, 260), "fp64", nlse.TILE_ROWS, (8, 16, 32), "2shoc"),
                                          ((70, 40, 100), "fp32", nlse.TILE_PLANES, (32, 64, 128), "2shoc"),
                                          ((100, 388), "fp32", nlse.TILE_ROWS, (8, 16, 32), "2shoc_ms"),
                                          ((70, 40, 100), "fp32", nlse.TILE_PLANES, (32, 64, 128), "2shoc_ms")]:
        psi, V = _problem(shape, 600)
        h, a, s = 0.5, 0.9, -1.0
        prob = oracle.Problem(shape, h, a, s)
        _, _, dtmax = oracle.invariants(prob, rounded(psi, prec), rounded(V, prec))
        solver = nlse.Solver(to_dev(V, prec), h, 0.5 * dtmax, a, s, prec=prec, lap=lap)
        outs = []
        for v in values:
            solver.set_tiling(key, v)
            assert solver.get_tiling(key) == v
            x = to_dev(psi, prec)
            solver.run(x, 40)
            outs.append(x)
        for o in outs[1:]:
            assert torch.equal(o, outs[0]), (shape, prec)
        with pytest.raises(nlse.NLSEError):
            solver.set_tiling(key, 7)
        rep = autotune.tune(solver, to_dev(psi, prec), steps=2, use_cache=False)
        assert rep[key]["choice"] in values


@pytest.mark.parametrize("n,prec,bc", [(3, "fp64", "dirichlet"), (1030, "fp32", "dirichlet"), (2048, "fp64", "dirichlet"),
                                       (4096, "fp32", "dirichlet"), (2049, "fp32", "msd"), (5, "fp64", "msd"),
                                       (130, "fp64", "msd"), (4096, "fp64", "msd")])
def test_1d_resident_loop_equals_tiled_steps(n, prec, bc):
    """The resident 1D time loop, on one CTA or spread over a cluster, gives
    the bits of the tiled kernels."""
    psi, V = _problem((n,), 700 + n)
    if bc == "msd":
        psi = psi + 2.5
    h, a, s = 0.5, 0.8, -1.0
    prob = oracle.Problem((n,), h, a, s, bc=oracle.BC_MSD if bc == "msd" else 0)
    _, _, dtmax = oracle.invariants(prob, rounded(psi, prec), rounded(V, prec))
    solver = nlse.Solver(to_dev(V, prec), h, 0.5 * dtmax, a, s, bc=bc, prec=prec)
    outs = []
    for cluster in (0, 1, 2, 4, 8, 16):
        solver.set_tiling(nlse.TILE_1D_RESIDENT, cluster)
        assert solver.get_tiling(nlse.TILE_1D_RESIDENT) == cluster
        x = to_dev(psi, prec)
        solver.run(x, 37)
        solver.rk4_step(x)
        outs.append(x)
    for x in outs[1:]:
        assert torch.equal(x, outs[0])
    solver.check()
    for bad in (3, 32, -1):
        with pytest.raises(nlse.NLSEError):
            solver.set_tiling(nlse.TILE_1D_RESIDENT, bad)


@pytest.mark.parametrize("shape,prec", [((67, 200), "fp32"), ((35, 18, 40), "fp64"), ((1030,), "fp32")])
def test_run_host_equals_a_device_run(shape, prec):
    """nlse_run_host on a pinned host state gives the bits of nlse_run on the
    same state in device memory (fresh compensated part in both)."""
    psi, V = _problem(shape, 57)
    h, a, s = 0.5, 0.9, -1.0
    prob = oracle.Problem(shape, h, a, s)
    _, _, dtmax = oracle.invariants(prob, rounded(psi, prec), rounded(V, prec))
    solver = nlse.Solver(to_dev(V, prec), h, 0.5 * dtmax, a, s, prec=prec)
    x = to_dev(psi, prec)
    solver.run(x, 40)
    host = to_dev(psi, prec).cpu().pin_memory()
    solver.run_host(host, 40)
    assert torch.equal(host, x.cpu())
    solver.run_host(host, 0)
    assert torch.equal(host, x.cpu())
    with pytest.raises(ValueError):
        solver.run_host(x, 1)                       # a device tensor is not a host state


@pytest.mark.parametrize("shape,prec,stack", [((300, 516), "fp32", 0), ((300, 516), "fp64", 0),
                                              ((2048, 260), "fp32", 0), ((64, 128), "fp32", 5)])
@pytest.mark.parametrize("check", [False, True])
def test_run_host_tall_grids_and_stacks_equal_a_device_run(shape, prec, stack, check):
    """nlse_run_host on taller 2D grids and on a stack, with and without the
    entry check: 1, 2 and 33 steps give the bits of nlse_run on the device."""
    _, V = _problem(shape, 1800)
    n = max(stack, 1)
    psis = [_problem(shape, 1810 + i)[0] for i in range(n)]
    h, a, s = 0.5, 0.9, -1.0
    prob = oracle.Problem(shape, h, a, s)
    dt = 0.5 * min(oracle.invariants(prob, rounded(p, prec), rounded(V, prec))[2] for p in psis)
    psi = np.stack(psis) if stack else psis[0]
    solver = nlse.Solver(to_dev(V, prec), h, dt, a, s, prec=prec, stack=stack, check_stability=check)
    for steps in (1, 2, 33):
        x = to_dev(psi, prec)
        solver.run(x, steps)
        host = to_dev(psi, prec).cpu().pin_memory()
        solver.run_host(host, steps)
        assert torch.equal(host, x.cpu()), steps
    solver.check()


# -- stacks of equal-shape instances sharing V (NLSE_FLAG_STACK) ---------------

@pytest.mark.parametrize("shape,prec,lap", [((70, 128), "fp32", "2shoc"), ((70, 128), "fp64", "2shoc"),
                                            ((40, 131), "fp32", "cd"), ((45, 260), "fp32", "2shoc_ms"),
                                            ((17, 68), "fp64", "2shoc_ms")])
def test_stack_equals_single_grid_runs(shape, prec, lap):
    """Each instance of a stack advances exactly as it would alone (same bits),
    and the stack's Laplacian is the instances' Laplacians."""
    n = 5
    _, V = _problem(shape, 900)
    psis = [_problem(shape, 910 + i)[0] for i in range(n)]
    h, a, s = 0.5, 0.9, -1.0
    prob = oracle.Problem(shape, h, a, s)
    dt = 0.5 * min(oracle.invariants(prob, rounded(p, prec), rounded(V, prec))[2] for p in psis)
    Vd = to_dev(V, prec)
    st = nlse.Solver(Vd, h, dt, a, s, prec=prec, lap=lap, stack=n)
    xs = torch.stack([to_dev(p, prec) for p in psis]).contiguous()
    lap_stack = st.lap2shoc(xs)
    st.run(xs, 37)
    st.check()
    one = nlse.Solver(Vd, h, dt, a, s, prec=prec, lap=lap)
    for i, p in enumerate(psis):
        x = to_dev(p, prec)
        assert torch.equal(one.lap2shoc(x), lap_stack[i]), i
        one.run(x, 37)
        assert torch.equal(x, xs[i]), i


def test_stack_invariants_are_the_instances_totals():
    shape, n = (70, 128), 4
    _, V = _problem(shape, 930)
    psis = [_problem(shape, 931 + i)[0] for i in range(n)]
    h, a, s = 0.5, 0.9, -1.0
    st = nlse.Solver(to_dev(V, "fp64"), h, 1e-4, a, s, prec="fp64", stack=n)
    m, e, d = st.invariants(torch.stack([to_dev(p, "fp64") for p in psis]).contiguous())
    one = nlse.Solver(to_dev(V, "fp64"), h, 1e-4, a, s, prec="fp64")
    parts = [one.invariants(to_dev(p, "fp64")) for p in psis]
    assert m == pytest.approx(sum(q[0] for q in parts), rel=1e-13)
    assert e == pytest.approx(sum(q[1] for q in parts), rel=1e-12)
    assert d == min(q[2] for q in parts)


# -- temporal blocking: two RK4 stages per launch (NLSE_TILE_2D_FUSE) ------------

FUSE_SHAPES = [(3, 4), (17, 68), (70, 128), (100, 388), (45, 260), (9, 1024), (301, 516)]


@pytest.mark.parametrize("shape", FUSE_SHAPES)
@pytest.mark.parametrize("lap", ["2shoc", "cd"])
def test_two_stages_per_launch_equal_four_launches(shape, lap):
    """Stages 1+2 and 3+4 in one launch each give the bits of the four
    single-stage launches: ragged CTA tails in x and y, grids narrower than
    one CTA and than the extra rows of the first stage of a pair, steps
    through nlse_run (graph) and nlse_rk4_step."""
    psi, V = _problem(shape, 1200 + shape[1])
    h, a, s = 0.5, 0.9, -1.0
    prob = oracle.Problem(shape, h, a, s)
    _, _, dtmax = oracle.invariants(prob, rounded(psi, "fp32"), rounded(V, "fp32"))
    solver = nlse.Solver(to_dev(V, "fp32"), h, 0.5 * dtmax, a, s, prec="fp32", lap=lap)
    outs = []
    for fuse in (0, 1):
        solver.set_tiling(nlse.TILE_2D_FUSE, fuse)
        assert solver.get_tiling(nlse.TILE_2D_FUSE) == fuse
        x = to_dev(psi, "fp32")
        solver.run(x, 37)
        solver.rk4_step(x)
        solver.check()
        outs.append(x)
    assert torch.equal(outs[1], outs[0])


def test_two_stages_per_launch_match_oracle():
    """The fused path against the oracle directly (10 steps, FP32 tolerance)."""
    shape = (100, 388)
    psi, V = _problem(shape, 1300)
    h, a, s = 0.5, 0.9, -1.0
    prob = oracle.Problem(shape, h, a, s)
    psi_r, V_r = rounded(psi, "fp32"), rounded(V, "fp32")
    _, _, dtmax = oracle.invariants(prob, psi_r, V_r)
    k = 0.5 * dtmax
    solver = nlse.Solver(to_dev(V, "fp32"), h, k, a, s, prec="fp32")
    solver.set_tiling(nlse.TILE_2D_FUSE, 1)
    x = to_dev(psi, "fp32")
    solver.run(x, 10)
    ref = oracle.run(prob, psi_r, V_r, k, 10)
    got = x.cpu().numpy().astype(np.complex128)
    assert rel_l2(got, ref) < 1e-5
    assert np.abs(got - ref).max() < 1e-5 * np.abs(ref).max()


@pytest.mark.parametrize("shape,lap", [((17, 68), "2shoc"), ((45, 260), "cd"), ((70, 128), "2shoc")])
def test_stack_two_stages_per_launch(shape, lap):
    """A stack on the fused path: every instance equals its own single-grid run
    on the four-launch path, the stage pairs crossing instance boundaries
    inside a CTA's rows."""
    n = 5
    _, V = _problem(shape, 1400)
    psis = [_problem(shape, 1410 + i)[0] for i in range(n)]
    h, a, s = 0.5, 0.9, -1.0
    prob = oracle.Problem(shape, h, a, s)
    dt = 0.5 * min(oracle.invariants(prob, rounded(p, "fp32"), rounded(V, "fp32"))[2] for p in psis)
    Vd = to_dev(V, "fp32")
    st = nlse.Solver(Vd, h, dt, a, s, prec="fp32", lap=lap, stack=n)
    st.set_tiling(nlse.TILE_2D_FUSE, 1)
    xs = torch.stack([to_dev(p, "fp32") for p in psis]).contiguous()
    st.run(xs, 37)
    st.check()
    one = nlse.Solver(Vd, h, dt, a, s, prec="fp32", lap=lap)
    for i, p in enumerate(psis):
        x = to_dev(p, "fp32")
        one.run(x, 37)
        assert torch.equal(x, xs[i]), i


def test_two_stages_per_launch_key_validation():
    """Values other than 0 and 1 are refused; contexts the fused kernels do not
    cover (FP64, multi storage) accept the key and keep their results."""
    shape = (45, 260)
    psi, V = _problem(shape, 1500)
    for prec, lap in (("fp64", "2shoc"), ("fp32", "2shoc_ms")):
        solver = nlse.Solver(to_dev(V, prec), 0.5, 1e-4, 0.9, -1.0, prec=prec, lap=lap)
        outs = []
        for fuse in (0, 1):
            solver.set_tiling(nlse.TILE_2D_FUSE, fuse)
            x = to_dev(psi, prec)
            solver.run(x, 5)
            outs.append(x)
        assert torch.equal(outs[0], outs[1])
        for bad in (2, -1):
            with pytest.raises(nlse.NLSEError):
                solver.set_tiling(nlse.TILE_2D_FUSE, bad)


# -- degenerate cases of the method ----------------------------------------------

@pytest.mark.parametrize("shape", [(1030,), (45, 260), (40, 131), (9, 20, 37), (70, 40, 100)])
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_linear_free_equation_matches_oracle(shape, prec):
    """s = 0 and V = 0: the free linear Schroedinger equation, where F is a
    times the Laplacian alone; 12 steps against the oracle."""
    psi = wl.random_field(shape, seed=1600)
    V = np.zeros(shape)
    h, a, s = 0.5, 0.7, 0.0
    prob = oracle.Problem(shape, h, a, s)
    psi_r = rounded(psi, prec)
    _, _, dtmax = oracle.invariants(prob, psi_r, V)
    k = 0.5 * dtmax
    solver = nlse.Solver(to_dev(V, prec), h, k, a, s, prec=prec)
    x = to_dev(psi, prec)
    solver.run(x, 12)
    ref = oracle.run(prob, psi_r, V, k, 12)
    got = x.cpu().numpy().astype(np.complex128)
    tol = 1e-12 if prec == "fp64" else 1e-5
    assert rel_l2(got, ref) < tol


@pytest.mark.parametrize("shape", [(1030,), (45, 260), (70, 40, 100)])
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_zero_state_stays_zero(shape, prec):
    """Psi = 0 is a fixed point of Eq. (NLSE) for any V: every step returns
    exact zeros (no rounding can create a value from nothing)."""
    V = wl.random_potential(shape, seed=1700, scale=2.0)
    solver = nlse.Solver(to_dev(V, prec), 0.5, 1e-3, 0.9, -1.0, prec=prec)
    x = to_dev(np.zeros(shape, complex), prec)
    solver.run(x, 33)
    solver.check()
    assert not torch.any(x != 0)


@pytest.mark.parametrize("shape", [(45, 260), (70, 40, 100)])
def test_constant_state_turns_at_the_nonlinear_frequency(shape):
    """A constant field with V = 0 has Lap = 0 at interior points, so each
    interior point follows the scalar ODE dPsi/dt = i s |Psi|^2 Psi, stepped
    here by the textbook scalar RK4 (not the linear R(i k s |c|^2) c: |Y|^2
    changes between the stages); the Dirichlet boundary holds c.  The boundary's D_b reaches distance 1 in stage 1 and the radius-2
    stencil carries it 2 points further per stage, so after one step the
    points at distance >= 8 follow the scalar step (FP64)."""
    c = 0.8 - 0.6j
    psi = np.full(shape, c)
    V = np.zeros(shape)
    h, a, s, k = 0.5, 0.9, -1.0, 0.01
    solver = nlse.Solver(to_dev(V, "fp64"), h, k, a, s, prec="fp64")
    x = to_dev(psi, "fp64")
    solver.rk4_step(x)
    f = lambda y: 1j * s * abs(y) ** 2 * y
    k1 = f(c)
    k2 = f(c + k / 2 * k1)
    k3 = f(c + k / 2 * k2)
    k4 = f(c + k * k3)
    expect = c + k / 6 * (k1 + 2 * k2 + 2 * k3 + k4)
    got = x.cpu().numpy()
    inner = got[tuple(slice(8, n - 8) for n in shape)]
    assert np.abs(inner - expect).max() < 1e-14
    edge = got[(0,) * len(shape)]
    assert edge == c
