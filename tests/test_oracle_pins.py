"""Pins of the CPU oracle against what arXiv 1109.1027 and the mathematics fix.

None of these tests compare the oracle with itself.  Each checks it against an
independent fact: the non-compact stencils the paper says 2SHOC equals, exact
polynomial and plane-wave results, exact stationary and travelling solutions,
the textbook RK4 stability polynomial, the paper's closed-form stability
bound, and the error tables the paper prints (tests/golden/paper_tables.txt).
"""
import os

import numpy as np
import pytest

import oracle
import paper_experiments as pe
from paper_1109_1027_gb300 import workloads as wl

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_tables.txt")


def noncompact_lap(psi, h):
    """Standard non-compact fourth-order Laplacian: the 1D five-point stencil
    (Sec. 2.1) summed over axes (the 13-point 2D stencil, Eq. (2dnonhoc), and
    its 3D analogue, Sec. 2.3); valid at points >= 2 from the boundary."""
    d = psi.ndim
    core = tuple(slice(2, -2) for _ in range(d))
    out = np.zeros(psi[core].shape, dtype=psi.dtype)
    for ax in range(d):
        def sh(o):
            sl = [slice(2, -2)] * d
            n = psi.shape[ax]
            sl[ax] = slice(2 + o, n - 2 + o)
            return psi[tuple(sl)]
        out += (-sh(2) + 16 * sh(1) - 30 * sh(0) + 16 * sh(-1) - sh(-2)) / (12 * h * h)
    return out


SHAPES = [(41,), (13, 17), (9, 10, 11)]


@pytest.mark.parametrize("shape", SHAPES)
def test_interior_equals_noncompact_stencil(shape):
    """Secs. 2.1-2.3: 2SHOC (single storage) is algebraically the non-compact
    fourth-order stencil at interior points."""
    h = 0.37
    psi = wl.random_field(shape, seed=11)
    V = wl.random_potential(shape, seed=12)
    prob = oracle.Problem(shape, h, 0.8, -1.3)
    lap = oracle.laplacian(prob, psi, V)
    core = tuple(slice(2, -2) for _ in shape)
    ref = noncompact_lap(psi, h)
    scale = np.abs(psi).max() * 64 / 12 * len(shape) / h ** 2
    assert np.abs(lap[core] - ref).max() <= 1e-13 * scale


@pytest.mark.parametrize("shape", SHAPES[1:])
def test_multi_storage_interior_equals_noncompact_stencil(shape):
    """Eqs. (2d2shocMs1-2) and (3d2shocMs1-2): the multi-storage 2SHOC is the
    1D fourth-order stencil along each axis, i.e. the non-compact stencil."""
    h = 0.37
    psi = wl.random_field(shape, seed=13)
    V = wl.random_potential(shape, seed=14)
    prob = oracle.Problem(shape, h, 0.8, -1.3, lap=oracle.LAP_2SHOC_MS)
    lap = oracle.laplacian(prob, psi, V)
    core = tuple(slice(2, -2) for _ in shape)
    scale = np.abs(psi).max() * 64 / 12 * len(shape) / h ** 2
    assert np.abs(lap[core] - noncompact_lap(psi, h)).max() <= 1e-13 * scale


@pytest.mark.parametrize("shape", [(9, 11), (17, 6), (6, 7, 8), (9, 5, 7)])
def test_multi_storage_boundary_split_matches_single_storage(shape):
    """With D^a_b = D_b(Eq. dbc_lap) - (the other axes' second differences) at a
    point on the boundary of axis a only, the two storage forms are the same
    operator at every point, including the ring next to the boundary (where
    the single-storage form reads D_b directly); boundary points carry D_b in
    both.  A wrong split (e.g. one axis left out in 3D) breaks the ring."""
    h = 0.41
    psi = wl.random_field(shape, seed=15) + 0.7
    V = wl.random_potential(shape, seed=16, scale=2.0)
    single = oracle.laplacian(oracle.Problem(shape, h, 0.6, 1.1), psi, V)
    multi = oracle.laplacian(oracle.Problem(shape, h, 0.6, 1.1, lap=oracle.LAP_2SHOC_MS), psi, V)
    scale = np.abs(psi).max() * 64 / 12 * len(shape) / h ** 2
    assert np.abs(multi - single).max() <= 1e-13 * scale
    ring = np.zeros(shape, bool)
    ring[tuple(slice(1, -1) for _ in shape)] = True
    ring[tuple(slice(2, -2) for _ in shape)] = False
    assert np.abs(single[ring]).max() > 1e-3 * scale          # the ring is exercised


def test_multi_storage_is_single_storage_in_1d_and_rejects_msd_in_2d():
    shape = (37,)
    psi = wl.random_field(shape, seed=17) + 2.0
    V = wl.random_potential(shape, seed=18)
    for bc in (oracle.BC_DIRICHLET, oracle.BC_MSD):
        a = oracle.run(oracle.Problem(shape, 0.3, 0.9, -1.0, bc=bc), psi, V, 1e-3, 5)
        b = oracle.run(oracle.Problem(shape, 0.3, 0.9, -1.0, bc=bc, lap=oracle.LAP_2SHOC_MS), psi, V, 1e-3, 5)
        assert np.array_equal(a, b)
    with pytest.raises(ValueError):
        oracle.laplacian(oracle.Problem((6, 6), 0.3, 0.9, -1.0, bc=oracle.BC_MSD, lap=oracle.LAP_2SHOC_MS),
                         np.ones((6, 6), complex), np.zeros((6, 6)))


PERIODIC = [((24,), 3), ((12, 10), 2), ((8, 6, 10), 2)]


@pytest.mark.parametrize("shape,modes", PERIODIC)
@pytest.mark.parametrize("lap", [oracle.LAP_2SHOC, oracle.LAP_2SHOC_MS])
def test_periodic_plane_wave_is_an_exact_eigenfunction(shape, modes, lap):
    """On a periodic grid (n points, spacing h = L/n, wrapping indices) every
    point is interior and a plane wave exp(i sum_a theta_a j_a) is an exact
    eigenfunction of 2SHOC with the closed-form symbol
    sum_a (-2 cos 2theta_a + 32 cos theta_a - 30) / (12 h^2)."""
    h = 0.3
    idx = np.meshgrid(*[np.arange(n) for n in shape], indexing="ij")
    thetas = [2 * np.pi * (modes + a) / n for a, n in enumerate(shape)]
    phase = sum(t * j for t, j in zip(thetas, idx))
    psi = 1.7 * np.exp(1j * phase)
    lam = sum(symbol(t) for t in thetas) / h ** 2
    prob = oracle.Problem(shape, h, 1.0, 0.0, bc=oracle.BC_PERIODIC, lap=lap)
    lap_f = oracle.laplacian(prob, psi, np.zeros(shape))
    assert np.abs(lap_f - lam * psi).max() <= 1e-12 * abs(lam) * 1.7


@pytest.mark.parametrize("shape,modes", PERIODIC)
def test_periodic_nonlinear_plane_wave_follows_the_scalar_rk4(shape, modes):
    """With V constant a plane wave stays a plane wave; its amplitude then obeys
    y' = i (a lam + s|y|^2 - V) y exactly, stepped by a textbook scalar RK4."""
    h, a, s, V0, k = 0.3, 0.8, -1.2, 0.4, 2e-3
    idx = np.meshgrid(*[np.arange(n) for n in shape], indexing="ij")
    thetas = [2 * np.pi * (modes + a_) / n for a_, n in enumerate(shape)]
    wave = np.exp(1j * sum(t * j for t, j in zip(thetas, idx)))
    lam = sum(symbol(t) for t in thetas) / h ** 2
    y0 = 0.9 + 0.3j
    prob = oracle.Problem(shape, h, a, s, bc=oracle.BC_PERIODIC)
    out = oracle.run(prob, y0 * wave, np.full(shape, V0), k, 7)
    y = scalar_rk4(y0, lambda v: 1j * (a * lam + s * abs(v) ** 2 - V0) * v, k, 7)
    assert np.abs(out - y * wave).max() <= 1e-12


@pytest.mark.parametrize("dim", [1, 2, 3])
def test_laplacian_zero_boundary_on_a_harmonic_field(dim):
    """Laplacian-zero: on a harmonic polynomial (degree 2, where 2SHOC is exact)
    the Laplacian vanishes everywhere, interior by exactness and boundary by
    the rule.  With s = 0 and a constant V every point then turns by the same
    factor, y' = -i V y, which keeps the field harmonic: one step is exactly
    the RK4 polynomial R(-i k V) at every point, boundary included (Dirichlet
    would hold the boundary still)."""
    n = {1: 13, 2: 9, 3: 7}[dim]
    shape = (n,) * dim
    coords = wl.mesh(shape, -1.0, 1.0)
    h = wl.spacing(n, -1.0, 1.0)
    if dim == 1:
        psi = (0.5 + 0.3 * coords[0]) + 1j * (0.2 - 0.4 * coords[0])
    elif dim == 2:
        x, y = coords
        psi = (x * x - y * y + 1.0) + 1j * (x * y + 0.5)
    else:
        x, y, z = coords
        psi = (x * x - z * z + 1.0) + 1j * (x * y + y * z + 0.5)
    V0, a, k = 0.7, 0.9, 1e-2
    V = np.full(shape, V0)
    prob = oracle.Problem(shape, h, a, 0.0, bc=oracle.BC_LAPZERO)
    assert np.abs(oracle.laplacian(prob, psi, V)).max() <= 1e-11 / h ** 2
    out = oracle.run(prob, psi, V, k, 5)
    assert np.abs(out - stability_poly(-1j * k * V0) ** 5 * psi).max() <= 1e-12
    dirichlet = oracle.run(oracle.Problem(shape, h, a, 0.0), psi, V, k, 5)
    assert np.abs(out[(0,) * dim] - dirichlet[(0,) * dim]) > 1e-3


@pytest.mark.parametrize("dim", [1, 2, 3])
def test_laplacian_zero_nonlinear_constant_state(dim):
    """A constant state has zero Laplacian everywhere under the
    Laplacian-zero rule; every point, boundary included, then follows
    y' = i (s|y|^2 - V) y, stepped exactly by the scalar RK4."""
    shape = ({1: 11, 2: 7, 3: 5}[dim],) * dim
    y0, s, V0, k = 0.8 - 0.6j, 1.4, 0.3, 5e-3
    prob = oracle.Problem(shape, 0.2, 0.9, s, bc=oracle.BC_LAPZERO)
    out = oracle.run(prob, np.full(shape, y0), np.full(shape, V0), k, 6)
    y = scalar_rk4(y0, lambda v: 1j * (s * abs(v) ** 2 - V0) * v, k, 6)
    assert np.abs(out - y).max() <= 1e-13


@pytest.mark.parametrize("dim", [1, 2, 3])
def test_polynomial_exactness(dim):
    """The fourth-order stencil's error term is h^4 times sixth derivatives, so
    2SHOC is exact (to rounding) on polynomials of degree <= 5 in each variable."""
    rng = np.random.Generator(np.random.PCG64(5))
    n = {1: 15, 2: 11, 3: 9}[dim]
    shape = (n,) * dim
    coords = wl.mesh(shape, -1.0, 1.3)
    h = wl.spacing(n, -1.0, 1.3)
    P = np.polynomial.polynomial
    # separable sum of products: f = sum_t prod_ax p_{t,ax}(x_ax), complex coefficients
    f = np.zeros(shape, complex)
    lap_exact = np.zeros(shape, complex)
    for _ in range(3):
        cs = [rng.standard_normal(6) + 1j * rng.standard_normal(6) for _ in range(dim)]
        vals = [P.polyval(coords[ax], cs[ax]) for ax in range(dim)]
        dd = [P.polyval(coords[ax], P.polyder(cs[ax], 2)) for ax in range(dim)]
        f += np.prod(vals, axis=0)
        for ax in range(dim):
            lap_exact += np.prod([dd[b] if b == ax else vals[b] for b in range(dim)], axis=0)
    prob = oracle.Problem(shape, h, 1.0, 0.0)
    lap = oracle.laplacian(prob, f, np.zeros(shape))
    core = tuple(slice(2, -2) for _ in shape)
    assert np.abs(lap[core] - lap_exact[core]).max() <= 1e-9 * np.abs(lap_exact).max()


def symbol(theta):
    """h^2 x eigenvalue of the fourth-order stencil on exp(i theta j) per axis."""
    return (-2 * np.cos(2 * theta) + 32 * np.cos(theta) - 30) / 12


@pytest.mark.parametrize("dim", [1, 2, 3])
def test_plane_wave_symbol_and_msd_boundary(dim):
    """A constant-modulus plane wave is an exact discrete eigenfunction: the
    interior 2SHOC gives the closed-form symbol, and the MSD rule of
    Eq. (msdbc_lap) returns exactly the second difference at the boundary, so
    with MSD the symbol holds at every point up to the boundary."""
    n = {1: 21, 2: 12, 3: 8}[dim]
    shape = (n,) * dim
    h = 0.3
    kv = [0.7, -1.1, 0.4][:dim]
    coords = wl.mesh(shape, 0.0, h * (n - 1))
    psi = 0.8 * np.exp(1j * sum(k * c for k, c in zip(kv, coords)))
    lam4 = sum(symbol(k * h) for k in kv) / h ** 2
    lam2 = sum(2 * np.cos(k * h) - 2 for k in kv) / h ** 2
    V = np.zeros(shape)
    # Dirichlet: interior points >= 2 from the boundary
    lap = oracle.laplacian(oracle.Problem(shape, h, 1.0, 0.5), psi, V)
    core = tuple(slice(2, -2) for _ in shape)
    assert np.allclose(lap[core], lam4 * psi[core], rtol=0, atol=1e-12 * abs(lam4))
    # MSD: every interior point, and D_b = second difference at the boundary
    lap, D = oracle.laplacian(oracle.Problem(shape, h, 1.0, 0.5, bc=oracle.BC_MSD), psi, V,
                              return_D=True)
    inner = tuple(slice(1, -1) for _ in shape)
    assert np.allclose(lap[inner], lam4 * psi[inner], rtol=0, atol=1e-12 * abs(lam4))
    assert np.allclose(D, lam2 * psi, rtol=0, atol=1e-12 * abs(lam2))


def test_fourth_order_convergence_on_analytic_field():
    """O(h^4) at interior points on exp(-r^2) exp(i k x) (Sec. 2.2)."""
    errs = []
    for n in (41, 81, 161):
        shape = (n, n)
        x, y = wl.mesh(shape, -3.0, 3.0)
        h = wl.spacing(n, -3.0, 3.0)
        g = np.exp(-(x * x + y * y)) * np.exp(1.5j * x)
        # exact Laplacian of g
        ex = g * ((-2 * x + 1.5j) ** 2 - 2 + 4 * y * y - 2)
        lap = oracle.laplacian(oracle.Problem(shape, h, 1.0, 0.0), g, np.zeros(shape))
        core = (slice(2, -2), slice(2, -2))
        errs.append(np.abs(lap[core] - ex[core]).max())
    orders = [np.log2(errs[i] / errs[i + 1]) for i in range(2)]
    assert all(3.8 < o < 4.2 for o in orders), orders


def stationary_sech(x):
    """psi = sqrt(2) sech x solves psi'' - V psi + |psi|^2 psi = 0 for V = 1
    (a = s = 1): a time-independent solution of Eq. (NLSE)."""
    return np.sqrt(2.0) / np.cosh(x)


def test_dirichlet_boundary_laplacian_is_exact_on_stationary_state():
    """Eq. (dbc_lap) sets psi_t = 0 at the boundary; on a stationary state it
    returns the exact second derivative there."""
    n = 61
    x = wl.axis(n, -3.0, 3.0)
    h = wl.spacing(n, -3.0, 3.0)
    psi = stationary_sech(x).astype(complex)
    d2 = np.sqrt(2.0) * (1 / np.cosh(x) - 2 / np.cosh(x) ** 3)
    lap = oracle.laplacian(oracle.Problem((n,), h, 1.0, 1.0), psi, np.ones(n))
    assert abs(lap[0] - d2[0]) < 1e-14 and abs(lap[-1] - d2[-1]) < 1e-14


@pytest.mark.parametrize("dim", [1, 2, 3])
def test_dirichlet_boundary_value_on_a_stationary_state_with_general_a(dim):
    """Eq. (dbc_lap) for any a: with V = s|psi|^2 + a Lap(psi)/psi, the smooth
    real field psi = 1 + exp(-r^2) is a stationary state (psi_t = 0
    everywhere), so D_b = -(s|psi_b|^2 - V_b) psi_b / a must be the analytic
    Laplacian at every boundary point; a = 0.6, s = -1.3 (a D_b missing its 1/a,
    or with the sign of N reversed, is off by a visible factor)."""
    n = {1: 21, 2: 13, 3: 9}[dim]
    shape = (n,) * dim
    coords = wl.mesh(shape, -1.5, 1.5)
    h = wl.spacing(n, -1.5, 1.5)
    a, s = 0.6, -1.3
    r2 = sum(c * c for c in coords)
    g = np.exp(-r2)
    psi = 1.0 + g
    lap_exact = g * (4.0 * r2 - 2.0 * dim)
    V = s * psi ** 2 + a * lap_exact / psi
    lap = oracle.laplacian(oracle.Problem(shape, h, a, s), psi.astype(complex), V)
    bnd = np.zeros(shape, bool)
    for ax in range(dim):
        sl = [slice(None)] * dim
        sl[ax] = 0
        bnd[tuple(sl)] = True
        sl[ax] = -1
        bnd[tuple(sl)] = True
    assert np.abs(lap[bnd] - lap_exact[bnd]).max() <= 1e-13 * np.abs(lap_exact).max()
    assert np.abs(oracle.rhs(oracle.Problem(shape, h, a, s), psi.astype(complex), V)[bnd]).max() == 0.0


def test_stationary_state_is_kept_to_fourth_order():
    """RK4+2SHOC with Dirichlet holds the stationary sech state; the error
    falls ~16x per halving of h, and boundary values never move."""
    errs = []
    for n in (41, 81):
        x = wl.axis(n, -5.0, 5.0)
        h = wl.spacing(n, -5.0, 5.0)
        psi0 = stationary_sech(x).astype(complex)
        prob = oracle.Problem((n,), h, 1.0, 1.0)
        k = 0.2 * h * h
        out = oracle.run(prob, psi0, np.ones(n), k, int(round(1.0 / k)))
        assert out[0] == psi0[0] and out[-1] == psi0[-1]
        errs.append(np.abs(out - psi0).max())
    assert 3.7 < np.log2(errs[0] / errs[1]) < 4.3, errs


def stability_poly(z):
    return 1 + z + z * z / 2 + z ** 3 / 6 + z ** 4 / 24


@pytest.mark.parametrize("dim", [1, 2])
def test_rk4_step_is_stability_polynomial_on_linear_problem(dim):
    """For s = 0 the semi-discrete system is linear, psi_t = A psi, and one
    classic RK4 step is exactly R(kA) psi, R(z) = 1 + z + z^2/2 + z^3/6 + z^4/24."""
    shape = (9,) if dim == 1 else (5, 6)
    h, k, a = 0.5, 0.03, 0.7
    V = wl.random_potential(shape, seed=3)
    prob = oracle.Problem(shape, h, a, 0.0)
    N = int(np.prod(shape))
    A = np.zeros((N, N), complex)
    for j in range(N):
        e = np.zeros(N, complex)
        e[j] = 1.0
        A[:, j] = oracle.rhs(prob, e.reshape(shape), V).ravel()
    # F is C-linear when s = 0: check that before using A
    psi = wl.random_field(shape, seed=4)
    assert np.allclose(A @ psi.ravel(), oracle.rhs(prob, psi, V).ravel(), atol=1e-12)
    kA = k * A
    R = np.eye(N) + kA + kA @ kA / 2 + kA @ kA @ kA / 6 + kA @ kA @ kA @ kA / 24
    out = oracle.run(prob, psi, V, k, 1)
    assert np.allclose(out.ravel(), R @ psi.ravel(), rtol=0, atol=1e-13)


def scalar_rk4(y, f, k, n):
    """Classic RK4 in its textbook k1..k4 form."""
    for _ in range(n):
        k1 = f(y)
        k2 = f(y + 0.5 * k * k1)
        k3 = f(y + 0.5 * k * k2)
        k4 = f(y + k * k3)
        y = y + k / 6 * (k1 + 2 * k2 + 2 * k3 + k4)
    return y


@pytest.mark.parametrize("dim", [1, 2, 3])
def test_msd_plane_wave_nonlinear_rk4(dim):
    """Under MSD a plane wave stays a plane wave: every point follows the scalar
    ODE y' = i(a lam + s|y|^2 - V) y.  This fixes F (Sec. 3.1), the MSD rules
    Eqs. (msdbc_ut), (msdbc_lap), and the RK4 schedule of Eq. (RK4) against an
    independent textbook RK4."""
    n = {1: 16, 2: 9, 3: 7}[dim]
    shape = (n,) * dim
    h, a, s, V0, k = 0.4, 0.6, -1.7, 0.3, 0.004
    kv = [0.9, -0.5, 1.3][:dim]
    coords = wl.mesh(shape, 0.0, h * (n - 1))
    amp = 0.9 * np.exp(0.3j)
    psi = amp * np.exp(1j * sum(kk * c for kk, c in zip(kv, coords)))
    lam = sum(symbol(kk * h) for kk in kv) / h ** 2
    prob = oracle.Problem(shape, h, a, s, bc=oracle.BC_MSD)
    out = oracle.run(prob, psi, np.full(shape, V0), k, 25)
    y = scalar_rk4(amp, lambda y: 1j * (a * lam + s * abs(y) ** 2 - V0) * y, k, 25)
    expect = y * np.exp(1j * sum(kk * c for kk, c in zip(kv, coords)))
    assert np.abs(out - expect).max() < 1e-12


@pytest.mark.parametrize("dim", [1, 2, 3])
def test_linear_stability_bound(dim):
    """Eq. (kdfull) with s = 0, V = 0 reduces to Eq. (kd2shoclin):
    k < (3/4) h^2 / (d sqrt(2) a)."""
    n = 7
    shape = (n,) * dim
    h, a = 0.3, 0.8
    _, _, dt = oracle.invariants(oracle.Problem(shape, h, a, 0.0), np.ones(shape, complex),
                                 np.zeros(shape))
    assert dt == pytest.approx(0.75 * h * h / (dim * np.sqrt(2) * a), rel=1e-14)


def test_stability_bound_is_sharp():
    """RK4 is stable at 0.9x the bound and blows up at 1.2x (Sec. 3.3): the
    bound sits at the RK4 imaginary-axis limit sqrt(8) of the scheme's spectrum."""
    n, h, a = 64, 0.25, 1.0
    prob = oracle.Problem((n,), h, a, 0.0)
    V = np.zeros(n)
    psi = wl.random_field((n,), seed=9) * 1e-3
    psi[0] = psi[-1] = 0
    _, _, dt = oracle.invariants(prob, psi, V)
    m0 = np.sum(np.abs(psi) ** 2)
    ok = oracle.run(prob, psi, V, 0.9 * dt, 400)
    bad = oracle.run(prob, psi, V, 1.2 * dt, 60)
    assert np.sum(np.abs(ok) ** 2) <= m0
    assert np.sum(np.abs(bad) ** 2) > 1e3 * m0


@pytest.mark.parametrize("name,h,k", [("E1", 1 / 32, 0.0005), ("E2", 1 / 16, 0.001)])
def test_paper_time_steps_sit_just_under_the_bound(name, h, k):
    """Sec. 4.1: k = 0.0005 is 'slightly less' than the bound at h = 1/32;
    Sec. 4.2's k = 0.001 is likewise just inside at h = 1/16."""
    st = pe.setup(name, h)
    prob = oracle.Problem(st["shape"], h, st["a"], st["s"], st["bc"])
    _, _, dt = oracle.invariants(prob, st["psi0"], st["V"])
    assert k < dt < 1.1 * k


def test_mass_and_energy_of_bright_soliton():
    """Mass and energy (this project's definitions; the paper defines none)
    converge to the continuum values of sqrt(2) sech(x) exp(icx):
    M = 4, E = int |psi_x|^2 - |psi|^4 / 2 = -4/3 + 4 c^2.  The energy uses
    the fourth-order Laplacian, so its error falls ~16x per halving of h."""
    errs = []
    for n in (1025, 2049):
        inst = wl.bright_soliton_1d(n=n)
        prob = oracle.Problem(inst.shape, inst.h, inst.a, inst.s)
        m, e, _ = oracle.invariants(prob, inst.psi0, inst.V)
        c = inst.meta["c"]
        assert m == pytest.approx(4.0, rel=1e-12)
        errs.append(abs(e - (-4 / 3 + 4 * c * c)))
    assert errs[1] < 1e-6
    assert 3.8 < np.log2(errs[0] / errs[1]) < 4.2, errs


def test_bright_soliton_travels_exactly_to_fourth_order():
    """The travelling sech soliton (Galilean boost of the stationary state)
    is reproduced with error falling ~16x per halving of h."""
    errs = []
    for n in (513, 1025):
        x = wl.axis(n, -25.0, 25.0)
        h = wl.spacing(n, -25.0, 25.0)
        ex = lambda t: pe.bright_soliton(x, t, x0=-5.0, c=0.5)
        prob = oracle.Problem((n,), h, 1.0, 1.0)
        k = 0.4 * h * h
        steps = int(round(0.5 / k))
        out = oracle.run(prob, ex(0.0), np.zeros(n), k, steps)
        errs.append(np.abs(out - ex(steps * k)).max())
    assert 3.7 < np.log2(errs[0] / errs[1]) < 4.3, errs


TABLES = pe.read_tables(GOLDEN)


def _oracle_runner(name, h, lap):
    st = pe.setup(name, h)
    prob = oracle.Problem(st["shape"], h, st["a"], st["s"], st["bc"], lap)
    return lambda p, n: oracle.run(prob, p, st["V"], st["k"], n)


@pytest.mark.parametrize("scheme,lap", [("2SHOC", oracle.LAP_2SHOC), ("CD", oracle.LAP_CD)])
def test_paper_table_2d(scheme, lap):
    """Fig. f:num2d table (Sec. 4.2): the printed errors at h = 1, 1/2, 1/4."""
    for i, h in enumerate(pe.E23_H[:3]):
        er, ei = pe.measure("E2", h, _oracle_runner("E2", h, lap))
        assert er == pytest.approx(TABLES[("E2", scheme, "real")][i], rel=2e-4)
        assert ei == pytest.approx(TABLES[("E2", scheme, "imag")][i], rel=2e-4)


@pytest.mark.parametrize("scheme,lap", [("2SHOC", oracle.LAP_2SHOC), ("CD", oracle.LAP_CD)])
def test_paper_table_1d(scheme, lap):
    """Fig. f:num1d table (Sec. 4.1), MSD boundaries, all five h.  The domain is
    not printed (reading in paper_experiments), so values agree to 1% and the
    printed orders to 0.01."""
    got = [pe.measure("E1", h, _oracle_runner("E1", h, lap)) for h in pe.E1_H]
    for part, j in (("real", 0), ("imag", 1)):
        ref = TABLES[("E1", scheme, part)]
        for i in range(5):
            assert got[i][j] == pytest.approx(ref[i], rel=1e-2)
        for i in range(4):
            o = pe.order(got[i][j], got[i + 1][j], pe.E1_H[i], pe.E1_H[i + 1])
            assert o == pytest.approx(pe.order(ref[i], ref[i + 1], 2, 1), abs=1e-2)


def test_paper_table_3d():
    """Fig. f:num3d table (Sec. 4.3): the printed 2SHOC errors at h = 1, 1/2."""
    for i, h in enumerate(pe.E23_H[:2]):
        er, ei = pe.measure("E3", h, _oracle_runner("E3", h, oracle.LAP_2SHOC))
        assert er == pytest.approx(TABLES[("E3", "2SHOC", "real")][i], rel=2e-4)
        assert ei == pytest.approx(TABLES[("E3", "2SHOC", "imag")][i], rel=2e-4)


def test_oracle_rejects_invalid_problems():
    with pytest.raises(ValueError):
        oracle.laplacian(oracle.Problem((2,), 0.1, 1.0, 0.0), np.zeros(2), np.zeros(2))
    with pytest.raises(ValueError):
        oracle.laplacian(oracle.Problem((5,), 0.1, -1.0, 0.0), np.zeros(5), np.zeros(5))


@pytest.mark.parametrize("dim", [1, 2, 3])
def test_cd_laplacian_symbol_and_order(dim):
    """The second-order CD Laplacian (the paper's comparison scheme, Sec. 4):
    on a periodic plane wave it is the exact eigenvalue sum_a 2(cos theta_a - 1)/h^2;
    it is exact on cubics and not on quartics, where 2SHOC is exact (so a CD
    silently replaced by 2SHOC, or the reverse, fails here)."""
    shape = {1: (24,), 2: (12, 10), 3: (8, 6, 10)}[dim]
    h = 0.3
    idx = np.meshgrid(*[np.arange(n) for n in shape], indexing="ij")
    thetas = [2 * np.pi * (2 + a) / n for a, n in enumerate(shape)]
    psi = 1.3 * np.exp(1j * sum(t * j for t, j in zip(thetas, idx)))
    lam2 = sum(2 * np.cos(t) - 2 for t in thetas) / h ** 2
    prob = oracle.Problem(shape, h, 1.0, 0.0, bc=oracle.BC_PERIODIC, lap=oracle.LAP_CD)
    lap = oracle.laplacian(prob, psi, np.zeros(shape))
    assert np.abs(lap - lam2 * psi).max() <= 1e-12 * abs(lam2) * 1.3

    n = {1: 15, 2: 11, 3: 9}[dim]
    grid = (n,) * dim
    coords = wl.mesh(grid, -1.0, 1.3)
    hh = wl.spacing(n, -1.0, 1.3)
    core = tuple(slice(2, -2) for _ in grid)
    cubic = sum((1.0 + 0.5j) * c ** 3 - 0.7 * c ** 2 for c in coords)
    cubic_lap = sum((6.0 + 3.0j) * c - 1.4 for c in coords)
    cd = oracle.laplacian(oracle.Problem(grid, hh, 1.0, 0.0, lap=oracle.LAP_CD), cubic, np.zeros(grid))
    assert np.abs(cd[core] - cubic_lap[core]).max() <= 1e-9 * np.abs(cubic_lap).max()
    quartic = sum(c ** 4 for c in coords).astype(complex)
    quartic_lap = sum(12 * c ** 2 for c in coords)
    cd = oracle.laplacian(oracle.Problem(grid, hh, 1.0, 0.0, lap=oracle.LAP_CD), quartic, np.zeros(grid))
    shoc = oracle.laplacian(oracle.Problem(grid, hh, 1.0, 0.0), quartic, np.zeros(grid))
    # CD's error on x^4 is h^2 f''''/12 = 2 h^2 per axis; 2SHOC's is zero
    assert np.allclose(cd[core] - quartic_lap[core], 2 * dim * hh ** 2, rtol=1e-9)
    assert np.abs(shoc[core] - quartic_lap[core]).max() <= 1e-9 * np.abs(quartic_lap).max()


_D, _M, _P, _Z = oracle.BC_DIRICHLET, oracle.BC_MSD, oracle.BC_PERIODIC, oracle.BC_LAPZERO
SYM_CASES = [((17,), _D, oracle.LAP_2SHOC), ((17,), _M, oracle.LAP_2SHOC),
             ((9, 9), _D, oracle.LAP_2SHOC), ((9, 9), _D, oracle.LAP_CD), ((9, 9), _D, oracle.LAP_2SHOC_MS),
             ((9, 9), _M, oracle.LAP_2SHOC), ((8, 8), _P, oracle.LAP_2SHOC), ((9, 9), _Z, oracle.LAP_CD),
             ((7, 7, 7), _D, oracle.LAP_2SHOC), ((7, 7, 7), _D, oracle.LAP_2SHOC_MS),
             ((7, 7, 7), _M, oracle.LAP_2SHOC), ((6, 6, 6), _P, oracle.LAP_CD)]


@pytest.mark.parametrize("shape,bc,lap", SYM_CASES)
def test_laplacian_and_steps_commute_with_grid_symmetries(shape, bc, lap):
    """The continuous operator has no preferred direction, and neither has any
    boundary rule of Sec. 3.2: reflecting the grid along an axis, or (on cubic
    grids) exchanging two axes, commutes with the Laplacian, with F and with
    an RK4 step, boundaries included.  A stencil or boundary applied on one
    side only, a swapped extent or a shifted index breaks this."""
    psi = wl.random_field(shape, seed=77) + (1.5 if bc == oracle.BC_MSD else 0.0)
    V = wl.random_potential(shape, seed=78)
    h = 0.4
    prob = oracle.Problem(shape, h, 0.8, -1.0, bc=bc, lap=lap)
    lap0 = oracle.laplacian(prob, psi, V)
    F0 = oracle.rhs(prob, psi, V)
    k = 0.2 * oracle.invariants(prob, psi, V)[2]
    step0 = oracle.run(prob, psi, V, k, 2)
    scale = np.abs(lap0).max()
    maps = [lambda z, ax=ax: np.flip(z, axis=ax) for ax in range(len(shape))]
    if len(shape) > 1:
        maps.append(lambda z: np.swapaxes(z, 0, len(shape) - 1))
    for m in maps:
        ps, Vs = np.ascontiguousarray(m(psi)), np.ascontiguousarray(m(V))
        assert np.abs(oracle.laplacian(prob, ps, Vs) - m(lap0)).max() <= 1e-13 * scale
        assert np.abs(oracle.rhs(prob, ps, Vs) - m(F0)).max() <= 1e-13 * np.abs(F0).max()
        assert np.abs(oracle.run(prob, ps, Vs, k, 2) - m(step0)).max() <= 1e-13 * np.abs(step0).max()
