"""Plain FP64 reference for the gradient of a final-time loss through the
RK4 + 2SHOC integrator (the discrete adjoint), Dirichlet boundaries.

TEST INFRASTRUCTURE ONLY: like the rest of ``oracle/``, it is what the CUDA
adjoint is checked against; only tests, the smoke check and the benchmark's
CPU legs may use it.  The forward states come from the C oracle
(``oracle.run`` / ``oracle.rhs``); the transposed operators below are written
out in numpy, vectorised over the whole grid, from the definitions of F
(Sec. 3.1), the 2SHOC Laplacian (Secs. 2.1-2.3) and the Dirichlet boundary
rule (Eqs. dbc_lap, dbc_ut).

Conventions.  A complex field is treated as the pair (Re, Im) of real
fields; the gradient of a real loss with respect to it is stored as the
complex number dL/dRe + i dL/dIm.  With that convention the transpose of
z -> alpha z + beta conj(z) is w -> conj(alpha) w + beta conj(w), and the
inner product is <u, v> = Re sum conj(u) v.

The semi-discrete right-hand side at an interior point p is
    F_p = i a Lap_p + i (s|Y_p|^2 - V_p) Y_p,      F_b = 0 at boundary points,
with Lap_p = c0 D_p + c1 (sum of the 2d axial D) + c2 (sum of the 2d(d-1)
edge-neighbour Y - 2d(d-1) Y_p), c0 = (16 - 2d)/12, c1 = -1/12,
c2 = 1/(6h^2) (single-storage 2SHOC; for CD: Lap = D), where D_j = delta^2 Y_j
at interior j and D_b = -(s|Y_b|^2 - V_b) Y_b / a at boundary points.
"""
from __future__ import annotations

import itertools

import numpy as np

from . import Problem, LAP_CD, rhs, run


def _interior(shape):
    m = np.ones(shape, bool)
    for ax in range(len(shape)):
        sl = [slice(None)] * len(shape)
        sl[ax] = 0
        m[tuple(sl)] = False
        sl[ax] = -1
        m[tuple(sl)] = False
    return m


def _shift(f, offs):
    """g[x] = f[x + offs] with zeros outside the grid."""
    g = np.zeros_like(f)
    src, dst = [], []
    for o, n in zip(offs, f.shape):
        if o >= 0:
            src.append(slice(o, n)); dst.append(slice(0, n - o))
        else:
            src.append(slice(0, n + o)); dst.append(slice(-o, n))
    g[tuple(dst)] = f[tuple(src)]
    return g


def _axial_sum(f):
    d = f.ndim
    out = np.zeros_like(f)
    for ax in range(d):
        for sg in (-1, 1):
            offs = [0] * d
            offs[ax] = sg
            out += _shift(f, offs)
    return out


def _edge_sum(f):
    d = f.ndim
    out = np.zeros_like(f)
    for a1, a2 in itertools.combinations(range(d), 2):
        for s1 in (-1, 1):
            for s2 in (-1, 1):
                offs = [0] * d
                offs[a1], offs[a2] = s1, s2
                out += _shift(f, offs)
    return out


def rhs_vjp(prob: Problem, Y, V, w):
    """(J_F(Y)^T w, dF/dV^T w): the transposes of the derivative of F at Y
    with respect to the state and to V, applied to the cotangent w."""
    d = Y.ndim
    a, s, h = prob.a, prob.s, prob.h
    inner = _interior(Y.shape)
    bnd = ~inner
    # F = i a Lap + ...: transpose of Lap -> i a Lap is u -> -i a u; F_b = 0.
    u = np.where(inner, -1j * a * w, 0)
    if prob.lap == LAP_CD:
        E = u                                              # Lap = D
    else:
        E = (16 - 2 * d) / 12 * u - _axial_sum(u) / 12     # transpose of step 2 in D
    # Transpose of step 1 (interior D_j = delta^2 Y_j).
    E_in = np.where(inner, E, 0)
    Ybar = (_axial_sum(E_in) - 2 * d * E_in) / h ** 2
    if prob.lap != LAP_CD:                                 # edge terms of step 2
        ne = 2 * d * (d - 1)
        Ybar += (_edge_sum(u) - ne * u) / (6 * h * h)
    # Boundary D_b = -(s|Y_b|^2 - V_b) Y_b / a: derivative alpha dY + beta conj(dY).
    rho = np.abs(Y) ** 2
    alpha = -(2 * s * rho - V) / a
    beta = -s * Y * Y / a
    Ybar += np.where(bnd, alpha * E + beta * np.conj(E), 0)
    # Pointwise i(s|Y|^2 - V) Y at interior points.
    Ybar += np.where(inner, -1j * (2 * s * rho - V) * w + 1j * s * Y * Y * np.conj(w), 0)
    # V: dF_p/dV_p = -i Y_p (interior); dD_b/dV_b = Y_b / a (boundary).
    gV = np.where(inner, np.imag(np.conj(w) * Y), 0) + np.where(bnd, np.real(np.conj(E) * Y) / a, 0)
    return Ybar, gV


def step_vjp(prob: Problem, psi, V, k, lam):
    """Reverse of one classic RK4 step (Eq. RK4) at state psi: given
    lam = dL/dpsi_{n+1}, returns (dL/dpsi_n, this step's dL/dV)."""
    Y1 = psi
    K1 = rhs(prob, Y1, V)
    Y2 = psi + k / 2 * K1
    K2 = rhs(prob, Y2, V)
    Y3 = psi + k / 2 * K2
    K3 = rhs(prob, Y3, V)
    Y4 = psi + k * K3
    Kb = [k / 6 * lam, k / 3 * lam, k / 3 * lam, k / 6 * lam]
    out = lam.copy()
    gV = np.zeros(psi.shape)
    Yb4, g = rhs_vjp(prob, Y4, V, Kb[3]); out += Yb4; gV += g; Kb[2] = Kb[2] + k * Yb4
    Yb3, g = rhs_vjp(prob, Y3, V, Kb[2]); out += Yb3; gV += g; Kb[1] = Kb[1] + k / 2 * Yb3
    Yb2, g = rhs_vjp(prob, Y2, V, Kb[1]); out += Yb2; gV += g; Kb[0] = Kb[0] + k / 2 * Yb2
    Yb1, g = rhs_vjp(prob, Y1, V, Kb[0]); out += Yb1; gV += g
    return out, gV


def loss_and_gradient(prob: Problem, psi0, V, target, k, nsteps):
    """L = sum |psi_T - target|^2 after nsteps RK4 steps, with dL/dpsi0
    (complex convention above) and dL/dV, by storing every state."""
    states = [np.asarray(psi0, complex)]
    for _ in range(nsteps):
        states.append(run(prob, states[-1], V, k, 1))
    diff = states[-1] - target
    loss = float(np.sum(np.abs(diff) ** 2))
    lam = 2 * diff
    gV = np.zeros(np.shape(V))
    for n in range(nsteps - 1, -1, -1):
        lam, g = step_vjp(prob, states[n], V, k, lam)
        gV += g
    return loss, lam, gV
