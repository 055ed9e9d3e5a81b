"""Pins of the FP64 reference adjoint (oracle/adjoint.py) against facts that
do not come from it: finite-difference derivatives of the (already pinned)
forward oracle, and, for the linear equation, the exact transpose of the
assembled one-step matrix."""
import numpy as np
import pytest

import oracle
from oracle import adjoint as oadj
from paper_1109_1027_gb300 import workloads as wl


def rdot(u, v):
    """Real inner product of complex fields viewed as (Re, Im) pairs."""
    return float(np.real(np.sum(np.conj(u) * v)))


CASES = [((17,), 0), ((9, 11), 0), ((6, 7, 8), 0), ((9, 11), 1), ((6, 7, 8), 1)]


@pytest.mark.parametrize("shape,lap", CASES)
def test_rhs_vjp_is_the_transpose_of_the_rhs_derivative(shape, lap):
    """<w, J v> = <J^T w, v> for the state and <w, dF/dV dv> = <gV, dv>, with
    J v taken by central differences of the oracle's F (Sec. 3.1)."""
    prob = oracle.Problem(shape, 0.45, 0.8, -1.3, lap=lap)
    Y = wl.random_field(shape, seed=21) + 1.5
    V = wl.random_potential(shape, seed=22, scale=3.0)
    v = wl.random_field(shape, seed=23)
    dv = wl.random_potential(shape, seed=24) - 0.5
    w = wl.random_field(shape, seed=25)
    eps = 1e-6
    jv = (oracle.rhs(prob, Y + eps * v, V) - oracle.rhs(prob, Y - eps * v, V)) / (2 * eps)
    jV = (oracle.rhs(prob, Y, V + eps * dv) - oracle.rhs(prob, Y, V - eps * dv)) / (2 * eps)
    Ybar, gV = oadj.rhs_vjp(prob, Y, V, w)
    lhs, rhs_ = rdot(w, jv), rdot(Ybar, v)
    assert lhs == pytest.approx(rhs_, rel=1e-7, abs=1e-7 * np.abs(lhs))
    lhs, rhs_ = rdot(w, jV), float(np.sum(gV * dv))
    assert lhs == pytest.approx(rhs_, rel=1e-7)


@pytest.mark.parametrize("shape", [(20,), (10, 12)])
def test_loss_gradient_matches_central_differences(shape):
    """dL/d eps along random directions of psi0 and of V, L = sum |psi_T - target|^2
    after 6 RK4 steps, against central differences of the forward oracle."""
    prob = oracle.Problem(shape, 0.5, 0.7, -1.0)
    psi0 = 0.6 * wl.random_field(shape, seed=31) + 1.0
    V = wl.random_potential(shape, seed=32)
    target = wl.random_field(shape, seed=33)
    _, _, dtmax = oracle.invariants(prob, psi0, V)
    k, n = 0.5 * dtmax, 6
    loss, g_psi, g_V = oadj.loss_and_gradient(prob, psi0, V, target, k, n)

    def L(p, v):
        return float(np.sum(np.abs(oracle.run(prob, p, v, k, n) - target) ** 2))

    assert loss == pytest.approx(L(psi0, V), rel=1e-14)
    eps = 1e-5
    d = wl.random_field(shape, seed=34)
    fd = (L(psi0 + eps * d, V) - L(psi0 - eps * d, V)) / (2 * eps)
    assert rdot(g_psi, d) == pytest.approx(fd, rel=1e-7)
    dv = wl.random_potential(shape, seed=35) - 0.5
    fd = (L(psi0, V + eps * dv) - L(psi0, V - eps * dv)) / (2 * eps)
    assert float(np.sum(g_V * dv)) == pytest.approx(fd, rel=1e-7)


def test_linear_gradient_is_the_exact_matrix_transpose():
    """For s = 0 one step is psi_1 = M psi_0 with M complex-linear, so
    dL/dpsi0 = 2 M^H (M psi0 - target) exactly; M is assembled column by
    column from the forward oracle."""
    shape = (5, 6)
    prob = oracle.Problem(shape, 0.5, 0.9, 0.0)
    V = wl.random_potential(shape, seed=41)
    psi0 = wl.random_field(shape, seed=42)
    target = wl.random_field(shape, seed=43)
    k = 0.02
    N = psi0.size
    M = np.zeros((N, N), complex)
    for j in range(N):
        e = np.zeros(N, complex)
        e[j] = 1.0
        M[:, j] = oracle.run(prob, e.reshape(shape), V, k, 1).ravel()
    _, g, _ = oadj.loss_and_gradient(prob, psi0, V, target, k, 1)
    expect = 2 * M.conj().T @ (M @ psi0.ravel() - target.ravel())
    assert np.abs(g.ravel() - expect).max() <= 1e-12 * np.abs(expect).max()
