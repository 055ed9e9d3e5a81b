"""The OpenMP build of the oracle gives the serial build's bits: its
work-sharing pragmas sit only on loops that compute each grid point's value
independently, so the thread count changes nothing but the time.  Checked for
every boundary rule and Laplacian form, 1D to 3D, with 1, 3 and 4 threads."""
import numpy as np
import pytest

import oracle
from paper_1109_1027_gb300 import workloads as wl

CASES = [((37,), 0, 0), ((40, 33), 0, 0), ((40, 33), 1, 0), ((40, 33), 0, 1), ((40, 33), 0, 2),
         ((24, 26), 2, 0), ((24, 26), 3, 0), ((9, 11, 13), 0, 0), ((9, 11, 13), 0, 2), ((9, 11, 13), 1, 0)]


@pytest.mark.parametrize("shape,bc,lap", CASES)
def test_threaded_oracle_equals_serial_oracle(shape, bc, lap):
    if bc == oracle.BC_MSD:
        # the MSD rule is meant for a nearly constant modulus at the boundary
        # (on white noise it blows up in a few steps, in either build)
        xs = wl.mesh(shape, -1.0, 1.0)
        psi = (2.0 + 0.05 * np.cos(3.0 * xs[0])) * np.exp(1j * sum(0.7 * (i + 1) * x for i, x in enumerate(xs)))
        psi = psi + 1e-3 * wl.random_field(shape, seed=11)
    else:
        psi = wl.random_field(shape, seed=11) + 2.0
    V = wl.random_potential(shape, seed=12)
    prob = oracle.Problem(shape, 0.4, 0.8, -1.0, bc=bc, lap=lap)
    k = 0.3 * oracle.invariants(prob, psi, V)[2]
    ref = oracle.run(prob, psi, V, k, 6)
    assert np.isfinite(ref).all()
    for threads in (3, 4):
        got = oracle.run(prob, psi, V, k, 6, threads=threads)
        assert np.array_equal(got.view(np.uint64), ref.view(np.uint64)), threads


def test_threads_used_is_reported():
    assert oracle.threads_used(1) == 1
    n = oracle.threads_used(3)
    assert n in (1, 3)          # 1 only where the compiler has no OpenMP
