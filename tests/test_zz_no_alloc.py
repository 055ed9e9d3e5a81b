"""nlse_invariants_noalloc: the invariants for callers that cannot allocate
device memory (code inside a framework that owns all device memory, or a
latency-critical path that cannot take a cudaMalloc's synchronisation).

It runs the reductions of nlse_invariants with its scratch in a static device
array of the library instead of a context's allocation.  Checked here through
the C ABI against nlse_invariants, on two calls in a row with different
states, so that a call reading what the previous call left in the shared
array would show.  This file is collected last on purpose.
"""
import ctypes

import numpy as np
import pytest
import torch

from paper_1109_1027_gb300 import nlse
from paper_1109_1027_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

DEV = "cuda:0"


def _dev(arr, dtype):
    return torch.from_numpy(np.ascontiguousarray(arr)).to(DEV).to(dtype).contiguous()


@pytest.mark.parametrize("shape,prec", [((1030,), "fp64"), ((67, 200), "fp64"), ((67, 200), "fp32"),
                                        ((35, 18, 40), "fp64"), ((512, 512), "fp32")])
def test_noalloc_matches_invariants_on_two_calls(shape, prec):
    cdt = torch.complex64 if prec == "fp32" else torch.complex128
    rdt = torch.float32 if prec == "fp32" else torch.float64
    h, a, s = 0.4, 0.6, -0.9
    V = _dev(wl.random_potential(shape, seed=91, scale=2.0), rdt)
    solver = nlse.Solver(V, h, 1e-4, a, s, prec=prec)
    params = nlse.make_params(shape, h, 1e-4, a, s, prec=prec)
    for seed in (92, 93):                      # two calls in a row, different states
        psi = _dev(wl.random_field(shape, seed=seed), cdt)
        ref = solver.invariants(psi)
        got = nlse.nlse_invariants_noalloc(params, psi.data_ptr(), V.data_ptr())
        assert got[0] == pytest.approx(ref[0], rel=1e-12)
        assert got[1] == pytest.approx(ref[1], rel=1e-11)
        assert got[2] == pytest.approx(ref[2], rel=1e-12)
    solver.close()


def test_noalloc_rejects_grids_beyond_its_scratch():
    lib = nlse.load_library()
    params = nlse.make_params((8193, 8193), 0.1, 1e-4, 1.0, 1.0, prec="fp32")
    m = ctypes.c_double()
    rc = lib.nlse_invariants_noalloc(ctypes.byref(params), ctypes.c_void_p(4096), ctypes.c_void_p(4096),
                                     ctypes.byref(m), None, None, None)
    assert rc == nlse.EINVAL
    assert "67,108,864" in lib.nlse_last_error().decode()


def test_noalloc_refuses_a_stack():
    """A stack of grids (NLSE_FLAG_STACK) is refused before any device work."""
    lib = nlse.load_library()
    params = nlse.make_params((64, 64), 0.1, 1e-4, 1.0, 1.0, prec="fp32")
    params.n[2] = 3
    params.flags |= nlse.FLAG_STACK
    m = ctypes.c_double()
    rc = lib.nlse_invariants_noalloc(ctypes.byref(params), ctypes.c_void_p(4096), ctypes.c_void_p(4096),
                                     ctypes.byref(m), None, None, None)
    assert rc == nlse.EUNSUPPORTED
    assert "stack" in lib.nlse_last_error().decode()
