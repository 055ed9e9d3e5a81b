"""The bounds-check build (-DNLSE_BOUNDS_CHECK, libnlse_checked.so) on the
parity shapes: every kernel tests its shared-memory and global indices and
its TMA coordinates before the access and reports NLSE_EBOUNDS through
nlse_check instead of accessing out of range.  A child process loads the
checked library (NLSE_LIBRARY) and runs each kernel family -- 1D tiled and
resident, 2D TMA walk and generic tile, 3D TMA walk and generic 2.5D,
multi-storage, CD, MSD, periodic and Laplacian-zero through the unfused
kernels, stacks, batches, two stages per launch, the entry check, the
adjoint's TMA row walk and tile kernel -- on grids
of 3 to 9 points per axis, odd widths and tiles with ragged edges, checking
the status after every call and the results against the FP64 oracle.  This
stands in for a race/bounds checker, which is closed on this machine."""
import os
import subprocess
import sys

import pytest

from paper_1109_1027_gb300 import build as nbuild

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r'''
import sys
sys.path.insert(0, {root!r})
sys.path.insert(0, {tests!r})
import numpy as np
import torch
import oracle
from paper_1109_1027_gb300 import nlse
from paper_1109_1027_gb300 import workloads as wl
assert nlse.load_library()._name == {lib!r}, nlse.load_library()._name
DEV = "cuda:0"
OBC = {{"dirichlet": 0, "msd": 1, "periodic": 2, "lapzero": 3}}
OLAP = {{"2shoc": 0, "cd": 1, "2shoc_ms": 2}}

def dev(a, prec):
    if np.iscomplexobj(a):
        t = torch.complex64 if prec == "fp32" else torch.complex128
    else:
        t = torch.float32 if prec == "fp32" else torch.float64
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV).to(t).contiguous()

def rnd(a, prec):
    if prec == "fp64":
        return a
    return a.astype(np.complex64).astype(np.complex128) if np.iscomplexobj(a) else a.astype(np.float32).astype(np.float64)

def field(shape, bc, seed):
    if bc == "msd":
        xs = wl.mesh(shape, -1.0, 1.0)
        return (2.0 + 0.05 * np.cos(3.0 * xs[0])) * np.exp(1j * sum(0.7 * (i + 1) * x for i, x in enumerate(xs))) \
            + 1e-3 * wl.random_field(shape, seed=seed)
    return wl.random_field(shape, seed=seed) + 1.5

count = 0
def case(shape, prec, lap, bc, tiling=()):
    global count
    h, a, s = 0.45, 0.8, -1.1
    psi, V = field(shape, bc, 7 + len(shape)), wl.random_potential(shape, seed=9, scale=1.5)
    prob = oracle.Problem(shape, h, a, s, bc=OBC[bc], lap=OLAP[lap])
    k = 0.3 * oracle.invariants(prob, rnd(psi, prec), rnd(V, prec))[2]
    sv = nlse.Solver(dev(V, prec), h, k, a, s, bc=bc, prec=prec, lap=lap)
    for key, val in tiling:
        sv.set_tiling(key, val)
    x = dev(psi, prec)
    lap_ = sv.lap2shoc(x)
    sv.check()
    ref = oracle.laplacian(prob, rnd(psi, prec), rnd(V, prec))
    assert np.abs(lap_.cpu().numpy() - ref).max() <= (1e-11 if prec == "fp64" else 2e-5) * max(np.abs(ref).max(), 1.0), \
        (shape, prec, lap, bc)
    sv.run(x, 3)
    sv.check()
    sv.rk4_step(x)
    sv.check()
    sv.invariants(x)
    sv.check()
    ref = oracle.run(prob, rnd(psi, prec), rnd(V, prec), k, 4)
    err = np.linalg.norm(x.cpu().numpy() - ref) / np.linalg.norm(ref)
    assert err <= (1e-12 if prec == "fp64" else 1e-5), (shape, prec, lap, bc, err)
    sv.close()
    count += 1

shapes = {{1: [(3,), (5,), (9,), (1030,), (5000,)],
           2: [(3, 3), (5, 7), (9, 4), (17, 70), (40, 131), (45, 260), (33, 4), (70, 128), (19, 516)],
           3: [(3, 3, 3), (5, 7, 9), (9, 20, 37), (35, 18, 40), (5, 17, 64), (40, 9, 36)]}}
for d, ss in shapes.items():
    for shape in ss:
        for prec in ("fp64", "fp32"):
            for lap in ("2shoc", "cd", "2shoc_ms"):
                case(shape, prec, lap, "dirichlet")
            for bc in ("msd", "periodic", "lapzero"):
                if min(shape) >= 4:
                    case(shape, prec, "2shoc", bc)
# launch shapes: rows per CTA, planes per CTA, the 1D resident cluster, two stages per launch
for tl in ([(nlse.TILE_ROWS, 8)], [(nlse.TILE_ROWS, 32)], [(nlse.TILE_2D_FUSE, 1)]):
    for shape in [(17, 68), (45, 260), (70, 128), (5, 8)]:
        case(shape, "fp32", "2shoc", "dirichlet", tl)
for tl in ([(nlse.TILE_PLANES, 64)], [(nlse.TILE_PLANES, 128)]):
    case((70, 20, 36), "fp32", "2shoc", "dirichlet", tl)
for tl in ([(nlse.TILE_1D_RESIDENT, 0)], [(nlse.TILE_1D_RESIDENT, 1)], [(nlse.TILE_1D_RESIDENT, 4)]):
    case((37,), "fp32", "2shoc", "dirichlet", tl)
    case((2049,), "fp64", "2shoc", "msd", tl)

# stacks and batches
for prec in ("fp32", "fp64"):
    V = wl.random_potential((9, 12), seed=3, scale=1.0)
    st = nlse.Solver(dev(V, prec), 0.4, 1e-3, 0.7, -1.0, prec=prec, stack=3)
    x = dev(np.stack([wl.random_field((9, 12), seed=20 + i) for i in range(3)]), prec)
    st.run(x, 5)
    st.check()
    st.lap2shoc(x)
    st.invariants(x)
    st.check()
    st.close()
    shapes_b = [(5, 8), (64, 64), (33, 132), (3, 4), (130, 256)]
    Vs = [wl.random_potential(sh, seed=40 + i, scale=1.0) for i, sh in enumerate(shapes_b)]
    ps = [wl.random_field(sh, seed=50 + i) for i, sh in enumerate(shapes_b)]
    rdt = torch.float32 if prec == "fp32" else torch.float64
    cdt = torch.complex64 if prec == "fp32" else torch.complex128
    bs = nlse.BatchSolver(nlse.BatchSolver.pack(Vs, rdt, DEV), shapes_b, 0.4, 1e-3, 0.7, -1.0, prec=prec)
    x = nlse.BatchSolver.pack(ps, cdt, DEV)
    bs.run(x, 5)
    bs.check()
    bs.lap2shoc(x)
    bs.check()
    host = x.cpu().pin_memory()
    bs.run_host(host, 2)
    bs.close()
# the reversed stages of the adjoint: TMA row walk (8, 16, 32 rows) and tile kernel
for prec in ("fp32", "fp64"):
    rdt = torch.float32 if prec == "fp32" else torch.float64
    cdt = torch.complex64 if prec == "fp32" else torch.complex128
    for shape, stack in (((5, 8), 0), ((19, 68), 0), ((9, 260), 0), ((7, 12), 3), ((6, 10), 0)):
        V = wl.random_potential(shape, seed=61, scale=1.0)
        Vd = torch.from_numpy(V).to(DEV).to(rdt).contiguous()
        n = max(stack, 1)
        x0 = torch.stack([torch.from_numpy(wl.random_field(shape, seed=70 + i)) for i in range(n)]).to(DEV).to(cdt)
        tg = torch.stack([torch.from_numpy(wl.random_field(shape, seed=80 + i)) for i in range(n)]).to(DEV).to(cdt)
        if not stack:
            x0, tg = x0[0], tg[0]
        sv = nlse.Solver(Vd, 0.4, 1e-3, 0.7, -1.0, prec=prec, check_stability=False, stack=stack)
        outs = []
        for rows in (0, 8, 16, 32):
            sv.set_tiling(nlse.TILE_ADJ_ROWS, rows)
            outs.append(sv.adjoint(x0.contiguous(), tg.contiguous(), 3, 2))
            sv.check()
        for o in outs[1:]:
            assert o[0] == outs[0][0] and torch.equal(o[1], outs[0][1]) and torch.equal(o[2], outs[0][2]), shape
        sv.close()
        count += 1
print("checked cases:", count)
print("BOUNDS_CLEAN")
'''


def test_bounds_check_build_is_clean_on_the_parity_shapes():
    lib = nbuild.build(checked=True)
    script = CHILD.format(root=ROOT, tests=os.path.join(ROOT, "tests"), lib=lib)
    env = dict(os.environ, NLSE_LIBRARY=lib)
    r = subprocess.run([sys.executable, "-c", script], env=env, capture_output=True, text=True, timeout=1500)
    assert r.returncode == 0 and "BOUNDS_CLEAN" in r.stdout, (r.stdout[-3000:], r.stderr[-5000:])
