"""Each workload's accuracy statement checked at the workload's own step
count: the CUDA path against the FP64 oracle after the full run, on crops or
samples small enough for the oracle (run on all host cores; the threaded
oracle gives the serial oracle's bits).

Tolerances (relative L2 over the grid, as the workloads state them): FP32
<= 1e-5, FP64 <= 1e-12 against the oracle.  A crop is a separate, smaller
instance built from the workload's V and Psi0 cut out of the full grid, with
the workload's h and dt and Dirichlet boundaries on the cut.  Where a
workload misses its tolerance the test records the measured error instead
of passing silently (the batched focusing instances, which collapse).

Measured errors are printed (pytest -s shows them)."""
import numpy as np
import pytest
import torch

import oracle
from oracle import adjoint as oadj
from paper_1109_1027_gb300 import nlse
from paper_1109_1027_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

DEV = "cuda:0"
THREADS = oracle.threads_available()


def to_dev(arr, prec):
    if np.iscomplexobj(arr):
        dt = torch.complex64 if prec == "fp32" else torch.complex128
    else:
        dt = torch.float32 if prec == "fp32" else torch.float64
    return torch.from_numpy(np.ascontiguousarray(arr)).to(DEV).to(dt).contiguous()


def rounded(arr, prec):
    if prec == "fp64":
        return np.asarray(arr)
    if np.iscomplexobj(arr):
        return np.asarray(arr).astype(np.complex64).astype(np.complex128)
    return np.asarray(arr).astype(np.float32).astype(np.float64)


def rel_l2(a, b):
    return float(np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel()))


def _run_both(shape, h, a, s, psi, V, k, steps, prec):
    """(GPU result, oracle result) after `steps` RK4 steps from the same bytes."""
    prob = oracle.Problem(shape, h, a, s)
    ref = oracle.run(prob, rounded(psi, prec), rounded(V, prec), k, steps, threads=THREADS)
    solver = nlse.Solver(to_dev(V, prec), h, k, a, s, prec=prec)
    x = to_dev(psi, prec)
    solver.run(x, steps)
    solver.check()
    got = x.cpu().numpy()
    solver.close()
    return got, ref


@pytest.fixture(scope="module")
def vortex_crop():
    """The 2D dark vortex workload (2048^2 on [-60, 60]^2), its centred 256^2 crop."""
    full = wl.dark_vortex_2d(n=2048, steps=10000)
    c0 = (2048 - 256) // 2
    sl = (slice(c0, c0 + 256), slice(c0, c0 + 256))
    psi, V = full.psi0[sl].copy(), full.V[sl].copy()
    prob = oracle.Problem(psi.shape, full.h, full.a, full.s)
    k = 0.5 * oracle.invariants(prob, psi, V)[2]
    return full, psi, V, k


@pytest.mark.parametrize("prec,tol", [("fp32", 1e-5), ("fp64", 1e-12)])
def test_dark_vortex_crop_after_the_workloads_10000_steps(vortex_crop, prec, tol):
    full, psi, V, k = vortex_crop
    got, ref = _run_both(psi.shape, full.h, full.a, full.s, psi, V, k, full.steps, prec)
    err = rel_l2(got, ref)
    print(f"\ndark vortex 256^2 crop, {full.steps} steps, {prec}: rel L2 vs oracle {err:.3e}")
    assert err <= tol


def _ring_crops():
    full = wl.vortex_ring_3d(n=512, steps=2000)
    cx, cy = full.meta["centre"]
    ax = wl.axis(512, full.lo, full.hi)
    h = full.h
    out = {}
    # the centred crop, and one centred on the ring's core (the vortex line
    # crosses the crop; the centred one holds the ring's smooth interior)
    for name, (x0, y0, z0) in {"centre": (0.0, 0.0, 0.0), "ring core": (cx + full.meta["radius"], cy, 0.0)}.items():
        ix = int(np.argmin(np.abs(ax - x0))) - 32
        iy = int(np.argmin(np.abs(ax - y0))) - 32
        iz = int(np.argmin(np.abs(ax - z0))) - 32
        sl = (slice(iz, iz + 64), slice(iy, iy + 64), slice(ix, ix + 64))
        out[name] = (full.psi0[sl].copy(), full.V[sl].copy())
    return full, h, out


@pytest.fixture(scope="module")
def ring_crops():
    full, h, crops = _ring_crops()
    ks = {}
    for name, (psi, V) in crops.items():
        prob = oracle.Problem(psi.shape, h, full.a, full.s)
        ks[name] = 0.5 * oracle.invariants(prob, psi, V)[2]
    return full, h, crops, ks


@pytest.mark.parametrize("crop", ["centre", "ring core"])
@pytest.mark.parametrize("prec,tol", [("fp32", 1e-5), ("fp64", 1e-12)])
def test_vortex_ring_crop_after_the_workloads_2000_steps(ring_crops, crop, prec, tol):
    full, h, crops, ks = ring_crops
    psi, V = crops[crop]
    got, ref = _run_both(psi.shape, h, full.a, full.s, psi, V, ks[crop], full.steps, prec)
    err = rel_l2(got, ref)
    print(f"\nvortex ring 64^3 crop ({crop}), {full.steps} steps, {prec}: rel L2 vs oracle {err:.3e}")
    assert err <= tol


def test_vortex_ring_fp32_against_the_fp64_gpu_run(ring_crops):
    """The workload's own comparison: FP32 against an FP64 GPU run."""
    full, h, crops, ks = ring_crops
    psi, V = crops["ring core"]
    res = {}
    for prec in ("fp32", "fp64"):
        sv = nlse.Solver(to_dev(V, prec), h, ks["ring core"], full.a, full.s, prec=prec)
        x = to_dev(psi, prec)
        sv.run(x, full.steps)
        sv.check()
        res[prec] = x.cpu().numpy()
        sv.close()
    err = rel_l2(res["fp32"].astype(np.complex128), res["fp64"])
    print(f"\nvortex ring 64^3 crop (ring core), FP32 vs FP64 GPU: {err:.3e}")
    assert err <= 1e-5


def _batch_sample():
    """Sampled instances of the batched workload: for each sign of s, the two
    smallest sides present and one of side 256 (several tiles, ragged)."""
    params = wl.gaussian_batch_params(count=512, seed=4)
    chosen = []
    for sgn in (-1.0, 1.0):
        mine = sorted([i for i, p in enumerate(params) if p["s"] == sgn], key=lambda i: (params[i]["n"], i))
        chosen += mine[:2]
        chosen.append(next(i for i in mine if params[i]["n"] == 256))
    return wl.gaussian_batch_2d(count=512, seed=4, steps=5000, only=set(chosen))


def test_batched_sample_after_the_workloads_5000_steps():
    insts = _batch_sample()
    steps = insts[0].steps
    shapes = [q.shape for q in insts]
    ks = [0.5 * oracle.invariants(oracle.Problem(q.shape, q.h, q.a, q.s), q.psi0, q.V)[2] for q in insts]
    res = {}
    for prec, cdt, rdt in (("fp32", torch.complex64, torch.float32), ("fp64", torch.complex128, torch.float64)):
        V = nlse.BatchSolver.pack([rounded(q.V, prec) for q in insts], rdt, DEV)
        x = nlse.BatchSolver.pack([rounded(q.psi0, prec) for q in insts], cdt, DEV)
        bs = nlse.BatchSolver(V, shapes, [q.h for q in insts], ks, [q.a for q in insts], [q.s for q in insts],
                              prec=prec)
        bs.run(x, steps)
        try:
            bs.check()
        except nlse.NLSEError as err:
            assert err.code == nlse.ENONFINITE and "entry check" not in str(err)
        res[prec] = [g.cpu().numpy() for g in bs.unpack(x)]
        bs.close()
    for i, q in enumerate(insts):
        prob = oracle.Problem(q.shape, q.h, q.a, q.s)
        errs = {}
        finite = {}
        for prec in ("fp32", "fp64"):
            ref = oracle.run(prob, rounded(q.psi0, prec), rounded(q.V, prec), ks[i], steps, threads=THREADS)
            finite[prec] = bool(np.isfinite(ref).all())
            errs[prec] = rel_l2(res[prec][i], ref) if finite[prec] else None
        print(f"\nbatch {q.name}: side {q.shape[0]}, s = {q.s:+.0f}, a = {q.a:.3f}: oracle finite {finite}, "
              f"rel L2 {errs}")
        if q.s < 0:
            assert finite["fp32"] and finite["fp64"]
            assert errs["fp32"] <= 1e-5 and errs["fp64"] <= 1e-12
        else:
            # focusing: the oracle and the GPU collapse alike, or neither does
            for prec in ("fp32", "fp64"):
                assert finite[prec] == bool(np.isfinite(res[prec][i]).all()), (q.name, prec)


@pytest.fixture(scope="module")
def gradient_crop():
    """The gradient workload's V, first Psi0 and target (512^2 on [-16, 16]^2),
    their centred 64^2 crop."""
    V, psis, targets, h, a, s = wl.gradient_problem_2d(n=512, batch=1)
    c0 = (512 - 64) // 2
    sl = (slice(c0, c0 + 64), slice(c0, c0 + 64))
    V, psi0, target = V[sl].copy(), psis[0][sl].copy(), targets[0][sl].copy()
    prob = oracle.Problem((64, 64), h, a, s)
    k = 0.5 * oracle.invariants(prob, psi0, V)[2]
    L0, g0, gV0 = oadj.loss_and_gradient(prob, psi0, V, target, k, 3000)
    return V, psi0, target, h, a, s, k, (L0, g0, gV0)


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-10), ("fp32", 2e-4)])
def test_gradient_crop_after_the_workloads_3000_steps(gradient_crop, prec, tol):
    """The checkpointed adjoint (checkpoints every 100 steps) after 3000 steps
    against the FP64 reference gradient; FP64 also against central
    differences of the GPU forward (eps = 1e-4)."""
    V, psi0, target, h, a, s, k, (L0, g0, gV0) = gradient_crop
    solver = nlse.Solver(to_dev(V, prec), h, k, a, s, prec=prec, check_stability=False)
    t = lambda z: to_dev(z, prec)
    L, g, gV = solver.adjoint(t(psi0), t(target), 3000, ckpt_every=100)
    eg = np.abs(g.cpu().numpy() - g0).max() / np.abs(g0).max()
    ev = np.abs(gV.cpu().numpy() - gV0).max() / np.abs(gV0).max()
    print(f"\ngradient 64^2 crop, 3000 steps, {prec}: loss {L:.10e} vs {L0:.10e}, "
          f"dL/dpsi0 err {eg:.3e}, dL/dV err {ev:.3e}")
    assert L == pytest.approx(L0, rel=1e-12 if prec == "fp64" else 2e-5)
    assert eg <= tol and ev <= tol
    if prec == "fp64":
        def loss_of(p, v):
            sv = nlse.Solver(v, h, k, a, s, prec="fp64", check_stability=False)
            x = p.clone()
            sv.run(x, 3000)
            sv.close()
            return float(((x - t(target)).abs() ** 2).sum())
        eps = 1e-4
        d = t(wl.random_field((64, 64), seed=177))
        Vd = t(V)
        fd = (loss_of(t(psi0) + eps * d, Vd) - loss_of(t(psi0) - eps * d, Vd)) / (2 * eps)
        assert float(torch.real(torch.sum(torch.conj(g) * d))) == pytest.approx(fd, rel=1e-6)
    solver.close()
