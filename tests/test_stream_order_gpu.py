"""nlse_run is stream-ordered: its entry check runs on the device, its steps
are replays of cached CUDA graphs for any step count, and it can itself be
captured into a caller's CUDA graph (which fails if anything in it waits for
the host).  Through the C ABI on the GPU.

* Capture: torch.cuda.graph captures in the global mode, in which any host
  synchronisation or synchronous copy inside the capture is an error; the
  replayed graph must give the bits of an uncaptured nlse_run.
* Any step count: nlse_run(n) gives the bits of n calls of nlse_rk4_step.
* The device-side check gives, for the bound of Eq. (kdfull), the value that
  nlse_invariants computes on the host's request (FP64, including the FP32
  compensated part), to 1e-13: the FP32 pre-filter of check.cu may not change
  an extreme.
"""
import re

import numpy as np
import pytest
import torch

from paper_1109_1027_gb300 import nlse
from paper_1109_1027_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

DEV = "cuda:0"


def _dev(arr, prec):
    if np.iscomplexobj(arr):
        dt = torch.complex64 if prec == "fp32" else torch.complex128
    else:
        dt = torch.float32 if prec == "fp32" else torch.float64
    return torch.from_numpy(np.ascontiguousarray(arr)).to(DEV).to(dt).contiguous()


def _smooth(shape, seed):
    """A smooth field (Gaussian bump with a phase gradient, small noise)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    xs = wl.mesh(shape, -4.0, 4.0)
    r2 = sum(x * x for x in xs)
    ph = sum(rng.uniform(-1, 1) * x for x in xs)
    return np.exp(-r2 / 4.0) * np.exp(1j * ph) + 0.01 * wl.random_field(shape, seed=seed + 1)


def _solver(shape, prec, seed, stack=0, check=True, dt_frac=0.5, h=0.2, a=0.7, s=-1.0):
    V = 0.05 * wl.random_potential(shape, seed=seed, scale=1.0) + 0.1
    Vd = _dev(V, prec)
    probe = nlse.Solver(Vd, h, 1.0, a, s, prec=prec, check_stability=False, stack=stack)
    psi = np.stack([_smooth(shape, seed + 10 + i) for i in range(stack)]) if stack else _smooth(shape, seed + 10)
    x = _dev(psi, prec)
    dtmax = probe.invariants(x)[2]
    probe.close()
    sv = nlse.Solver(Vd, h, dt_frac * dtmax, a, s, prec=prec, check_stability=check, stack=stack)
    return sv, psi, Vd, dtmax


CAPTURE_CASES = [((70, 128), "fp32", 0), ((70, 128), "fp64", 0), ((40, 131), "fp32", 0), ((35, 18, 40), "fp32", 0),
                 ((35, 18, 40), "fp64", 0), ((1030,), "fp32", 0), ((5000,), "fp64", 0), ((24, 64), "fp32", 3)]


@pytest.mark.parametrize("shape,prec,stack", CAPTURE_CASES)
def test_run_can_be_captured_into_a_cuda_graph(shape, prec, stack):
    s1, psi, Vd, _ = _solver(shape, prec, 300, stack=stack)
    s2, _, _, _ = _solver(shape, prec, 300, stack=stack)
    x1 = _dev(psi, prec)
    s1.run(x1, 20)
    s1.check()
    x2 = _dev(psi, prec)
    # The first call for a state pointer binds it (in FP32: zeroes the
    # compensated part); bound outside the capture, the graph holds the steps
    # alone and can be replayed to continue the run.
    s2.run(x2, 0)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):                       # global capture mode: no host waits allowed
        s2.run(x2, 20)
    g.replay()
    torch.cuda.synchronize()
    s2.check()
    assert torch.equal(x1, x2)
    g.replay()                                      # 20 more steps
    s1.run(x1, 20)
    torch.cuda.synchronize()
    assert torch.equal(x1, x2)


def test_batch_run_can_be_captured_after_its_first_call():
    """A batch encodes its per-instance tensor maps when it first sees a
    state pointer (that step synchronises); later calls are stream-ordered."""
    sides = [(64, 64), (40, 68), (130, 256)]
    shapes, Vs, psis, hs = [], [], [], []
    for i, sh in enumerate(sides):
        shapes.append(sh)
        Vs.append(0.1 + 0.05 * wl.random_potential(sh, seed=400 + i, scale=1.0))
        psis.append(_smooth(sh, 410 + i))
        hs.append(0.2)
    V = nlse.BatchSolver.pack(Vs, torch.float32, DEV)
    probe = nlse.BatchSolver(V, shapes, hs, 1.0, 0.7, -1.0, prec="fp32", check_stability=False)
    x = nlse.BatchSolver.pack(psis, torch.complex64, DEV)
    dts = [0.5 * d for d in probe.invariants(x)[2]]
    probe.close()
    b1 = nlse.BatchSolver(V, shapes, hs, dts, 0.7, -1.0, prec="fp32")
    b2 = nlse.BatchSolver(V, shapes, hs, dts, 0.7, -1.0, prec="fp32")
    x1 = nlse.BatchSolver.pack(psis, torch.complex64, DEV)
    x2 = nlse.BatchSolver.pack(psis, torch.complex64, DEV)
    b1.run(x1, 12)
    b2.run(x2, 0)                                   # binds the state pointer outside the capture
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        b2.run(x2, 12)
    g.replay()
    torch.cuda.synchronize()
    b1.check()
    b2.check()
    assert torch.equal(x1, x2)


@pytest.mark.parametrize("fuse", [0, 1])
@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_any_step_count_gives_the_bits_of_single_steps(prec, fuse):
    if fuse and prec == "fp64":
        pytest.skip("two stages per launch is an FP32 schedule")
    s1, psi, Vd, _ = _solver((70, 128), prec, 500)
    s2, _, _, _ = _solver((70, 128), prec, 500)
    s1.set_tiling(nlse.TILE_2D_FUSE, fuse)
    x1, x2 = _dev(psi, prec), _dev(psi, prec)
    total = 0
    for n in (1, 2, 3, 5, 20, 31, 32, 33, 64, 70):
        s1.run(x1, n)
        for _ in range(n):
            s2.rk4_step(x2)
        total += n
        assert torch.equal(x1, x2), (n, total)
    s1.check()
    s2.check()


def _refusal(solver, x, n=3):
    """Runs n steps that the entry check must refuse; returns the bound the
    device reports (the state must be left as it was)."""
    x0 = x.clone()
    solver.run(x, n)
    with pytest.raises(nlse.NLSEError) as ei:
        solver.check()
    assert ei.value.code == nlse.EUNSTABLE, str(ei.value)
    assert torch.equal(x, x0)
    solver.check()                                  # cleared
    m = re.search(r"exceeds the bound ([-+0-9.eE]+)", str(ei.value))
    assert m, str(ei.value)
    return float(m.group(1))


def _fields(shape, kind, s, seed):
    rng = np.random.Generator(np.random.PCG64(seed))
    if kind == "random":
        return wl.random_field(shape, seed=seed), wl.random_potential(shape, seed=seed + 1, scale=2.0)
    if kind == "cancel":
        # V = s |psi|^2 up to FP32 rounding: u = s|psi|^2 - V is pure rounding noise
        psi = wl.random_field(shape, seed=seed).astype(np.complex64).astype(np.complex128)
        return psi, (s * np.abs(psi) ** 2).astype(np.float32).astype(np.float64)
    # |psi| = 1 + 1e-7 noise: FP32 cannot tell most points apart
    ph = rng.uniform(0, 2 * np.pi, shape)
    return (1.0 + 1e-7 * rng.standard_normal(shape)) * np.exp(1j * ph), np.zeros(shape)


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
@pytest.mark.parametrize("kind", ["random", "cancel", "flat"])
@pytest.mark.parametrize("shape", [(70, 128), (1030,), (9, 20, 36)])
def test_device_check_bound_equals_the_invariants_bound(shape, kind, prec):
    """The bound the device check computes (FP32 pre-filter, FP64 extremes)
    equals nlse_invariants' dt_max of the same state."""
    h, a, s = 0.3, 0.6, -1.3
    psi, V = _fields(shape, kind, s, 700)
    Vd = _dev(V, prec)
    sv = nlse.Solver(Vd, h, 1e3, a, s, prec=prec)
    x = _dev(psi, prec)
    bound = _refusal(sv, x)
    ref = sv.invariants(x, energy=False)[2]
    assert bound == pytest.approx(ref, rel=1e-13)
    # dt just below the bound is accepted, just above it refused
    ok = nlse.Solver(Vd, h, ref * (1 - 1e-12), a, s, prec=prec)
    y = _dev(psi, prec)
    ok.run(y, 1)
    ok.check()
    assert not torch.equal(y, x)
    bad = nlse.Solver(Vd, h, ref * (1 + 1e-12), a, s, prec=prec)
    _refusal(bad, _dev(psi, prec), n=1)


def test_device_check_reads_the_compensated_part():
    """A focusing state whose bound of Eq. (kdfull) shrinks as it steps: the
    check refuses once dt exceeds the current bound, and that bound -- taken
    from the FP32 state and its nonzero compensated part -- equals
    nlse_invariants' dt_max of the same state."""
    shape = (64, 96)
    h, a, s = 0.5, 0.5, 1.0
    xs, ys = wl.mesh(shape, -0.5 * h * (shape[1] - 1), 0.5 * h * (shape[1] - 1))
    psi = np.sqrt(24.0) * np.exp(-(xs ** 2 + ys ** 2)) * np.exp(0.3j * xs)
    Vd = _dev(np.zeros(shape), "fp32")
    probe = nlse.Solver(Vd, h, 1.0, a, s, prec="fp32", check_stability=False)
    dt0 = probe.invariants(_dev(psi, "fp32"), energy=False)[2]
    probe.close()
    sv = nlse.Solver(Vd, h, 0.98 * dt0, a, s, prec="fp32")
    x = _dev(psi, "fp32")
    for _ in range(400):
        before = x.clone()
        sv.run(x, 1)
        try:
            sv.check()
        except nlse.NLSEError as err:
            assert err.code == nlse.EUNSTABLE, str(err)
            assert torch.equal(x, before)
            m = re.search(r"exceeds the bound ([-+0-9.eE]+)", str(err))
            bound = float(m.group(1))
            break
    else:
        pytest.fail("the bound never fell below dt")
    ref = sv.invariants(x, energy=False)[2]
    assert bound == pytest.approx(ref, rel=1e-13)
    assert bound < 0.98 * dt0


def test_refusal_stops_every_step_until_checked():
    sv, psi, Vd, dtmax = _solver((70, 128), "fp32", 800, dt_frac=1.5)
    x = _dev(psi, "fp32")
    x0 = x.clone()
    sv.run(x, 5)                                    # refused on the device
    sv.rk4_step(x)                                  # no check of its own, still refused
    sv.run(x, 40)
    torch.cuda.synchronize()
    assert torch.equal(x, x0)
    with pytest.raises(nlse.NLSEError) as ei:
        sv.check()
    assert ei.value.code == nlse.EUNSTABLE
    sv.rk4_step(x)                                  # cleared: steps again
    sv.check()
    assert not torch.equal(x, x0)


def test_nonfinite_state_is_refused_at_entry():
    sv, psi, Vd, _ = _solver((70, 128), "fp32", 810)
    psi = psi.copy()
    psi[30, 40] = np.nan
    x = _dev(psi, "fp32")
    x0 = x.clone()
    sv.run(x, 4)
    with pytest.raises(nlse.NLSEError) as ei:
        sv.check()
    assert ei.value.code == nlse.ENONFINITE and "entry check" in str(ei.value)
    assert torch.equal(x.isnan(), x0.isnan()) and torch.equal(torch.nan_to_num(x), torch.nan_to_num(x0))


def test_run_host_and_adjoint_report_a_pending_refusal():
    sv, psi, Vd, _ = _solver((70, 128), "fp32", 820, dt_frac=1.5)
    host = _dev(psi, "fp32").cpu().pin_memory()
    h0 = host.clone()
    with pytest.raises(nlse.NLSEError) as ei:
        sv.run_host(host, 3)
    assert ei.value.code == nlse.EUNSTABLE
    assert torch.equal(host, h0)
    sv.check()                                      # run_host cleared it
    x = _dev(psi, "fp32")
    sv.run(x, 2)                                    # refused, not read
    with pytest.raises(nlse.NLSEError) as ei:
        sv.adjoint(x, x, 4, 2)
    assert ei.value.code == nlse.EUNSTABLE
    sv.check()


def test_a_bounded_wait_that_runs_out_is_reported_and_the_context_stays_usable():
    """The failure path of the kernels' bounded mbarrier waits, on purpose: a
    wait on a barrier nothing completes gives up after 20 ms, the status
    carries NLSE_ETIMEOUT, nlse_check reports and clears it, and the context
    keeps working (the GPU is not hung and nothing trapped)."""
    sv, psi, Vd, _ = _solver((70, 128), "fp32", 830)
    nlse.nlse_selftest_timeout(sv.ctx, 20.0)
    with pytest.raises(nlse.NLSEError) as ei:
        sv.check()
    assert ei.value.code == nlse.ETIMEOUT
    sv.check()                                      # cleared
    x, y = _dev(psi, "fp32"), _dev(psi, "fp32")
    sv.run(x, 7)
    sv.check()
    s2, _, _, _ = _solver((70, 128), "fp32", 830)
    s2.run(y, 7)
    s2.check()
    assert torch.equal(x, y)
    with pytest.raises(nlse.NLSEError) as ei:
        nlse.nlse_selftest_timeout(sv.ctx, 5000.0)   # limits above a second are refused
    assert ei.value.code == nlse.EINVAL
