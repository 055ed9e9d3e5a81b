"""The CUDA adjoint (nlse_adjoint) against the FP64 reference adjoint of
oracle/adjoint.py (itself pinned by finite differences), against central
finite differences of the GPU forward, and through torch.autograd.

Tolerances: FP64 1e-10 relative to the largest gradient entry (the reverse
sweep sums thousands of rounded terms per entry); FP32 state and cotangents
with FP64 loss and dL/dV accumulation: 2e-4."""
import numpy as np
import pytest
import torch

import oracle
from oracle import adjoint as oadj
from paper_1109_1027_gb300 import nlse
from paper_1109_1027_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

DEV = "cuda:0"


def _problem(shape, seed):
    x, y = wl.mesh(shape, -3.0, 3.0)
    rng = np.random.Generator(np.random.PCG64(seed))
    V = 0.3 * (x * x + y * y) + 0.1 * rng.standard_normal(shape)
    psi0 = np.exp(-(x * x + y * y) / 2.0) * np.exp(1j * (0.7 * x - 0.3 * y)) + 0.05 * wl.random_field(shape, seed)
    target = np.exp(-((x - 0.5) ** 2 + y * y) / 1.5) + 0.05 * wl.random_field(shape, seed + 1)
    h = wl.spacing(shape[1], -3.0, 3.0)
    return psi0, V, target, h


def _close(a, b, tol):
    return np.abs(a - b).max() <= tol * np.abs(b).max()


@pytest.mark.parametrize("shape,lap", [((16, 20), "2shoc"), ((40, 70), "2shoc"), ((33, 130), "2shoc"),
                                       ((24, 36), "cd")])
def test_adjoint_fp64_matches_reference(shape, lap):
    psi0, V, target, h = _problem(shape, 3)
    a, s = 0.6, -1.0
    prob = oracle.Problem(shape, h, a, s, lap=oracle.LAP_CD if lap == "cd" else 0)
    k = 0.5 * oracle.invariants(prob, psi0, V)[2]
    n = 7
    L0, g0, gV0 = oadj.loss_and_gradient(prob, psi0, V, target, k, n)
    solver = nlse.Solver(torch.from_numpy(V).to(DEV), h, k, a, s, prec="fp64", lap=lap, check_stability=False)
    t = lambda z: torch.from_numpy(z).to(DEV).to(torch.complex128).contiguous()
    L, g, gV = solver.adjoint(t(psi0), t(target), n, ckpt_every=3)
    assert L == pytest.approx(L0, rel=1e-12)
    assert _close(g.cpu().numpy(), g0, 1e-10)
    assert _close(gV.cpu().numpy(), gV0, 1e-10)


def test_adjoint_fp32_matches_reference():
    shape = (40, 68)
    psi0, V, target, h = _problem(shape, 9)
    a, s = 0.5, -1.0
    r32 = lambda z: z.astype(np.complex64).astype(np.complex128)
    psi0, target = r32(psi0), r32(target)
    V = V.astype(np.float32).astype(np.float64)
    prob = oracle.Problem(shape, h, a, s)
    k = 0.5 * oracle.invariants(prob, psi0, V)[2]
    n = 12
    L0, g0, gV0 = oadj.loss_and_gradient(prob, psi0, V, target, k, n)
    solver = nlse.Solver(torch.from_numpy(V).to(DEV).float(), h, k, a, s, prec="fp32", check_stability=False)
    t = lambda z: torch.from_numpy(z).to(DEV).to(torch.complex64).contiguous()
    L, g, gV = solver.adjoint(t(psi0), t(target), n, ckpt_every=5)
    assert L == pytest.approx(L0, rel=2e-5)
    assert _close(g.cpu().numpy(), g0, 2e-4)
    assert _close(gV.cpu().numpy(), gV0, 2e-4)


def test_gradient_workload_crop_reference_and_finite_differences():
    """The gradient workload's recipe on a 64 x 64 grid (domain [-16, 16]^2):
    the FP64 GPU gradient equals the FP64 CPU reference gradient, and central
    differences (eps = 1e-4) of the GPU forward along random directions of
    psi0 and V match it."""
    V, psis, targets, h, a, s = wl.gradient_problem_2d(n=64, batch=1)
    psi0, target = psis[0], targets[0]
    prob = oracle.Problem((64, 64), h, a, s)
    k = 0.5 * oracle.invariants(prob, psi0, V)[2]
    n = 30
    L0, g0, gV0 = oadj.loss_and_gradient(prob, psi0, V, target, k, n)
    Vd = torch.from_numpy(V).to(DEV)
    solver = nlse.Solver(Vd, h, k, a, s, prec="fp64", check_stability=False)
    t = lambda z: torch.from_numpy(z).to(DEV).to(torch.complex128).contiguous()
    L, g, gV = solver.adjoint(t(psi0), t(target), n, ckpt_every=10)
    assert L == pytest.approx(L0, rel=1e-12)
    assert _close(g.cpu().numpy(), g0, 1e-10)
    assert _close(gV.cpu().numpy(), gV0, 1e-10)

    def loss_of(p, v):
        sv = nlse.Solver(v, h, k, a, s, prec="fp64", check_stability=False)
        x = p.clone()
        sv.run(x, n)
        return float(((x - t(target)).abs() ** 2).sum())

    eps = 1e-4
    d = t(wl.random_field((64, 64), seed=77))
    fd = (loss_of(t(psi0) + eps * d, Vd) - loss_of(t(psi0) - eps * d, Vd)) / (2 * eps)
    ad = float(torch.real(torch.sum(torch.conj(g) * d)))
    assert ad == pytest.approx(fd, rel=1e-6)
    dv = torch.from_numpy(wl.random_potential((64, 64), seed=78) - 0.5).to(DEV)
    fd = (loss_of(t(psi0), Vd + eps * dv) - loss_of(t(psi0), Vd - eps * dv)) / (2 * eps)
    assert float((gV * dv).sum()) == pytest.approx(fd, rel=1e-6)


def test_autograd_function_gives_the_adjoint_gradients():
    V, psis, targets, h, a, s = wl.gradient_problem_2d(n=64, batch=2)
    prob = oracle.Problem((64, 64), h, a, s)
    k = 0.5 * oracle.invariants(prob, psis[0], V)[2]
    Vt = torch.from_numpy(V).to(DEV).float().requires_grad_(True)
    total = 0.0
    refs = []
    for p, tg in zip(psis, targets):
        p_t = torch.from_numpy(p).to(DEV).to(torch.complex64).requires_grad_(True)
        tg_t = torch.from_numpy(tg).to(DEV).to(torch.complex64)
        loss = nlse.final_loss(p_t, Vt, tg_t, h, k, a, s, nsteps=20, ckpt_every=7)
        loss.backward()
        sv = nlse.Solver(Vt.detach().contiguous(), h, k, a, s, prec="fp32", check_stability=False)
        L, g, gV = sv.adjoint(p_t.detach().contiguous(), tg_t, 20, 7)
        assert loss.item() == pytest.approx(L, rel=1e-12)
        assert torch.allclose(p_t.grad, g)
        refs.append(gV)
        total += L
    assert torch.allclose(Vt.grad.double(), (refs[0] + refs[1]), rtol=1e-5, atol=1e-6 * float(refs[0].abs().max()))


def test_adjoint_many_equals_per_instance_adjoints():
    """adjoint_many runs one stacked context: each dL/dpsi0 equals the
    instance's own adjoint bit for bit, the loss their sum, and dL/dV their
    sum in instance order (added in FP64 by the library)."""
    V, psis, targets, h, a, s = wl.gradient_problem_2d(n=64, batch=4)
    prob = oracle.Problem((64, 64), h, a, s)
    k = 0.5 * oracle.invariants(prob, psis[0], V)[2]
    Vd = torch.from_numpy(V).to(DEV).float().contiguous()
    xs = [torch.from_numpy(p).to(DEV).to(torch.complex64).contiguous() for p in psis]
    ts = [torch.from_numpy(t).to(DEV).to(torch.complex64).contiguous() for t in targets]
    loss, gps, gV = nlse.adjoint_many(xs, Vd, ts, h, k, a, s, 25, 10)
    sv = nlse.Solver(Vd, h, k, a, s, prec="fp32", check_stability=False)
    total, losses = None, []
    for i in range(4):
        L, g, g_V = sv.adjoint(xs[i], ts[i], 25, 10)
        losses.append(L)
        assert torch.equal(g, gps[i]), i
        total = g_V if total is None else total + g_V
    assert torch.equal(total, gV)
    assert loss == pytest.approx(sum(losses), rel=1e-12)


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_adjoint_halves_equal_the_whole(prec):
    """nlse_adjoint_forward then nlse_adjoint_backward(1) give nlse_adjoint's
    bits; a weight on the loss scales the gradients; a reverse sweep needs
    its own forward pass."""
    V, psis, targets, h, a, s = wl.gradient_problem_2d(n=64, batch=1)
    rdt, cdt = (torch.float32, torch.complex64) if prec == "fp32" else (torch.float64, torch.complex128)
    Vd = torch.from_numpy(np.ascontiguousarray(V)).to(DEV).to(rdt).contiguous()
    x0 = torch.from_numpy(psis[0]).to(DEV).to(cdt).contiguous()
    tg = torch.from_numpy(targets[0]).to(DEV).to(cdt).contiguous()
    sv = nlse.Solver(Vd, h, 1e-3, a, s, prec=prec, check_stability=False)
    L, g, gV = sv.adjoint(x0, tg, 23, 5)
    with pytest.raises(nlse.NLSEError) as ei:
        sv.adjoint_backward()                       # nlse_adjoint consumed its own forward pass
    assert ei.value.code == nlse.EINVAL
    L1 = sv.adjoint_forward(x0, tg, 23, 5)
    y = x0.clone()
    sv.run(y, 3)                                    # other calls in between are allowed
    g1, gV1 = sv.adjoint_backward(1.0)
    assert L1 == L and torch.equal(g1, g) and torch.equal(gV1, gV)
    with pytest.raises(nlse.NLSEError):
        sv.adjoint_backward(1.0)                    # one reverse sweep per forward pass
    sv.adjoint_forward(x0, tg, 23, 5)
    g2, gV2 = sv.adjoint_backward(2.5)
    tol = 1e-12 if prec == "fp64" else 1e-5
    assert _close(g2.cpu().numpy(), 2.5 * g.cpu().numpy(), tol)
    assert _close(gV2.cpu().numpy(), 2.5 * gV.cpu().numpy(), tol)


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_stack_adjoint_equals_per_instance_adjoints(prec):
    """A stack's adjoint gives each instance's dL/dpsi0 bit for bit, the loss
    as the sum of the instances' losses and dL/dV as the sum of theirs, added
    in instance order."""
    n = 3
    V, psis, targets, h, a, s = wl.gradient_problem_2d(n=64, batch=n)
    rdt, cdt = (torch.float32, torch.complex64) if prec == "fp32" else (torch.float64, torch.complex128)
    Vd = torch.from_numpy(np.ascontiguousarray(V)).to(DEV).to(rdt).contiguous()
    dt = 1e-3
    st = nlse.Solver(Vd, h, dt, a, s, prec=prec, check_stability=False, stack=n)
    x0 = torch.stack([torch.from_numpy(p).to(DEV).to(cdt) for p in psis]).contiguous()
    tg = torch.stack([torch.from_numpy(t).to(DEV).to(cdt) for t in targets]).contiguous()
    loss, g_psi, g_V = st.adjoint(x0, tg, 30, 7)
    one = nlse.Solver(Vd, h, dt, a, s, prec=prec, check_stability=False)
    losses, gVs = [], []
    for i in range(n):
        li, gi, gVi = one.adjoint(x0[i].contiguous(), tg[i].contiguous(), 30, 7)
        assert torch.equal(gi, g_psi[i]), i
        losses.append(li)
        gVs.append(gVi)
    total = gVs[0]
    for g in gVs[1:]:
        total = total + g
    assert torch.equal(total, g_V)
    assert loss == pytest.approx(sum(losses), rel=1e-12)


@pytest.mark.parametrize("stack", [0, 3])
def test_adjoint_with_two_stages_per_launch(stack):
    """The adjoint's forward pass and checkpoints on the fused schedule (two
    RK4 stages per launch) give the bits of the four-launch schedule: the
    loss, dL/dpsi0 and dL/dV are identical (odd segment lengths included)."""
    V, psis, targets, h, a, s = wl.gradient_problem_2d(n=64, batch=max(stack, 1))
    Vd = torch.from_numpy(np.ascontiguousarray(V)).to(DEV).to(torch.float32).contiguous()
    if stack:
        x0 = torch.stack([torch.from_numpy(p).to(DEV).to(torch.complex64) for p in psis]).contiguous()
        tg = torch.stack([torch.from_numpy(t).to(DEV).to(torch.complex64) for t in targets]).contiguous()
    else:
        x0 = torch.from_numpy(psis[0]).to(DEV).to(torch.complex64).contiguous()
        tg = torch.from_numpy(targets[0]).to(DEV).to(torch.complex64).contiguous()
    sv = nlse.Solver(Vd, h, 1e-3, a, s, prec="fp32", check_stability=False, stack=stack)
    out = []
    for fuse in (0, 1):
        sv.set_tiling(nlse.TILE_2D_FUSE, fuse)
        out.append(sv.adjoint(x0, tg, 31, 7))
    assert out[0][0] == out[1][0]
    assert torch.equal(out[0][1], out[1][1])
    assert torch.equal(out[0][2], out[1][2])


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
@pytest.mark.parametrize("shape,lap,stack", [((37, 68), "2shoc", 0), ((64, 260), "2shoc", 0), ((40, 132), "cd", 0),
                                             ((21, 36), "2shoc", 3), ((19, 516), "2shoc_ms", 0),
                                             ((30, 70), "2shoc", 0)])
def test_adjoint_walk_equals_tile_kernel(prec, shape, lap, stack):
    """The TMA row walk of the reversed stages (8, 16 or 32 rows per CTA)
    gives the shared-memory tile kernel's bits: the loss, dL/dpsi0 and dL/dV
    are identical, with row counts that are not a multiple of the walk's rows,
    column counts that are not a multiple of its 256 columns, stacks, and
    (FP32, 70 columns) rows the walk cannot address, where both keys run the
    tile kernel."""
    psi0, V, target, h = _problem(shape, 5)
    rdt, cdt = (torch.float32, torch.complex64) if prec == "fp32" else (torch.float64, torch.complex128)
    Vd = torch.from_numpy(np.ascontiguousarray(V)).to(DEV).to(rdt).contiguous()
    if stack:
        x0 = torch.stack([torch.from_numpy(psi0 * (1 + 0.1 * i)).to(DEV).to(cdt) for i in range(stack)]).contiguous()
        tg = torch.stack([torch.from_numpy(target * (1 - 0.1 * i)).to(DEV).to(cdt) for i in range(stack)]).contiguous()
    else:
        x0 = torch.from_numpy(psi0).to(DEV).to(cdt).contiguous()
        tg = torch.from_numpy(target).to(DEV).to(cdt).contiguous()
    prob = oracle.Problem(shape, h, 0.6, -1.0, lap={"2shoc": 0, "cd": oracle.LAP_CD, "2shoc_ms": 2}[lap])
    k = 0.5 * oracle.invariants(prob, psi0 * (1 + 0.1 * max(stack - 1, 0)), V)[2]
    sv = nlse.Solver(Vd, h, k, 0.6, -1.0, prec=prec, lap=lap, check_stability=False, stack=stack)
    out = {}
    for rows in (0, 8, 16, 32):
        sv.set_tiling(nlse.TILE_ADJ_ROWS, rows)
        assert sv.get_tiling(nlse.TILE_ADJ_ROWS) == rows
        out[rows] = sv.adjoint(x0, tg, 11, 4)
    ref = out[0]
    assert np.isfinite(ref[0]) and float(ref[1].abs().max()) > 0 and float(ref[2].abs().max()) > 0
    for rows in (8, 16, 32):
        assert out[rows][0] == ref[0], rows
        assert torch.equal(out[rows][1], ref[1]), rows
        assert torch.equal(out[rows][2], ref[2]), rows



@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_gradient_workload_full_size_directional_derivatives(prec):
    """The gradient workload at its full size (16 states of 512 x 512 sharing V,
    one stacked context: the launch configuration the benchmark times), 60
    steps with checkpoints every 20: the adjoint's directional derivatives
    along a random direction of the 16 initial states and of V equal central
    differences of the GPU forward loss in FP64 (eps = 1e-4, rel 1e-6); the
    FP32 gradient equals the FP64 one to 1e-4 of its largest entry."""
    V, psis, targets, h, a, s = wl.gradient_problem_2d(n=512, batch=16)
    rdt, cdt = (torch.float32, torch.complex64) if prec == "fp32" else (torch.float64, torch.complex128)
    probe = nlse.Solver(torch.from_numpy(V).to(DEV), h, 1.0, a, s, prec="fp64", check_stability=False)
    k = 0.5 * min(probe.invariants(torch.from_numpy(p).to(DEV).contiguous())[2] for p in psis)
    probe.close()
    n, ck = 60, 20
    stack = lambda zs, t: torch.stack([torch.from_numpy(z).to(t) for z in zs]).to(DEV).contiguous()
    x0, tg = stack(psis, torch.complex128), stack(targets, torch.complex128)
    V64 = torch.from_numpy(V).to(DEV).contiguous()
    sv64 = nlse.Solver(V64, h, k, a, s, prec="fp64", check_stability=False, stack=16)
    L, g, gV = sv64.adjoint(x0, tg, n, ck)
    if prec == "fp64":
        def loss_of(p, v):
            sv = nlse.Solver(v, h, k, a, s, prec="fp64", check_stability=False, stack=16)
            x = p.clone()
            sv.run(x, n)
            sv.close()
            return float(((x - tg).abs() ** 2).sum())

        eps = 1e-4
        d = stack([wl.random_field((512, 512), seed=500 + i) for i in range(16)], torch.complex128)
        fd = (loss_of(x0 + eps * d, V64) - loss_of(x0 - eps * d, V64)) / (2 * eps)
        assert float(torch.real(torch.sum(torch.conj(g) * d))) == pytest.approx(fd, rel=1e-6)
        dv = torch.from_numpy(wl.random_potential((512, 512), seed=600) - 0.5).to(DEV)
        fd = (loss_of(x0, V64 + eps * dv) - loss_of(x0, V64 - eps * dv)) / (2 * eps)
        assert float((gV * dv).sum()) == pytest.approx(fd, rel=1e-6)
    else:
        sv32 = nlse.Solver(V64.float().contiguous(), h, k, a, s, prec="fp32", check_stability=False, stack=16)
        L32, g32, gV32 = sv32.adjoint(x0.to(cdt), tg.to(cdt), n, ck)
        assert L32 == pytest.approx(L, rel=1e-5)
        assert float((g32.to(torch.complex128) - g).abs().max()) <= 1e-4 * float(g.abs().max())
        assert float((gV32 - gV).abs().max()) <= 1e-4 * float(gV.abs().max())
