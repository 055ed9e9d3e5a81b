"""The batched path (nlse_create_batch): many uneven 2D instances advanced by
one launch per RK4 stage must give, for every instance, what the single-grid
path gives for it alone (which the parity suite pins to the oracle), and the
oracle directly on small instances.

Tolerance: FP64 1e-12 and FP32 1e-6 relative to max|psi| after 40 steps.  The
batched and single-grid kernels run the same per-point arithmetic, so the
difference is at most a few rounding steps."""
import numpy as np
import pytest
import torch

import oracle
from paper_1109_1027_gb300 import nlse
from paper_1109_1027_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

DEV = "cuda:0"


def _batch(sides, seed=7):
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    for i, (ny, nx) in enumerate(sides):
        x, y = wl.mesh((ny, nx), -8.0, 8.0)
        w = rng.uniform(0.02, 0.1)
        V = w * w * (x * x + y * y)
        width = rng.uniform(1.0, 3.0)
        psi = np.exp(-(x * x + y * y) / (2 * width ** 2)) * np.exp(1j * (rng.uniform(-1, 1) * x + rng.uniform(-1, 1) * y))
        psi = psi + 0.05 * wl.random_field((ny, nx), seed=seed + i)
        h = wl.spacing(nx, -8.0, 8.0)
        a = float(rng.uniform(0.3, 1.0))
        s = float(rng.choice([-1.0, 1.0]))
        out.append(dict(shape=(ny, nx), V=V, psi=psi, h=h, a=a, s=s))
    return out


SIDES = [(64, 64), (40, 68), (128, 128), (96, 192), (70, 260), (33, 64), (200, 320), (17, 132), (256, 256), (3, 4)]


def _dts(insts, prec):
    dts = []
    for q in insts:
        prob = oracle.Problem(q["shape"], q["h"], q["a"], q["s"])
        psi = q["psi"].astype(np.complex64).astype(np.complex128) if prec == "fp32" else q["psi"]
        V = q["V"].astype(np.float32).astype(np.float64) if prec == "fp32" else q["V"]
        dts.append(0.5 * oracle.invariants(prob, psi, V)[2])
    return dts


@pytest.mark.parametrize("prec,lap", [("fp32", "2shoc"), ("fp64", "2shoc"), ("fp32", "2shoc_ms"), ("fp64", "2shoc_ms")])
def test_batch_equals_single_grid_runs(prec, lap):
    insts = _batch(SIDES)
    cdt, rdt = (torch.complex64, torch.float32) if prec == "fp32" else (torch.complex128, torch.float64)
    dts = _dts(insts, prec)
    V = nlse.BatchSolver.pack([q["V"] for q in insts], rdt, DEV)
    bs = nlse.BatchSolver(V, [q["shape"] for q in insts], [q["h"] for q in insts], dts,
                          [q["a"] for q in insts], [q["s"] for q in insts], prec=prec, lap=lap)
    psi = nlse.BatchSolver.pack([q["psi"] for q in insts], cdt, DEV)
    bs.run(psi, 40)
    bs.check()
    got = [g.cpu().numpy() for g in bs.unpack(psi)]
    for i, q in enumerate(insts):
        Vi = torch.from_numpy(q["V"]).to(DEV).to(rdt).contiguous()
        sv = nlse.Solver(Vi, q["h"], dts[i], q["a"], q["s"], prec=prec, lap=lap)
        x = torch.from_numpy(q["psi"]).to(DEV).to(cdt).contiguous()
        sv.run(x, 40)
        ref = x.cpu().numpy()
        tol = (1e-12 if prec == "fp64" else 1e-6) * np.abs(ref).max()
        assert np.abs(got[i] - ref).max() <= tol, (i, q["shape"])


@pytest.mark.parametrize("prec,lap", [("fp32", "2shoc"), ("fp64", "2shoc"), ("fp64", "2shoc_ms")])
def test_batch_matches_oracle_on_small_instances(prec, lap):
    insts = _batch([(64, 64), (40, 68), (33, 64), (17, 132)], seed=11)
    cdt, rdt = (torch.complex64, torch.float32) if prec == "fp32" else (torch.complex128, torch.float64)
    dts = _dts(insts, prec)
    V = nlse.BatchSolver.pack([q["V"] for q in insts], rdt, DEV)
    bs = nlse.BatchSolver(V, [q["shape"] for q in insts], [q["h"] for q in insts], dts,
                          [q["a"] for q in insts], [q["s"] for q in insts], prec=prec, lap=lap)
    psi = nlse.BatchSolver.pack([q["psi"] for q in insts], cdt, DEV)
    bs.run(psi, 10)
    for i, (g, q) in enumerate(zip(bs.unpack(psi), insts)):
        r = lambda a_, dt_: a_.astype(dt_).astype(np.complex128 if np.iscomplexobj(a_) else np.float64)
        p0 = r(q["psi"], np.complex64) if prec == "fp32" else q["psi"]
        V0 = r(q["V"], np.float32) if prec == "fp32" else q["V"]
        olap = oracle.LAP_2SHOC_MS if lap == "2shoc_ms" else oracle.LAP_2SHOC
        ref = oracle.run(oracle.Problem(q["shape"], q["h"], q["a"], q["s"], lap=olap), p0, V0, dts[i], 10)
        tol = (1e-12 if prec == "fp64" else 1e-5) * np.abs(ref).max()
        assert np.abs(g.cpu().numpy() - ref).max() <= tol, i


def test_batch_laplacian_and_invariants():
    insts = _batch(SIDES, seed=3)
    V = nlse.BatchSolver.pack([q["V"] for q in insts], torch.float64, DEV)
    bs = nlse.BatchSolver(V, [q["shape"] for q in insts], [q["h"] for q in insts], 1e-4,
                          [q["a"] for q in insts], [q["s"] for q in insts], prec="fp64")
    psi = nlse.BatchSolver.pack([q["psi"] for q in insts], torch.complex128, DEV)
    lap = [l.cpu().numpy() for l in bs.unpack(bs.lap2shoc(psi))]
    m, e, d = bs.invariants(psi)
    for i, q in enumerate(insts):
        prob = oracle.Problem(q["shape"], q["h"], q["a"], q["s"])
        ref = oracle.laplacian(prob, q["psi"], q["V"])
        assert np.abs(lap[i] - ref).max() <= 1e-12 * np.abs(ref).max() * 16, i
        m0, e0, d0 = oracle.invariants(prob, q["psi"], q["V"])
        assert m[i] == pytest.approx(m0, rel=1e-12)
        assert e[i] == pytest.approx(e0, rel=1e-11, abs=1e-12)
        assert d[i] == pytest.approx(d0, rel=1e-12)
    m2, e2, d2 = bs.invariants(psi, energy=False)
    assert (m2, d2) == (m, d) and e2 is None


def test_batch_refuses_an_unstable_instance():
    insts = _batch([(64, 64), (128, 128), (40, 68)], seed=5)
    dts = _dts(insts, "fp64")
    dts[1] *= 3.0                                   # 1.5x its bound
    V = nlse.BatchSolver.pack([q["V"] for q in insts], torch.float64, DEV)
    bs = nlse.BatchSolver(V, [q["shape"] for q in insts], [q["h"] for q in insts], dts,
                          [q["a"] for q in insts], [q["s"] for q in insts], prec="fp64")
    psi = nlse.BatchSolver.pack([q["psi"] for q in insts], torch.complex128, DEV)
    psi0 = psi.clone()
    bs.run(psi, 5)                                  # the check runs on the device
    with pytest.raises(nlse.NLSEError) as ei:
        bs.check()
    assert ei.value.code == nlse.EUNSTABLE and "instance 1" in str(ei.value)
    assert torch.equal(psi, psi0)                   # no instance was stepped


def test_batch_workload_sample_equals_single_grid():
    """The 512-instance batch workload (sides 64..1024) at full size, in the
    launch configuration the benchmark times: 3 steps of the whole batch;
    sampled instances compared with their single-grid runs and with the FP64
    oracle (FP32 inputs, relative L2 <= 1e-5).  The sampled instances' dt is
    the oracle's bound; the others take the library's."""
    insts = wl.gaussian_batch_2d(count=512, steps=0)
    sample = [0, 1, 17, 100, 255, 256, 400, 511]
    r32 = lambda z: z.astype(np.complex64).astype(np.complex128) if np.iscomplexobj(z) \
        else z.astype(np.float32).astype(np.float64)
    Vf = nlse.BatchSolver.pack([q.V for q in insts], torch.float32, DEV)
    probe = nlse.BatchSolver(Vf, [q.shape for q in insts], [q.h for q in insts], 1e-9,
                             [q.a for q in insts], [q.s for q in insts], prec="fp32", check_stability=False)
    psi = nlse.BatchSolver.pack([q.psi0 for q in insts], torch.complex64, DEV)
    _, _, dtmax = probe.invariants(psi)
    probe.close()
    dts = [0.5 * d for d in dtmax]
    probs = {i: oracle.Problem(insts[i].shape, insts[i].h, insts[i].a, insts[i].s) for i in sample}
    for i in sample:
        dts[i] = 0.5 * oracle.invariants(probs[i], r32(insts[i].psi0), r32(insts[i].V))[2]
    bs = nlse.BatchSolver(Vf, [q.shape for q in insts], [q.h for q in insts], dts,
                          [q.a for q in insts], [q.s for q in insts], prec="fp32")
    bs.run(psi, 3)
    bs.check()
    out = bs.unpack(psi)
    for i in sample:
        q = insts[i]
        sv = nlse.Solver(torch.from_numpy(q.V).to(DEV).float().contiguous(), q.h, dts[i], q.a, q.s)
        x = torch.from_numpy(q.psi0).to(DEV).to(torch.complex64).contiguous()
        sv.run(x, 3)
        diff = (out[i] - x).abs().max().item()
        assert diff <= 1e-6 * x.abs().max().item(), (i, q.shape, diff)
        ref = oracle.run(probs[i], r32(q.psi0), r32(q.V), dts[i], 3)
        got = out[i].cpu().numpy().astype(np.complex128)
        err = np.linalg.norm(got - ref) / np.linalg.norm(ref)
        assert err <= 1e-5, (i, q.shape, err)


def test_batch_tiling_variants_give_identical_results():
    insts = _batch(SIDES, seed=13)
    dts = _dts(insts, "fp32")
    V = nlse.BatchSolver.pack([q["V"] for q in insts], torch.float32, DEV)
    bs = nlse.BatchSolver(V, [q["shape"] for q in insts], [q["h"] for q in insts], dts,
                          [q["a"] for q in insts], [q["s"] for q in insts], prec="fp32")
    outs = []
    for narrow in (0, 64, 192, 1024):
        bs.set_tiling(nlse.TILE_BATCH_NARROW, narrow)
        assert bs.get_tiling(nlse.TILE_BATCH_NARROW) == narrow
        psi = nlse.BatchSolver.pack([q["psi"] for q in insts], torch.complex64, DEV)
        bs.run(psi, 20)
        outs.append(psi)
    for o in outs[1:]:
        assert torch.equal(o, outs[0])


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_batch_invariants_equal_the_single_grid_ones(prec):
    """The one-launch batch reduction covers each instance with the blocks a
    single-grid launch uses, so mass, energy and dt_max agree bit for bit."""
    insts = _batch(SIDES, seed=9)
    cdt, rdt = (torch.complex64, torch.float32) if prec == "fp32" else (torch.complex128, torch.float64)
    V = nlse.BatchSolver.pack([q["V"] for q in insts], rdt, DEV)
    bs = nlse.BatchSolver(V, [q["shape"] for q in insts], [q["h"] for q in insts], 1e-4,
                          [q["a"] for q in insts], [q["s"] for q in insts], prec=prec)
    psi = nlse.BatchSolver.pack([q["psi"] for q in insts], cdt, DEV)
    m, e, d = bs.invariants(psi)
    for i, q in enumerate(insts):
        sv = nlse.Solver(torch.from_numpy(q["V"]).to(DEV).to(rdt).contiguous(), q["h"], 1e-4, q["a"], q["s"],
                         prec=prec)
        mi, ei, di = sv.invariants(torch.from_numpy(q["psi"]).to(DEV).to(cdt).contiguous())
        assert (m[i], e[i], d[i]) == (mi, ei, di), (i, q["shape"])


@pytest.mark.parametrize("prec,check", [("fp32", True), ("fp32", False), ("fp64", True)])
def test_batch_run_host_equals_a_device_run(prec, check):
    """nlse_run_host of a batch moves the state in chunks of instances whose
    copies overlap the other chunks' steps; the result is the bits of
    nlse_run on the device, for 1, 2 and 33 steps."""
    sides = [(64, 64), (130, 256), (40, 68), (96, 128), (200, 200), (64, 64), (33, 132), (128, 384), (70, 100),
             (256, 256), (48, 64)]
    insts = _batch(sides, seed=31)
    rdt, cdt = (torch.float32, torch.complex64) if prec == "fp32" else (torch.float64, torch.complex128)
    dts = _dts(insts, prec)
    V = nlse.BatchSolver.pack([q["V"] for q in insts], rdt, DEV)
    bs = nlse.BatchSolver(V, [q["shape"] for q in insts], [q["h"] for q in insts], dts,
                          [q["a"] for q in insts], [q["s"] for q in insts], prec=prec, check_stability=check)
    for steps in (1, 2, 33):
        x = nlse.BatchSolver.pack([q["psi"] for q in insts], cdt, DEV)
        bs.run(x, steps)
        bs.check()
        host = nlse.BatchSolver.pack([q["psi"] for q in insts], cdt, "cpu").pin_memory()
        bs.run_host(host, steps)
        assert torch.equal(host, x.cpu()), steps


def test_batch_run_host_refuses_chunk_by_chunk():
    """A refusal of the entry check inside a pipelined host run leaves the
    refused instance's chunk unchanged and is returned."""
    sides = [(64, 64)] * 6 + [(128, 128)] * 6
    insts = _batch(sides, seed=33)
    dts = _dts(insts, "fp64")
    dts[9] *= 3.0                                   # 1.5x its bound
    V = nlse.BatchSolver.pack([q["V"] for q in insts], torch.float64, DEV)
    bs = nlse.BatchSolver(V, [q["shape"] for q in insts], [q["h"] for q in insts], dts,
                          [q["a"] for q in insts], [q["s"] for q in insts], prec="fp64")
    host = nlse.BatchSolver.pack([q["psi"] for q in insts], torch.complex128, "cpu").pin_memory()
    h0 = host.clone()
    with pytest.raises(nlse.NLSEError) as ei:
        bs.run_host(host, 4)
    assert ei.value.code == nlse.EUNSTABLE and "instance 9" in str(ei.value)
    parts0, parts = bs.unpack(h0), bs.unpack(host)
    assert torch.equal(parts[9], parts0[9])         # the refused instance is not stepped
    assert not torch.equal(parts[0], parts0[0])     # an instance of an earlier chunk is
    bs.check()                                      # run_host cleared the status
