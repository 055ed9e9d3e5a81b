"""A small, fixed run of one workload for profilers (ncu): builds the inputs,
takes a few warm-up steps, then a few more, and exits.

    python -m paper_1109_1027_gb300.profile_case --workload vortex2d --n 2048 --steps 3
    python -m paper_1109_1027_gb300.profile_case --workload ring3d --n 256 --steps 3

Workloads: vortex2d (2D dark vortex), ring3d (3D vortex ring), soliton1d
(1D bright soliton), batch2d (the first --count of the 512 uneven 2D
instances), gradient (the gradient workload's 16 x 512^2 stack: --steps RK4
steps forward and back, checkpoints every 10).  FP32 unless --fp64.
--fuse runs the 2D steps as two launches of two RK4 stages each.
"""
from __future__ import annotations

import argparse

import torch

from . import nlse
from . import workloads as wl


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--workload", default="vortex2d",
                    choices=["vortex2d", "ring3d", "soliton1d", "batch2d", "gradient"])
    ap.add_argument("--n", type=int, default=0, help="points per axis (default: the workload's)")
    ap.add_argument("--count", type=int, default=512, help="batch2d: instances (the first ones of the batch)")
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--fp64", action="store_true")
    ap.add_argument("--fuse", action="store_true", help="2D: two RK4 stages per launch")
    args = ap.parse_args()
    prec = "fp64" if args.fp64 else "fp32"
    rdt, cdt = (torch.float64, torch.complex128) if args.fp64 else (torch.float32, torch.complex64)
    dev = "cuda:0"
    if args.workload == "gradient":
        V, psis, targets, h, a, s = wl.gradient_problem_2d(n=512, batch=16)
        Vd = torch.from_numpy(V).to(dev).to(rdt).contiguous()
        x0 = torch.stack([torch.from_numpy(p_).to(cdt) for p_ in psis]).to(dev).contiguous()
        tg = torch.stack([torch.from_numpy(t_).to(cdt) for t_ in targets]).to(dev).contiguous()
        solver = nlse.Solver(Vd, h, 1e-3, a, s, prec=prec, check_stability=False, stack=len(psis))
        for _ in range(args.warmup):
            solver.adjoint(x0, tg, 2, 1)
        solver.adjoint(x0, tg, args.steps, 10)
        torch.cuda.synchronize()
        print("profile_case: ok")
        return
    if args.workload == "batch2d":
        insts = wl.gaussian_batch_2d(count=512, steps=0, only=set(range(args.count)))
        V = nlse.BatchSolver.pack([q.V for q in insts], rdt, dev)
        x = nlse.BatchSolver.pack([q.psi0 for q in insts], cdt, dev)
        shapes = [q.shape for q in insts]
        probe = nlse.BatchSolver(V, shapes, [q.h for q in insts], 1.0, [q.a for q in insts],
                                 [q.s for q in insts], prec=prec, check_stability=False)
        dts = [0.5 * d for d in probe.invariants(x)[2]]
        probe.close()
        solver = nlse.BatchSolver(V, shapes, [q.h for q in insts], dts, [q.a for q in insts],
                                  [q.s for q in insts], prec=prec, check_stability=False)
    else:
        make = {"vortex2d": wl.dark_vortex_2d, "ring3d": wl.vortex_ring_3d, "soliton1d": wl.bright_soliton_1d}
        inst = make[args.workload](n=args.n, steps=0) if args.n else make[args.workload](steps=0)
        V = torch.from_numpy(inst.V).to(dev).to(rdt).contiguous()
        x = torch.from_numpy(inst.psi0).to(dev).to(cdt).contiguous()
        probe = nlse.Solver(V, inst.h, 1.0, inst.a, inst.s, prec=prec, check_stability=False)
        dt = 0.5 * probe.invariants(x)[2]
        probe.close()
        solver = nlse.Solver(V, inst.h, dt, inst.a, inst.s, prec=prec, check_stability=False)
        if args.fuse:
            solver.set_tiling(nlse.TILE_2D_FUSE, 1)
    for _ in range(args.warmup):
        solver.rk4_step(x)
    for _ in range(args.steps):
        solver.rk4_step(x)
    torch.cuda.synchronize()
    solver.check()
    print("profile_case: ok")


if __name__ == "__main__":
    main()
