"""Autotuner for the launch shapes of the streaming kernels.

The tiling keys of nlse_set_tiling change only how the grid is cut into CTAs
(rows per CTA in 2D, z planes per CTA in 3D, which batch instances get
narrow tiles); the arithmetic, and so the result, is the same bit for bit.
`tune` times every candidate on the caller's own problem (a few RK4 steps
through nlse_run, CUDA events), keeps the fastest, and caches the choice in a
JSON file keyed by GPU, dimension, precision, Laplacian and grid shape, so a
later solver for the same problem class reuses it without timing.
"""
from __future__ import annotations

import json
import os

import torch

from . import nlse

CANDIDATES = {
    nlse.TILE_ROWS: (8, 16, 32),
    nlse.TILE_PLANES: (32, 64, 128),
    nlse.TILE_BATCH_NARROW: (0, 64, 128, 192, 256),
    nlse.TILE_1D_RESIDENT: (0, 1, 2, 4, 8, 16),
    nlse.TILE_2D_FUSE: (0, 1),
}


def cache_path() -> str:
    return os.environ.get("NLSE_TILING_CACHE",
                          os.path.join(os.path.expanduser("~"), ".cache", "nlse_gb300_tiling.json"))


def _load():
    try:
        with open(cache_path()) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def _store(table):
    path = cache_path()
    try:
        os.makedirs(os.path.dirname(path), exist_ok=True)
        tmp = path + f".tmp{os.getpid()}"
        with open(tmp, "w") as f:
            json.dump(table, f, indent=1, sort_keys=True)
        os.replace(tmp, path)
    except OSError:
        pass


def _key(solver, tile_key) -> str:
    dev = torch.cuda.get_device_name(solver.V.device)
    p = solver.params if isinstance(solver, nlse.Solver) else solver.params[0]
    if isinstance(solver, nlse.BatchSolver):
        shape = f"batch{solver.count}:{sum(solver.sizes)}"
    else:
        shape = "x".join(str(v) for v in solver.shape)
        if p.flags & nlse.FLAG_STACK:
            shape += f"s{p.n[2]}"
    return f"{dev}|key{tile_key}|dim{p.dim}|prec{p.prec}|lap{p.lap}|{shape}"


def _keys_for(solver):
    if isinstance(solver, nlse.BatchSolver):
        return [nlse.TILE_BATCH_NARROW]
    d = len(solver.shape)
    if d == 1 and solver.shape[0] <= 4096:
        return [nlse.TILE_1D_RESIDENT]
    if d == 2:
        p = solver.params
        if (solver.prec == "fp32" and p.bc == nlse.BC["dirichlet"] and p.lap in (nlse.LAP["2shoc"], nlse.LAP["cd"])
                and not p.flags & nlse.FLAG_PLAIN_SCHEDULE):
            # Rows per CTA first (single-stage launches), then one against two stages per launch.
            return [nlse.TILE_ROWS, nlse.TILE_2D_FUSE]
        return [nlse.TILE_ROWS]
    if d == 3 and solver.prec == "fp32":
        return [nlse.TILE_PLANES]
    return []


def _require_steps_taken(solver):
    """Raises if nlse_run's entry check refused the timed steps (they would
    not have run); a NaN or Inf that the steps themselves produced (a
    collapsing instance of a batch) does not void the timing."""
    try:
        solver.check()
    except nlse.NLSEError as err:
        if err.code == nlse.EUNSTABLE or "entry check" in str(err):
            raise


def tune(solver, psi: torch.Tensor, steps: int = 8, use_cache: bool = True) -> dict:
    """Chooses and sets the fastest tiling for `solver` on state `psi` (which
    is not modified).  Returns {tiling key: {"choice": v, "ms_per_step": {v: ms}}}."""
    table = _load() if use_cache else {}
    report = {}
    for tile_key in _keys_for(solver):
        k = _key(solver, tile_key)
        if use_cache and k in table:
            solver.set_tiling(tile_key, table[k]["choice"])
            report[tile_key] = dict(table[k], cached=True)
            continue
        times = {}
        work = psi.clone()
        for v in CANDIDATES[tile_key]:
            solver.set_tiling(tile_key, v)
            work.copy_(psi)                          # every candidate starts from the caller's state
            solver.reset_compensation()
            solver.run(work, 2)                      # captures the graphs for this tiling
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            solver.run(work, steps)
            e1.record()
            torch.cuda.synchronize()
            _require_steps_taken(solver)
            times[v] = e0.elapsed_time(e1) / steps
        best = min(times, key=times.get)
        solver.set_tiling(tile_key, best)
        entry = {"choice": best, "ms_per_step": {str(v): t for v, t in times.items()}}
        table[k] = entry
        report[tile_key] = entry
    if use_cache and report:
        _store(table)
    return report
