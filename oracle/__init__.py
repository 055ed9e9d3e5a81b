"""Plain FP64 CPU oracle for the 2SHOC Laplacian and the RK4 NLSE integrator.

TEST INFRASTRUCTURE ONLY.  The oracle is what the CUDA library is checked
against.  Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg
of ``bench.py`` may import it.  It shares no code with the CUDA library, and
the library never calls it.

The arithmetic lives in ``nlse_oracle.c`` (plain C, double precision, compiled
with ``-ffp-contract=off``); this module only compiles it with gcc and marshals
numpy arrays through ctypes.  Each wrapper names the passage of arXiv 1109.1027
that the C function follows.

Arrays: ``psi`` is complex128 and ``V`` float64, shaped ``(nx,)``, ``(ny, nx)``
or ``(nz, ny, nx)`` (x fastest, as in storage order).  Boundary points are the
first and last index along every axis.
"""
from __future__ import annotations

import ctypes
import hashlib
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "nlse_oracle.c")
_BUILD = os.path.join(_HERE, "_build")

BC_DIRICHLET = 0
BC_MSD = 1
BC_PERIODIC = 2      # n points per axis, spacing h, indices wrap (x_n = x_0)
BC_LAPZERO = 3       # D_b = 0, F_b = i (s|psi_b|^2 - V_b) psi_b
LAP_2SHOC = 0
LAP_CD = 1
LAP_2SHOC_MS = 2     # multi-storage 2SHOC (Eqs. 2d2shocMs1-2, 3d2shocMs1-2); 1D: same as LAP_2SHOC

_libs = {}


def _lib_path(threaded: bool) -> str:
    with open(_SRC, "rb") as f:
        digest = hashlib.sha1(f.read()).hexdigest()[:12]
    return os.path.join(_BUILD, f"libnlse_oracle{'_omp' if threaded else ''}_{digest}.so")


def build(threaded: bool = False) -> str:
    """Compile the oracle (gcc, -O2, no FMA contraction); return the .so path.

    ``threaded`` builds it with -fopenmp: the per-point loops are then shared
    among threads, with the same bits as the serial build (each point's
    arithmetic is unchanged; the reductions stay serial)."""
    path = _lib_path(threaded)
    if not os.path.exists(path):
        os.makedirs(_BUILD, exist_ok=True)
        tmp = path + f".tmp{os.getpid()}"
        flags = ["-fopenmp"] if threaded else ["-Wno-unknown-pragmas"]
        subprocess.check_call(["gcc", "-std=c11", "-O2", "-ffp-contract=off", "-fPIC", "-shared",
                               "-Wall"] + flags + ["-o", tmp, _SRC, "-lm"])
        os.replace(tmp, path)
    return path


def threads_available() -> int:
    """Host cores this process may run on."""
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def _load(threads: int = 1):
    """The serial oracle, or with threads > 1 the OpenMP build set to use that
    many threads (falls back to the serial build where OpenMP is missing)."""
    threaded = threads > 1
    if threaded and "omp" not in _libs:
        try:
            _libs["omp"] = _bind(ctypes.CDLL(build(threaded=True)))
        except (OSError, subprocess.CalledProcessError):
            _libs["omp"] = None
    if threaded and _libs["omp"] is not None:
        _libs["omp"].oracle_set_threads(int(threads))
        return _libs["omp"]
    if "serial" not in _libs:
        _libs["serial"] = _bind(ctypes.CDLL(build()))
    return _libs["serial"]


def threads_used(threads: int) -> int:
    """Threads the oracle actually runs with when asked for ``threads``."""
    lib = _load(threads)
    return int(lib.oracle_set_threads(int(threads) if threads > 1 else 1))


def _bind(lib):
    dp = ctypes.POINTER(ctypes.c_double)
    lp = ctypes.POINTER(ctypes.c_long)
    common = [ctypes.c_int, lp, ctypes.c_double, ctypes.c_double, ctypes.c_double,
              ctypes.c_int, ctypes.c_int]
    lib.oracle_laplacian.argtypes = common + [dp, dp, dp, dp]
    lib.oracle_rhs.argtypes = common + [dp, dp, dp]
    lib.oracle_run.argtypes = common + [ctypes.c_double, ctypes.c_long, dp, dp]
    lib.oracle_invariants.argtypes = common + [dp, dp, dp, dp, dp]
    for fn in (lib.oracle_laplacian, lib.oracle_rhs, lib.oracle_run, lib.oracle_invariants):
        fn.restype = ctypes.c_int
    lib.oracle_set_threads.argtypes = [ctypes.c_int]
    lib.oracle_set_threads.restype = ctypes.c_int
    return lib


@dataclass(frozen=True)
class Problem:
    """Grid and NLSE coefficients: i psi_t + a Lap psi - V psi + s|psi|^2 psi = 0 (Eq. NLSE)."""
    shape: tuple          # (nx,), (ny, nx) or (nz, ny, nx); boundary points included
    h: float
    a: float
    s: float
    bc: int = BC_DIRICHLET
    lap: int = LAP_2SHOC

    @property
    def dim(self) -> int:
        return len(self.shape)

    def _args(self):
        n = (ctypes.c_long * 3)(*([int(v) for v in reversed(self.shape)] + [1] * (3 - self.dim)))
        return [self.dim, n, float(self.h), float(self.a), float(self.s), int(self.bc), int(self.lap)]


def _cplx(psi, shape) -> np.ndarray:
    out = np.ascontiguousarray(psi, dtype=np.complex128)
    if out.shape != tuple(shape):
        raise ValueError(f"psi has shape {out.shape}, expected {tuple(shape)}")
    return out


def _real(V, shape) -> np.ndarray:
    out = np.ascontiguousarray(V, dtype=np.float64)
    if out.shape != tuple(shape):
        raise ValueError(f"V has shape {out.shape}, expected {tuple(shape)}")
    return out


def _dp(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _check(rc: int):
    if rc != 0:
        raise ValueError(f"oracle rejected the problem (code {rc})")


def laplacian(prob: Problem, psi, V, return_D: bool = False):
    """2SHOC Laplacian (Secs. 2.1-2.3, single storage) or CD, boundary = D_b (Sec. 3.2)."""
    psi = _cplx(psi, prob.shape)
    V = _real(V, prob.shape)
    lap = np.empty_like(psi)
    D = np.empty_like(psi)
    _check(_load().oracle_laplacian(*prob._args(), _dp(psi), _dp(V), _dp(lap), _dp(D)))
    return (lap, D) if return_D else lap


def rhs(prob: Problem, psi, V) -> np.ndarray:
    """F(psi) = i[a Lap psi + (s|psi|^2 - V) psi] with the boundary rule (Secs. 3.1, 3.2)."""
    psi = _cplx(psi, prob.shape)
    V = _real(V, prob.shape)
    F = np.empty_like(psi)
    _check(_load().oracle_rhs(*prob._args(), _dp(psi), _dp(V), _dp(F)))
    return F


def run(prob: Problem, psi, V, k: float, nsteps: int, threads: int = 1) -> np.ndarray:
    """nsteps classic RK4 steps of size k, the ten lines of Eq. (RK4); returns a new array.
    ``threads`` > 1 shares each step's per-point loops among host threads
    (the same bits)."""
    out = _cplx(psi, prob.shape).copy()
    V = _real(V, prob.shape)
    _check(_load(threads).oracle_run(*prob._args(), float(k), int(nsteps), _dp(out), _dp(V)))
    return out


def invariants(prob: Problem, psi, V):
    """(mass, energy, dt_max) of the state; dt_max is Eq. (kdfull) with Tables t:bc2, t:sumresults."""
    psi = _cplx(psi, prob.shape)
    V = _real(V, prob.shape)
    m, e, d = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    _check(_load().oracle_invariants(*prob._args(), _dp(psi), _dp(V), ctypes.byref(m),
                                     ctypes.byref(e), ctypes.byref(d)))
    return m.value, e.value, d.value
