"""Python binding of libnlse (include/nlse.h): argument marshalling only.

Every step of the numerical method runs in the CUDA library; this module
checks tensors, hands their device pointers and the current torch stream to
the C ABI and turns status codes into exceptions.  PyTorch is used for device
memory and streams, nothing else.  There is no CPU fallback: if the library is
missing or cannot be loaded, every call raises.

The functions ``nlse_create``, ``nlse_lap2shoc``, ``nlse_rk4_step``,
``nlse_run``, ``nlse_invariants``, ``nlse_reset_compensation``, ``nlse_check``
and ``nlse_destroy`` mirror the C entry points one to one; :class:`Solver`
wraps them for convenience.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np
import torch

from . import build as _build

OK, EINVAL, ENOMEM, ECUDA, EUNSTABLE, ENONFINITE, ETIMEOUT, EUNSUPPORTED, EBOUNDS = range(9)
BC = {"dirichlet": 0, "msd": 1, "periodic": 2, "lapzero": 3}
PREC = {"fp32": 0, "fp64": 1}
LAP = {"2shoc": 0, "cd": 1, "2shoc_ms": 2}
FLAG_NO_STABILITY_CHECK = 1
FLAG_PLAIN_SCHEDULE = 2
FLAG_STACK = 4
TILE_ROWS, TILE_PLANES, TILE_BATCH_NARROW, TILE_1D_RESIDENT, TILE_2D_FUSE, TILE_ADJ_ROWS = 1, 2, 3, 4, 5, 6

_STATUS_NAMES = ["NLSE_OK", "NLSE_EINVAL", "NLSE_ENOMEM", "NLSE_ECUDA", "NLSE_EUNSTABLE",
                 "NLSE_ENONFINITE", "NLSE_ETIMEOUT", "NLSE_EUNSUPPORTED", "NLSE_EBOUNDS"]


class NLSEError(RuntimeError):
    def __init__(self, code: int, msg: str):
        name = _STATUS_NAMES[code] if 0 <= code < len(_STATUS_NAMES) else str(code)
        super().__init__(f"{name}: {msg}")
        self.code = code


class Params(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int), ("n", ctypes.c_int64 * 3), ("h", ctypes.c_double),
                ("dt", ctypes.c_double), ("a", ctypes.c_double), ("s", ctypes.c_double),
                ("bc", ctypes.c_int), ("prec", ctypes.c_int), ("lap", ctypes.c_int),
                ("flags", ctypes.c_uint)]


_lib = None


def library_path() -> str:
    return _build.LIB


def load_library(build_if_missing: bool = True) -> ctypes.CDLL:
    """Loads libnlse.so (building it first when it is absent or stale)."""
    global _lib
    if _lib is not None:
        return _lib
    override = os.environ.get("NLSE_LIBRARY")       # e.g. the bounds-check build (build.build(checked=True))
    if override:
        path = override
    else:
        path = _build.build() if build_if_missing else _build.LIB
    if not os.path.exists(path):
        raise RuntimeError(f"libnlse.so not found at {path}; build it with "
                           "paper_1109_1027_gb300.build.build()")
    lib = ctypes.CDLL(path)
    vp, i64, dp = ctypes.c_void_p, ctypes.c_int64, ctypes.POINTER(ctypes.c_double)
    sig = {
        "nlse_create": ([ctypes.POINTER(Params), vp, ctypes.POINTER(vp)], ctypes.c_int),
        "nlse_destroy": ([vp], None),
        "nlse_lap2shoc": ([vp, vp, vp, vp], ctypes.c_int),
        "nlse_rk4_step": ([vp, vp, vp], ctypes.c_int),
        "nlse_run": ([vp, vp, i64, vp], ctypes.c_int),
        "nlse_run_host": ([vp, vp, i64, vp], ctypes.c_int),
        "nlse_invariants": ([vp, vp, dp, dp, dp, vp], ctypes.c_int),
        "nlse_reset_compensation": ([vp, vp], ctypes.c_int),
        "nlse_check": ([vp, vp], ctypes.c_int),
        "nlse_last_error": ([], ctypes.c_char_p),
        "nlse_invariants_noalloc": ([ctypes.POINTER(Params), vp, vp, dp, dp, dp, vp], ctypes.c_int),
        "nlse_create_batch": ([ctypes.c_int, ctypes.POINTER(Params), vp, ctypes.POINTER(vp)], ctypes.c_int),
        "nlse_invariants_batch": ([vp, vp, dp, dp, dp, vp], ctypes.c_int),
        "nlse_batch_count": ([vp], ctypes.c_int),
        "nlse_adjoint": ([vp, vp, vp, i64, i64, vp, vp, dp, vp], ctypes.c_int),
        "nlse_adjoint_forward": ([vp, vp, vp, i64, i64, dp, vp], ctypes.c_int),
        "nlse_adjoint_backward": ([vp, ctypes.c_double, vp, vp, vp], ctypes.c_int),
        "nlse_set_tiling": ([vp, ctypes.c_int, ctypes.c_int], ctypes.c_int),
        "nlse_get_tiling": ([vp, ctypes.c_int, ctypes.POINTER(ctypes.c_int)], ctypes.c_int),
        "nlse_measure_fp64_rate": ([dp, vp], ctypes.c_int),
        "nlse_selftest_timeout": ([vp, ctypes.c_double, vp], ctypes.c_int),
    }
    for name, (args, res) in sig.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = res
    _lib = lib
    return lib


def _raise(rc: int):
    if rc != OK:
        raise NLSEError(rc, load_library().nlse_last_error().decode(errors="replace"))


def _stream(stream) -> ctypes.c_void_p:
    if stream is None:
        stream = torch.cuda.current_stream()
    if isinstance(stream, torch.cuda.Stream):
        return ctypes.c_void_p(stream.cuda_stream)
    return ctypes.c_void_p(int(stream))


def make_params(shape, h, dt, a, s, bc="dirichlet", prec="fp32", lap="2shoc",
                check_stability=True, plain=False) -> Params:
    """Params for a grid of ``shape`` = (nx,), (ny, nx) or (nz, ny, nx) (x fastest)."""
    p = Params()
    p.dim = len(shape)
    n = list(reversed([int(v) for v in shape])) + [1] * (3 - len(shape))
    for i in range(3):
        p.n[i] = n[i]
    p.h, p.dt, p.a, p.s = float(h), float(dt), float(a), float(s)
    p.bc = BC[bc] if isinstance(bc, str) else int(bc)
    p.prec = PREC[prec] if isinstance(prec, str) else int(prec)
    p.lap = LAP[lap] if isinstance(lap, str) else int(lap)
    p.flags = (0 if check_stability else FLAG_NO_STABILITY_CHECK) | (FLAG_PLAIN_SCHEDULE if plain else 0)
    return p


def nlse_create(params: Params, V_ptr: int) -> ctypes.c_void_p:
    ctx = ctypes.c_void_p()
    _raise(load_library().nlse_create(ctypes.byref(params), ctypes.c_void_p(V_ptr),
                                      ctypes.byref(ctx)))
    return ctx


def nlse_create_batch(params_list, V_ptr: int) -> ctypes.c_void_p:
    arr = (Params * len(params_list))(*params_list)
    ctx = ctypes.c_void_p()
    _raise(load_library().nlse_create_batch(len(params_list), arr, ctypes.c_void_p(V_ptr), ctypes.byref(ctx)))
    return ctx


def nlse_invariants_batch(ctx, psi_ptr: int, count: int, stream=None, energy: bool = True):
    m, e, d = (ctypes.c_double * count)(), (ctypes.c_double * count)(), (ctypes.c_double * count)()
    _raise(load_library().nlse_invariants_batch(ctx, ctypes.c_void_p(psi_ptr), m, e if energy else None, d,
                                                _stream(stream)))
    return list(m), (list(e) if energy else None), list(d)


def nlse_batch_count(ctx) -> int:
    return load_library().nlse_batch_count(ctx)


def nlse_destroy(ctx) -> None:
    load_library().nlse_destroy(ctx)


def nlse_lap2shoc(ctx, psi_ptr: int, lap_ptr: int, stream=None) -> None:
    _raise(load_library().nlse_lap2shoc(ctx, ctypes.c_void_p(psi_ptr), ctypes.c_void_p(lap_ptr),
                                        _stream(stream)))


def nlse_rk4_step(ctx, psi_ptr: int, stream=None) -> None:
    _raise(load_library().nlse_rk4_step(ctx, ctypes.c_void_p(psi_ptr), _stream(stream)))


def nlse_run(ctx, psi_ptr: int, nsteps: int, stream=None) -> None:
    _raise(load_library().nlse_run(ctx, ctypes.c_void_p(psi_ptr), int(nsteps), _stream(stream)))


def nlse_run_host(ctx, host_ptr: int, nsteps: int, stream=None) -> None:
    _raise(load_library().nlse_run_host(ctx, ctypes.c_void_p(host_ptr), int(nsteps), _stream(stream)))


def _check_host(t: torch.Tensor, dtype, numel: int):
    if t.is_cuda or t.dtype != dtype or not t.is_contiguous() or t.numel() != numel:
        raise ValueError(f"expected a contiguous host tensor of {numel} {dtype}")


def nlse_invariants(ctx, psi_ptr: int, stream=None, energy: bool = True):
    """(mass, energy, dt_max); energy=False skips the energy sum and returns None for it."""
    m, e, d = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    _raise(load_library().nlse_invariants(ctx, ctypes.c_void_p(psi_ptr), ctypes.byref(m),
                                          ctypes.byref(e) if energy else None, ctypes.byref(d), _stream(stream)))
    return m.value, (e.value if energy else None), d.value


def nlse_invariants_noalloc(params: Params, psi_ptr: int, V_ptr: int, stream=None):
    """(mass, energy, dt_max) without a context: for callers that cannot
    allocate device memory; the library's static scratch is used instead."""
    m, e, d = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    _raise(load_library().nlse_invariants_noalloc(ctypes.byref(params), ctypes.c_void_p(psi_ptr),
                                                  ctypes.c_void_p(V_ptr), ctypes.byref(m),
                                                  ctypes.byref(e), ctypes.byref(d), _stream(stream)))
    return m.value, e.value, d.value


def nlse_adjoint(ctx, psi0_ptr: int, target_ptr: int, nsteps: int, ckpt_every: int, dpsi0_ptr: int,
                 dV_ptr: int, stream=None) -> float:
    loss = ctypes.c_double()
    _raise(load_library().nlse_adjoint(ctx, ctypes.c_void_p(psi0_ptr), ctypes.c_void_p(target_ptr), int(nsteps),
                                       int(ckpt_every), ctypes.c_void_p(dpsi0_ptr), ctypes.c_void_p(dV_ptr),
                                       ctypes.byref(loss), _stream(stream)))
    return loss.value


def nlse_adjoint_forward(ctx, psi0_ptr: int, target_ptr: int, nsteps: int, ckpt_every: int, stream=None) -> float:
    loss = ctypes.c_double()
    _raise(load_library().nlse_adjoint_forward(ctx, ctypes.c_void_p(psi0_ptr), ctypes.c_void_p(target_ptr),
                                               int(nsteps), int(ckpt_every), ctypes.byref(loss), _stream(stream)))
    return loss.value


def nlse_adjoint_backward(ctx, dloss: float, dpsi0_ptr: int, dV_ptr: int, stream=None) -> None:
    _raise(load_library().nlse_adjoint_backward(ctx, float(dloss), ctypes.c_void_p(dpsi0_ptr),
                                                ctypes.c_void_p(dV_ptr), _stream(stream)))


def nlse_measure_fp64_rate(stream=None) -> float:
    """FP64 flops per second of the current GPU (a chain-of-FMAs probe)."""
    r = ctypes.c_double()
    _raise(load_library().nlse_measure_fp64_rate(ctypes.byref(r), _stream(stream)))
    return r.value


def nlse_set_tiling(ctx, key: int, value: int) -> None:
    _raise(load_library().nlse_set_tiling(ctx, int(key), int(value)))


def nlse_get_tiling(ctx, key: int) -> int:
    v = ctypes.c_int()
    _raise(load_library().nlse_get_tiling(ctx, int(key), ctypes.byref(v)))
    return v.value


def nlse_reset_compensation(ctx, stream=None) -> None:
    _raise(load_library().nlse_reset_compensation(ctx, _stream(stream)))


def nlse_selftest_timeout(ctx, limit_ms: float, stream=None) -> None:
    _raise(load_library().nlse_selftest_timeout(ctx, float(limit_ms), _stream(stream)))


def nlse_check(ctx, stream=None) -> None:
    _raise(load_library().nlse_check(ctx, _stream(stream)))


class Solver:
    """One NLSE problem i psi_t + a Lap psi - V psi + s|psi|^2 psi = 0 on the GPU.

    ``V`` is a CUDA tensor shaped (nx,), (ny, nx) or (nz, ny, nx); float32 for
    ``prec="fp32"`` (state complex64) or float64 for ``prec="fp64"``
    (complex128).  The solver keeps a reference to V.  ``plain=True`` selects
    the paper's unfused schedule (a baseline).  ``stack=n`` (2D, n >= 1) makes
    the state a stack of n instances of V's grid, shape (n, ny, nx), that share
    V and advance together (NLSE_FLAG_STACK)."""

    def __init__(self, V: torch.Tensor, h: float, dt: float, a: float, s: float,
                 bc: str = "dirichlet", prec: str = "fp32", lap: str = "2shoc",
                 check_stability: bool = True, plain: bool = False, stack: int = 0):
        load_library()
        want = torch.float32 if prec == "fp32" else torch.float64
        if not V.is_cuda or V.dtype != want or not V.is_contiguous():
            raise ValueError(f"V must be a contiguous CUDA {want} tensor")
        self.V = V
        self.shape = tuple(V.shape)
        self.prec = prec
        self.cdtype = torch.complex64 if prec == "fp32" else torch.complex128
        self.params = make_params(self.shape, h, dt, a, s, bc, prec, lap, check_stability, plain)
        if stack:
            if V.dim() != 2:
                raise ValueError("stacks are of 2D grids")
            self.params.n[2] = int(stack)
            self.params.flags |= FLAG_STACK
            self.shape = (int(stack),) + self.shape
        with torch.cuda.device(V.device):
            self.ctx = nlse_create(self.params, V.data_ptr())

    def _check_psi(self, psi: torch.Tensor):
        if (not psi.is_cuda or psi.dtype != self.cdtype or tuple(psi.shape) != self.shape
                or not psi.is_contiguous() or psi.device != self.V.device):
            raise ValueError(f"psi must be a contiguous {self.cdtype} tensor of shape {self.shape} "
                             f"on {self.V.device}")

    def lap2shoc(self, psi: torch.Tensor, out: torch.Tensor | None = None) -> torch.Tensor:
        self._check_psi(psi)
        out = torch.empty_like(psi) if out is None else out
        self._check_psi(out)
        nlse_lap2shoc(self.ctx, psi.data_ptr(), out.data_ptr())
        return out

    def rk4_step(self, psi: torch.Tensor) -> torch.Tensor:
        self._check_psi(psi)
        nlse_rk4_step(self.ctx, psi.data_ptr())
        return psi

    def run(self, psi: torch.Tensor, nsteps: int) -> torch.Tensor:
        self._check_psi(psi)
        nlse_run(self.ctx, psi.data_ptr(), nsteps)
        return psi

    def run_host(self, psi_host: torch.Tensor, nsteps: int) -> torch.Tensor:
        """nsteps steps of a state held in (preferably pinned) host memory, in place."""
        _check_host(psi_host, self.cdtype, int(np.prod(self.shape)))
        nlse_run_host(self.ctx, psi_host.data_ptr(), nsteps)
        return psi_host

    def invariants(self, psi: torch.Tensor, energy: bool = True):
        """(mass, energy, dt_max) in FP64 (energy None when not asked for)."""
        self._check_psi(psi)
        return nlse_invariants(self.ctx, psi.data_ptr(), energy=energy)

    def adjoint(self, psi0: torch.Tensor, target: torch.Tensor, nsteps: int, ckpt_every: int = 100):
        """(loss, dL/dpsi0, dL/dV) of L = sum |Psi_T - target|^2 after nsteps
        steps from psi0; dL/dpsi0 has psi0's dtype (d/dRe + i d/dIm), dL/dV is
        float64."""
        self._check_psi(psi0)
        self._check_psi(target)
        g_psi = torch.empty_like(psi0)
        g_V = torch.empty(tuple(self.V.shape), dtype=torch.float64, device=psi0.device)
        loss = nlse_adjoint(self.ctx, psi0.data_ptr(), target.data_ptr(), nsteps, ckpt_every,
                            g_psi.data_ptr(), g_V.data_ptr())
        return loss, g_psi, g_V

    def adjoint_forward(self, psi0: torch.Tensor, target: torch.Tensor, nsteps: int, ckpt_every: int = 100) -> float:
        """The loss L = sum |Psi_T - target|^2, keeping the checkpoints for one
        later adjoint_backward."""
        self._check_psi(psi0)
        self._check_psi(target)
        return nlse_adjoint_forward(self.ctx, psi0.data_ptr(), target.data_ptr(), nsteps, ckpt_every)

    def adjoint_backward(self, dloss: float = 1.0):
        """(d(dloss L)/dpsi0, d(dloss L)/dV) of the held forward pass."""
        g_psi = torch.empty(self.shape, dtype=self.cdtype, device=self.V.device)
        g_V = torch.empty(tuple(self.V.shape), dtype=torch.float64, device=self.V.device)
        nlse_adjoint_backward(self.ctx, dloss, g_psi.data_ptr(), g_V.data_ptr())
        return g_psi, g_V

    def reset_compensation(self):
        nlse_reset_compensation(self.ctx)

    def check(self):
        nlse_check(self.ctx)

    def set_tiling(self, key: int, value: int):
        nlse_set_tiling(self.ctx, key, value)

    def get_tiling(self, key: int) -> int:
        return nlse_get_tiling(self.ctx, key)

    def close(self):
        if getattr(self, "ctx", None):
            nlse_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class BatchSolver:
    """Many independent 2D instances advanced together (nlse_create_batch).

    ``shapes`` lists each instance's (ny, nx); ``h``, ``dt``, ``a``, ``s`` are
    scalars or per-instance sequences.  ``V`` is the flat potential: the
    instances' arrays raveled and concatenated in order (see :meth:`pack`).
    Psi is the same kind of flat complex tensor."""

    def __init__(self, V: torch.Tensor, shapes, h, dt, a, s, prec: str = "fp32", lap: str = "2shoc",
                 check_stability: bool = True):
        load_library()
        want = torch.float32 if prec == "fp32" else torch.float64
        if not V.is_cuda or V.dtype != want or not V.is_contiguous() or V.dim() != 1:
            raise ValueError(f"V must be a flat contiguous CUDA {want} tensor")
        self.shapes = [tuple(int(v) for v in sh) for sh in shapes]
        n = len(self.shapes)
        self.sizes = [sh[0] * sh[1] for sh in self.shapes]
        self.offsets = [sum(self.sizes[:i]) for i in range(n)]
        if V.numel() != sum(self.sizes):
            raise ValueError("V has the wrong number of points for these shapes")
        per = lambda v: [float(x) for x in v] if hasattr(v, "__len__") else [float(v)] * n
        hs, dts, as_, ss = per(h), per(dt), per(a), per(s)
        self.params = [make_params(self.shapes[i], hs[i], dts[i], as_[i], ss[i], "dirichlet", prec, lap,
                                   check_stability) for i in range(n)]
        self.V = V
        self.count = n
        self.cdtype = torch.complex64 if prec == "fp32" else torch.complex128
        with torch.cuda.device(V.device):
            self.ctx = nlse_create_batch(self.params, V.data_ptr())

    @staticmethod
    def pack(arrays, dtype, device):
        """Flat tensor of the arrays raveled and concatenated in order."""
        return torch.cat([torch.as_tensor(a).reshape(-1) for a in arrays]).to(device=device, dtype=dtype).contiguous()

    def unpack(self, flat: torch.Tensor):
        """Views of a flat tensor as the instances' (ny, nx) grids."""
        return [flat[o:o + z].view(sh) for o, z, sh in zip(self.offsets, self.sizes, self.shapes)]

    def _check_psi(self, psi):
        if (not psi.is_cuda or psi.dtype != self.cdtype or psi.dim() != 1 or psi.numel() != sum(self.sizes)
                or not psi.is_contiguous() or psi.device != self.V.device):
            raise ValueError(f"psi must be a flat contiguous {self.cdtype} tensor on {self.V.device}")

    def run(self, psi, nsteps):
        self._check_psi(psi)
        nlse_run(self.ctx, psi.data_ptr(), nsteps)
        return psi

    def run_host(self, psi_host, nsteps):
        """nsteps steps of the flat batch state held in host memory, in place."""
        _check_host(psi_host, self.cdtype, sum(int(np.prod(s_)) for s_ in self.shapes))
        nlse_run_host(self.ctx, psi_host.data_ptr(), nsteps)
        return psi_host

    def rk4_step(self, psi):
        self._check_psi(psi)
        nlse_rk4_step(self.ctx, psi.data_ptr())
        return psi

    def lap2shoc(self, psi, out=None):
        self._check_psi(psi)
        out = torch.empty_like(psi) if out is None else out
        self._check_psi(out)
        nlse_lap2shoc(self.ctx, psi.data_ptr(), out.data_ptr())
        return out

    def invariants(self, psi, energy: bool = True):
        """Per-instance (mass, energy, dt_max) lists, FP64 (energy None when not asked for)."""
        self._check_psi(psi)
        return nlse_invariants_batch(self.ctx, psi.data_ptr(), self.count, energy=energy)

    def set_tiling(self, key: int, value: int):
        nlse_set_tiling(self.ctx, key, value)

    def get_tiling(self, key: int) -> int:
        return nlse_get_tiling(self.ctx, key)

    def reset_compensation(self):
        nlse_reset_compensation(self.ctx)

    def check(self):
        nlse_check(self.ctx)

    def close(self):
        if getattr(self, "ctx", None):
            nlse_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class _FinalLoss(torch.autograd.Function):
    """L = sum |Psi_T(psi0, V) - target|^2 through the CUDA library.  The
    forward call runs the forward pass with its checkpoints
    (nlse_adjoint_forward) and keeps the context; backward runs the reverse
    sweep (nlse_adjoint_backward) with the incoming gradient as the loss's
    weight, so a forward call whose gradient is never asked for pays for the
    forward pass only."""

    @staticmethod
    def forward(ctx, psi0, V, target, h, dt, a, s, nsteps, ckpt_every, lap):
        prec = "fp32" if psi0.dtype == torch.complex64 else "fp64"
        solver = Solver(V.detach().contiguous(), h, dt, a, s, prec=prec, lap=lap, check_stability=False)
        loss = solver.adjoint_forward(psi0.detach().contiguous(), target.detach().contiguous(), nsteps, ckpt_every)
        ctx.solver = solver
        ctx.v_dtype = V.dtype
        return torch.tensor(loss, dtype=torch.float64, device=psi0.device)

    @staticmethod
    def backward(ctx, grad_out):
        solver = ctx.solver
        ctx.solver = None
        g_psi, g_V = solver.adjoint_backward(float(grad_out))
        solver.close()
        return g_psi, g_V.to(ctx.v_dtype), None, None, None, None, None, None, None, None


def final_loss(psi0, V, target, h, dt, a, s, nsteps, ckpt_every=100, lap="2shoc"):
    """Differentiable L = sum |Psi_T - target|^2 (FP64 scalar) of an RK4+2SHOC
    run on a 2D Dirichlet grid; gradients w.r.t. psi0 and V come from the
    library's adjoint (torch.autograd.Function)."""
    return _FinalLoss.apply(psi0, V, target, h, dt, a, s, nsteps, ckpt_every, lap)


def adjoint_many(psi0s, V: torch.Tensor, targets, h, dt, a, s, nsteps: int, ckpt_every: int = 100,
                 lap: str = "2shoc"):
    """Gradients of the summed loss sum_b |Psi_T^b - target_b|^2 for a batch
    of initial states sharing V: one stacked context (NLSE_FLAG_STACK) that
    advances every state in one launch per stage.  Returns (the summed loss,
    [dL/dpsi0_b], dL/dV summed over the batch in FP64 by the library)."""
    prec = "fp32" if psi0s[0].dtype == torch.complex64 else "fp64"
    solver = Solver(V, h, dt, a, s, prec=prec, lap=lap, check_stability=False, stack=len(psi0s))
    x0 = torch.stack(list(psi0s)).contiguous()
    tg = torch.stack(list(targets)).contiguous()
    loss, g_psi, g_V = solver.adjoint(x0, tg, nsteps, ckpt_every)
    solver.close()
    return loss, list(g_psi.unbind(0)), g_V
