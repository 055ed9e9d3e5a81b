"""Seeded synthetic inputs: grids, potentials and initial wavefunctions.

This module holds no arithmetic of the numerical method (no Laplacian, no
right-hand side, no time stepping, no invariants).  It only builds the inputs
that both the CUDA path and the CPU oracle consume, so the two sides are fed
identical bytes.  Every generator is deterministic in its ``seed`` (numpy
PCG64) and works in float64; callers cast once.

Grids are endpoint-inclusive: ``n`` points per axis on ``[lo, hi]`` give
``h = (hi - lo) / (n - 1)`` and boundary points at index 0 and n-1 (the grid
x_i = x_min + h*i of Sec. 2.1 of arXiv 1109.1027; the 25^3 / 97^3 point counts
of Sec. 4.3 fix the endpoint convention).  Arrays are shaped ``(nx,)``,
``(ny, nx)`` or ``(nz, ny, nx)``: x is the fastest (contiguous) axis.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np


def axis(n: int, lo: float, hi: float) -> np.ndarray:
    return lo + (hi - lo) / (n - 1) * np.arange(n, dtype=np.float64)


def spacing(n: int, lo: float, hi: float) -> float:
    return (hi - lo) / (n - 1)


def mesh(shape, lo: float, hi: float):
    """Coordinate arrays (x, y, z as needed) for a cube domain [lo, hi]^d."""
    axes = [axis(n, lo, hi) for n in reversed(shape)]          # x first
    grids = np.meshgrid(*reversed(axes), indexing="ij")         # slowest axis first
    return tuple(reversed(grids))                               # (x, y, z)


def random_field(shape, seed: int, amp: float = 1.0) -> np.ndarray:
    """Unit-variance complex Gaussian field (real and imaginary parts N(0, amp^2))."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return amp * (rng.standard_normal(shape) + 1j * rng.standard_normal(shape))


def random_potential(shape, seed: int, scale: float = 1.0) -> np.ndarray:
    rng = np.random.Generator(np.random.PCG64(seed))
    return scale * rng.uniform(0.0, 1.0, shape)


@dataclass
class Instance:
    """One NLSE problem i psi_t + a Lap psi - V psi + s|psi|^2 psi = 0 on a grid."""
    name: str
    shape: tuple
    lo: float
    hi: float
    a: float
    s: float
    V: np.ndarray
    psi0: np.ndarray
    bc: int = 0                  # 0 Dirichlet, 1 MSD
    steps: int = 0
    meta: dict = field(default_factory=dict)

    @property
    def h(self) -> float:
        return spacing(self.shape[-1], self.lo, self.hi)

    @property
    def dim(self) -> int:
        return len(self.shape)


def bright_soliton_1d(n: int = 2048, lo: float = -40.0, hi: float = 40.0, x0: float = -10.0,
                      c: float = 0.5, steps: int = 2000) -> Instance:
    """1D bright soliton: a = s = 1, V = 0, psi0 = sqrt(2) sech(x - x0) exp(i c x)."""
    x = axis(n, lo, hi)
    psi0 = np.sqrt(2.0) / np.cosh(x - x0) * np.exp(1j * c * x)
    return Instance("bright_soliton_1d", (n,), lo, hi, 1.0, 1.0, np.zeros(n), psi0, 0, steps,
                    {"x0": x0, "c": c})


def dark_vortex_2d(n: int = 2048, lo: float = -60.0, hi: float = 60.0, seed: int = 2,
                   mu: float = 1.0, noise: float = 1e-3, steps: int = 10000) -> Instance:
    """2D dark vortex in a harmonic trap: a = 0.5, s = -1, V = 0.01 r^2.

    psi0 = sqrt(max(mu - V, 0)) * tanh(r) * exp(i theta) + noise, the noise a
    complex Gaussian with standard deviation ``noise`` per component."""
    x, y = mesh((n, n), lo, hi)
    r2 = x * x + y * y
    V = 0.01 * r2
    amp = np.sqrt(np.maximum(mu - V, 0.0)) * np.tanh(np.sqrt(r2))
    psi0 = amp * np.exp(1j * np.arctan2(y, x)) + random_field((n, n), seed, noise)
    return Instance("dark_vortex_2d", (n, n), lo, hi, 0.5, -1.0, V, psi0, 0, steps,
                    {"seed": seed, "mu": mu})


def vortex_ring_3d(n: int = 512, lo: float = -30.0, hi: float = 30.0, seed: int = 3,
                   mu: float = 1.0, radius: float = 8.0, steps: int = 2000) -> Instance:
    """3D vortex ring: a = 0.5, s = -1, V = 0.005 (x^2 + y^2 + 4 z^2).

    Thomas-Fermi amplitude times the phase atan2(z, rho - R) winding once
    around a ring of radius R in the z = 0 plane, centred at a seeded offset
    U(-1, 1) in x and y."""
    rng = np.random.Generator(np.random.PCG64(seed))
    cx, cy = rng.uniform(-1.0, 1.0, 2)
    x, y, z = mesh((n, n, n), lo, hi)
    V = 0.005 * (x * x + y * y + 4.0 * z * z)
    rho = np.sqrt((x - cx) ** 2 + (y - cy) ** 2)
    theta = np.arctan2(z, rho - radius)
    core = np.tanh(np.sqrt((rho - radius) ** 2 + z * z))
    psi0 = np.sqrt(np.maximum(mu - V, 0.0)) * core * np.exp(1j * theta)
    return Instance("vortex_ring_3d", (n, n, n), lo, hi, 0.5, -1.0, V, psi0, 0, steps,
                    {"seed": seed, "centre": (float(cx), float(cy)), "radius": radius})


def gaussian_batch_params(count: int = 512, seed: int = 4, sides=range(64, 1025, 64)):
    """The per-instance draws of gaussian_batch_2d, without building any
    array: a list of dicts with the side n, a, s, w, the Gaussian's width and
    its phase gradient (kx, ky)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    sides = np.asarray(list(sides))
    out = []
    for _ in range(count):
        n = int(rng.choice(sides))
        a = float(rng.uniform(0.3, 1.0))
        s = float(rng.choice([-1.0, 1.0]))
        w = float(rng.uniform(0.0, 0.1))
        width = float(rng.uniform(2.0, 8.0))
        kx, ky = rng.uniform(-1.0, 1.0, 2)
        out.append({"n": n, "a": a, "s": s, "w": w, "width": width, "k": (float(kx), float(ky))})
    return out


def gaussian_batch_2d(count: int = 512, seed: int = 4, sides=range(64, 1025, 64),
                      lo: float = -32.0, hi: float = 32.0, steps: int = 5000, only=None):
    """Independent 2D problems of uneven size: side ~ U(sides), a ~ U[0.3, 1],
    s = +-1, V = w^2 r^2 with w ~ U[0, 0.1], psi0 a Gaussian of width U[2, 8]
    with a random phase gradient (wavenumbers U[-1, 1]).  With ``only`` (a
    set of indices) just those instances are built -- the same ones, since
    every instance's draws are still taken in order -- and returned in order."""
    out = []
    for i, p in enumerate(gaussian_batch_params(count, seed, sides)):
        if only is not None and i not in only:
            continue
        n, w, width = p["n"], p["w"], p["width"]
        kx, ky = p["k"]
        x, y = mesh((n, n), lo, hi)
        V = w * w * (x * x + y * y)
        psi0 = np.exp(-(x * x + y * y) / (2.0 * width * width)) * np.exp(1j * (kx * x + ky * y))
        out.append(Instance(f"gauss_{i}", (n, n), lo, hi, p["a"], p["s"], V, psi0, 0, steps,
                            {"w": w, "width": width, "k": p["k"]}))
    return out


def gradient_problem_2d(n: int = 512, lo: float = -16.0, hi: float = 16.0, seed: int = 5, batch: int = 16,
                        modes: int = 8, steps: int = 3000):
    """Inputs of the final-time-loss gradient problem: a = 0.5, s = -1,
    V = 0.01 r^2 + a smooth seeded perturbation (modes x modes Fourier modes,
    coefficients N(0, 0.02^2) / (1 + |m|^2)), a batch of Gaussian initial
    states (width U[2, 4], centre U(-2, 2)^2, phase gradient U[-1, 1]^2) and
    a batch of Gaussian targets drawn the same way from a second stream.
    Returns (V, [psi0], [target], h, a, s)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    x, y = mesh((n, n), lo, hi)
    L = hi - lo
    V = 0.01 * (x * x + y * y)
    for mx in range(modes):
        for my in range(modes):
            c1, c2 = rng.standard_normal(2) * 0.02 / (1.0 + mx * mx + my * my)
            arg = 2 * np.pi * (mx * (x - lo) + my * (y - lo)) / L
            V = V + c1 * np.cos(arg) + c2 * np.sin(arg)

    def gauss(r):
        w = r.uniform(2.0, 4.0)
        cx, cy = r.uniform(-2.0, 2.0, 2)
        kx, ky = r.uniform(-1.0, 1.0, 2)
        return np.exp(-((x - cx) ** 2 + (y - cy) ** 2) / (2 * w * w)) * np.exp(1j * (kx * x + ky * y))

    psi0 = [gauss(rng) for _ in range(batch)]
    rng2 = np.random.Generator(np.random.PCG64(seed + 1000))
    targets = [gauss(rng2) for _ in range(batch)]
    return V, psi0, targets, spacing(n, lo, hi), 0.5, -1.0
