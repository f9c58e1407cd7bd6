"""Seeded synthetic inputs shared by the tests, the benchmark and the oracle checks.

This module holds workload recipes only (initial fields, velocity-field draws,
instance lists); none of the lattice Boltzmann method's arithmetic lives here,
so both the CUDA path and the CPU oracle can take their inputs from it.

The single-vortex workload is the paper's benchmark (Section 3, Eq. 14): a disk
of radius R centred at (xc, yc) on a periodic L x L lattice, with a tanh
profile of width parameter eps across its rim, deformed by a time-reversed
vortex of period T steps.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np


def disk_phi0(nx: int, ny: int, xc: float, yc: float, R: float, eps: float) -> np.ndarray:
    """phi0 = 0.5 (1 + tanh((R - r) / (2 eps))) with r the distance from (xc, yc),
    nodes at integer coordinates; float64, shape [ny, nx]."""
    y, x = np.mgrid[0:ny, 0:nx].astype(np.float64)
    r = np.sqrt((x - xc) ** 2 + (y - yc) ** 2)
    return 0.5 * (1.0 + np.tanh((R - r) / (2.0 * eps)))


def slab_phi0(nx: int, ny: int, y_lo: float, y_hi: float, eps: float) -> np.ndarray:
    """A flat slab (phi ~ 1 for y_lo < y < y_hi) with two tanh rims, constant in x."""
    y = np.arange(ny, dtype=np.float64)[:, None] * np.ones((1, nx))
    a = 0.5 * (1.0 + np.tanh((y - y_lo) / (2.0 * eps)))
    b = 0.5 * (1.0 + np.tanh((y_hi - y) / (2.0 * eps)))
    return a + b - 1.0


def random_smooth_phi(nx: int, ny: int, seed: int, n_disks: int = 3, eps: float = 1.0) -> np.ndarray:
    """A few random disks (periodic images included) plus a little noise, in (0, 1)."""
    rng = np.random.default_rng(seed)
    phi = np.zeros((ny, nx))
    y, x = np.mgrid[0:ny, 0:nx].astype(np.float64)
    for _ in range(n_disks):
        xc, yc = rng.uniform(0, nx), rng.uniform(0, ny)
        R = rng.uniform(0.1, 0.3) * min(nx, ny)
        dx = np.minimum(np.abs(x - xc), nx - np.abs(x - xc))
        dy = np.minimum(np.abs(y - yc), ny - np.abs(y - yc))
        r = np.sqrt(dx * dx + dy * dy)
        phi = np.maximum(phi, 0.5 * (1.0 + np.tanh((R - r) / (2.0 * eps))))
    phi += 1e-3 * rng.standard_normal((ny, nx))
    return phi


@dataclass(frozen=True)
class Vortex:
    """Single-vortex run: lattice L x L, disk (xc, yc, R), eps, tau, U0, period T."""
    L: int
    eps: float = 1.0
    tau: float = 0.8
    U0: float = 0.04
    T: int = 2000
    R_frac: float = 0.15
    xc_frac: float = 0.5
    yc_frac: float = 0.75
    sign: float = -1.0  # -1: u = -U0 ..., v = +U0 ... ; +1: the sign printed in Eq. 14

    @property
    def R(self) -> float:
        return self.R_frac * self.L

    @property
    def xc(self) -> float:
        return self.xc_frac * self.L

    @property
    def yc(self) -> float:
        return self.yc_frac * self.L

    def phi0(self) -> np.ndarray:
        return disk_phi0(self.L, self.L, self.xc, self.yc, self.R, self.eps)


# Plain FP64 method: 64^2 lattice, R = 9.6 at (32, 48), eps 1, tau 0.8, U0 0.04, T 2000.
VORTEX_64_F64 = Vortex(L=64, T=2000)


def vortex_fp32(L: int, eps: float = 1.0) -> Vortex:
    """FP32 workloads: L in {1024, 2048} (and 256 for the oracle), T = 16 L steps."""
    return Vortex(L=L, eps=eps, T=16 * L)


# Batched form: 256 instances with sides from this set and seeded parameter draws.
BATCH_SIDES = (128, 192, 256, 384, 512, 768, 1024)


@dataclass(frozen=True)
class Instance:
    L: int
    xc: float
    yc: float
    R: float
    eps: float
    tau: float
    U0: float
    T: int


def batched_instances(count: int = 256, seed: int = 0) -> list:
    """Seeded (PCG64) draws: side from BATCH_SIDES, centre in [0.3, 0.7] L, radius in
    [0.1, 0.2] L, eps in [0.5, 2], tau in [0.6, 1.0], U0 in [0.02, 0.05], T in [8 L, 16 L]."""
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    for _ in range(count):
        L = int(rng.choice(BATCH_SIDES))
        out.append(Instance(
            L=L,
            xc=float(rng.uniform(0.3, 0.7) * L), yc=float(rng.uniform(0.3, 0.7) * L),
            R=float(rng.uniform(0.1, 0.2) * L), eps=float(rng.uniform(0.5, 2.0)),
            tau=float(rng.uniform(0.6, 1.0)), U0=float(rng.uniform(0.02, 0.05)),
            T=int(round(rng.uniform(8 * L, 16 * L)))))
    return out


def stream_function_field(n: int, seed: int, modes: int = 4, umax: float = 0.05):
    """Divergence-free periodic velocity on an n x n lattice from a stream function
    that is a sum of `modes` random sin/cos modes, scaled so max |u| <= umax.
    Returns (u, v) float64 [n, n] with u = d(chi)/dy, v = -d(chi)/dx taken analytically."""
    rng = np.random.default_rng(seed)
    y, x = np.mgrid[0:n, 0:n].astype(np.float64)
    u = np.zeros((n, n))
    v = np.zeros((n, n))
    for _ in range(modes):
        kx, ky = rng.integers(1, 4, size=2)
        a = rng.standard_normal()
        ph = rng.uniform(0, 2 * math.pi)
        arg = 2 * math.pi * (kx * x + ky * y) / n + ph
        # chi = a sin(arg): u = a cos(arg) 2 pi ky / n, v = -a cos(arg) 2 pi kx / n
        u += a * np.cos(arg) * 2 * math.pi * ky / n
        v -= a * np.cos(arg) * 2 * math.pi * kx / n
    scale = umax * rng.uniform(0.3, 1.0) / max(np.sqrt(u * u + v * v).max(), 1e-30)
    return u * scale, v * scale
