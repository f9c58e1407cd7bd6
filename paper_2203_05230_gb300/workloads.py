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


# Learned surrogate: training trajectories and initial weights.
SURROGATE_TILE = 256          # periodic tiles of 256 x 256 nodes
SURROGATE_K = 16              # LB steps per surrogate application
SURROGATE_WIDTHS = (3, 32, 32, 32, 32, 1)


def circles_phi0(n: int, rng: np.random.Generator, eps: float = 1.0) -> np.ndarray:
    """1-4 disks of radius 0.05-0.2 n at uniform centres on a periodic n x n lattice
    (minimum-image distance), each with the tanh rim of disk_phi0; phi0 is their
    pointwise maximum. float64 [n, n]."""
    y, x = np.mgrid[0:n, 0:n].astype(np.float64)
    phi = np.zeros((n, n))
    for _ in range(int(rng.integers(1, 5))):
        xc, yc = rng.uniform(0, n, size=2)
        R = rng.uniform(0.05, 0.2) * n
        dx = (x - xc + 0.5 * n) % n - 0.5 * n
        dy = (y - yc + 0.5 * n) % n - 0.5 * n
        r = np.sqrt(dx * dx + dy * dy)
        phi = np.maximum(phi, 0.5 * (1.0 + np.tanh((R - r) / (2.0 * eps))))
    return phi


def mode_field(n: int, rng: np.random.Generator, modes: int = 4, umax: float = 0.05):
    """Divergence-free periodic velocity from the stream function
    chi = sum_m a_m sin(2 pi (kx_m x + ky_m y) / n + p_m) with integer wavenumbers
    |kx|, |ky| <= 2 (not both 0), a_m standard normal, p_m uniform; u = d(chi)/dy and
    v = -d(chi)/dx analytically, scaled so that max |(u, v)| is uniform in [0.4, 1] umax.
    float64 [n, n] each."""
    y, x = np.mgrid[0:n, 0:n].astype(np.float64)
    u = np.zeros((n, n))
    v = np.zeros((n, n))
    for _ in range(modes):
        while True:
            kx, ky = (int(k) for k in rng.integers(-2, 3, size=2))
            if kx or ky:
                break
        a = rng.standard_normal()
        p = rng.uniform(0, 2 * math.pi)
        c = a * np.cos(2 * math.pi * (kx * x + ky * y) / n + p) * 2 * math.pi / n
        u += c * ky
        v -= c * kx
    scale = umax * rng.uniform(0.4, 1.0) / max(float(np.sqrt(u * u + v * v).max()), 1e-30)
    return u * scale, v * scale


def surrogate_trajectories(count: int, n: int = SURROGATE_TILE, seed: int = 0):
    """`count` seeded (PCG64) trajectory starts: (phi0, u, v) with 1-4 circles (eps 1)
    in a frozen 4-mode divergence-free field of max speed <= 0.05."""
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    for _ in range(count):
        phi0 = circles_phi0(n, rng)
        u, v = mode_field(n, rng)
        out.append((phi0, u, v))
    return out


def surrogate_init_params(widths=SURROGATE_WIDTHS, seed: int = 0) -> np.ndarray:
    """Initial weights as one flat float64 vector (W_1, b_1, ..., W_L, b_L; each W in
    [co][ci][row offset][column offset] order): normal with standard deviation
    sqrt(2 / (9 ci)) for the GELU layers and 0.1 sqrt(1 / (9 ci)) for the output layer,
    zero biases."""
    rng = np.random.Generator(np.random.PCG64(seed))
    parts = []
    nl = len(widths) - 1
    for l, (ci, co) in enumerate(zip(widths[:-1], widths[1:])):
        sd = math.sqrt(2.0 / (9 * ci)) if l < nl - 1 else 0.1 * math.sqrt(1.0 / (9 * ci))
        parts.append(rng.standard_normal(co * ci * 9) * sd)
        parts.append(np.zeros(co))
    return np.concatenate(parts)
