"""FP64 CPU oracle for the interface-capturing LB method (TEST INFRASTRUCTURE ONLY).

This package is the plain, slow reference that the CUDA library is checked
against. Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg
of ``bench.py`` may import it; the product path never does. It shares no code
with the CUDA library. The arithmetic lives in ``lbm_ace_oracle.c`` (plain C,
FP64, the paper's own step order); this module only marshals numpy arrays.

Every function here follows H. Liang, "An accurate lattice Boltzmann method for
interface capturing" (arXiv 2203.05230); the readings R1-R8 taken where the
paper is silent or inconsistent are listed at the top of the C file.

State layout: ``f[i, y, x]`` holds f_i(x, t) after streaming (D2Q9 order
c_0=(0,0), c_1..c_4=(1,0),(0,1),(-1,0),(0,-1), c_5..c_8=(1,1),(-1,1),(-1,-1),
(1,-1)); ``phi_prev[y, x]`` holds phi(x, t-1).
"""
from __future__ import annotations

import ctypes
import math
import os
from dataclasses import dataclass, field
from typing import Optional

import numpy as np

from .build import build_oracle

MODIFIED, CONSERVATIVE = 0, 1          # Eq. 8 (the paper's model) / Eq. 1 ablation
VORTEX, UNIFORM, FIELD = 0, 1, 2       # velocity kinds
DELTA = math.exp(-20.0)                # regulariser of Eq. 13

_lib = None


class _Params(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int),
                ("model", ctypes.c_int), ("vel_kind", ctypes.c_int),
                ("tau", ctypes.c_double), ("eps", ctypes.c_double),
                ("delta", ctypes.c_double),
                ("U0", ctypes.c_double), ("T", ctypes.c_double), ("sign", ctypes.c_double),
                ("ux", ctypes.c_double), ("uy", ctypes.c_double),
                ("ufield", ctypes.POINTER(ctypes.c_double)),
                ("vfield", ctypes.POINTER(ctypes.c_double))]


_D = ctypes.POINTER(ctypes.c_double)
_I = ctypes.POINTER(ctypes.c_int)


def lib():
    """Load (building on first use) the oracle's shared object."""
    global _lib
    if _lib is None:
        path = build_oracle()
        L = ctypes.CDLL(path)
        L.oracle_lattice.argtypes = [_D, _I, _I]
        L.oracle_profile.argtypes = [ctypes.c_double, ctypes.c_double]
        L.oracle_profile.restype = ctypes.c_double
        L.oracle_psi.argtypes = [ctypes.c_double, ctypes.c_double, ctypes.c_double]
        L.oracle_psi.restype = ctypes.c_double
        L.oracle_sharpen.argtypes = [ctypes.c_double, ctypes.c_double]
        L.oracle_sharpen.restype = ctypes.c_double
        L.oracle_feq.argtypes = [ctypes.c_double, ctypes.c_double, ctypes.c_double, _D]
        L.oracle_forcing.argtypes = [ctypes.c_double, ctypes.c_double, _D]
        L.oracle_grad.argtypes = [_D, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, _D]
        L.oracle_velocity.argtypes = [ctypes.POINTER(_Params), ctypes.c_int, ctypes.c_int,
                                      ctypes.c_double, _D, _D]
        L.oracle_init.argtypes = [ctypes.POINTER(_Params), _D, _D, _D]
        L.oracle_phi.argtypes = [ctypes.POINTER(_Params), _D, _D]
        L.oracle_mass.argtypes = [ctypes.POINTER(_Params), _D]
        L.oracle_mass.restype = ctypes.c_double
        L.oracle_step.argtypes = [ctypes.POINTER(_Params), _D, _D, ctypes.c_longlong,
                                  ctypes.c_longlong, ctypes.c_int]
        L.oracle_step.restype = ctypes.c_int
        L.oracle_step_cells.argtypes = [ctypes.POINTER(_Params), _D, _D, ctypes.c_longlong,
                                        ctypes.c_int, _I, _I, _D, _D]
        L.oracle_step_cells.restype = ctypes.c_int
        _lib = L
    return _lib


def _dp(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(_D)


def lattice():
    """D2Q9 weights and velocities (after Eq. 10): (w[9], cx[9], cy[9])."""
    w = np.zeros(9)
    cx = np.zeros(9, dtype=np.int32)
    cy = np.zeros(9, dtype=np.int32)
    lib().oracle_lattice(_dp(w), cx.ctypes.data_as(_I), cy.ctypes.data_as(_I))
    return w, cx, cy


def profile(s: float, eps: float) -> float:
    """Eq. 2 (reading R1): equilibrium phi at signed normal distance s."""
    return lib().oracle_profile(s, eps)


def psi(phi: float, eps: float, delta: float = DELTA) -> float:
    """Eq. 13 with the clip: regularised signed distance."""
    return lib().oracle_psi(phi, eps, delta)


def sharpen(psi_: float, eps: float) -> float:
    """Eqs. 6, 11 (reading R1): (1/(4 eps)) [1 - tanh^2(psi/(2 eps))]."""
    return lib().oracle_sharpen(psi_, eps)


def feq(phi: float, u: float, v: float) -> np.ndarray:
    """Eq. 10."""
    out = np.zeros(9)
    lib().oracle_feq(phi, u, v, _dp(out))
    return out


def forcing(gx: float, gy: float) -> np.ndarray:
    """Eq. 11 for a given bracket vector G = d_t(phi u) + c_s^2 S n."""
    out = np.zeros(9)
    lib().oracle_forcing(gx, gy, _dp(out))
    return out


def grad(chi: np.ndarray, x: int, y: int) -> np.ndarray:
    """Isotropic gradient (reading R2) of a periodic [ny, nx] field at (x, y)."""
    chi = np.ascontiguousarray(chi, dtype=np.float64)
    out = np.zeros(2)
    lib().oracle_grad(_dp(chi), chi.shape[1], chi.shape[0], x, y, _dp(out))
    return out


@dataclass
class Params:
    """Problem statement: periodic nx x ny lattice, tau (Eq. 9), eps (R1),
    delta (Eq. 13) and the prescribed velocity."""
    nx: int
    ny: int
    tau: float = 0.8
    eps: float = 1.0
    delta: float = DELTA
    model: int = MODIFIED
    vel_kind: int = VORTEX
    U0: float = 0.04
    T: float = 2000.0
    sign: float = -1.0
    ux: float = 0.0
    uy: float = 0.0
    ufield: Optional[np.ndarray] = None
    vfield: Optional[np.ndarray] = None
    _keep: list = field(default_factory=list, repr=False)

    def c(self) -> _Params:
        p = _Params(self.nx, self.ny, self.model, self.vel_kind, self.tau, self.eps,
                    self.delta, self.U0, self.T, self.sign, self.ux, self.uy, None, None)
        if self.vel_kind == FIELD:
            u = np.ascontiguousarray(self.ufield, dtype=np.float64).reshape(self.ny, self.nx)
            v = np.ascontiguousarray(self.vfield, dtype=np.float64).reshape(self.ny, self.nx)
            self._keep[:] = [u, v]
            p.ufield = _dp(u)
            p.vfield = _dp(v)
        return p


def velocity(p: Params, x: int, y: int, t: float):
    """Prescribed velocity (Eq. 14, readings R4 and R5) at a node."""
    u = ctypes.c_double()
    v = ctypes.c_double()
    cp = p.c()
    lib().oracle_velocity(ctypes.byref(cp), x, y, t, ctypes.byref(u), ctypes.byref(v))
    return u.value, v.value


class Sim:
    """State (f, phi_prev, t) of the oracle and its time stepping."""

    def __init__(self, p: Params, phi0: Optional[np.ndarray] = None):
        self.p = p
        n = p.nx * p.ny
        self.f = np.zeros((9, p.ny, p.nx))
        self.phi_prev = np.zeros((p.ny, p.nx))
        self.t = 0
        if phi0 is not None:
            phi0 = np.ascontiguousarray(phi0, dtype=np.float64).reshape(p.ny, p.nx)
            cp = p.c()
            lib().oracle_init(ctypes.byref(cp), _dp(phi0), _dp(self.f), _dp(self.phi_prev))
        assert self.f.size == 9 * n

    @classmethod
    def from_state(cls, p: Params, f: np.ndarray, phi_prev: np.ndarray, t: int) -> "Sim":
        s = cls(p)
        s.f[...] = f.reshape(9, p.ny, p.nx)
        s.phi_prev[...] = phi_prev.reshape(p.ny, p.nx)
        s.t = int(t)
        return s

    def copy(self) -> "Sim":
        return Sim.from_state(self.p, self.f.copy(), self.phi_prev.copy(), self.t)

    def step(self, n: int = 1, threads: int = 1) -> "Sim":
        cp = self.p.c()
        rc = lib().oracle_step(ctypes.byref(cp), _dp(self.f), _dp(self.phi_prev),
                               self.t, n, threads)
        if rc != 0:
            raise MemoryError("oracle_step: out of host memory")
        self.t += n
        return self

    def phi(self) -> np.ndarray:
        out = np.zeros((self.p.ny, self.p.nx))
        cp = self.p.c()
        lib().oracle_phi(ctypes.byref(cp), _dp(self.f), _dp(out))
        return out

    def mass(self) -> float:
        cp = self.p.c()
        return lib().oracle_mass(ctypes.byref(cp), _dp(self.f))

    def step_cells(self, xs, ys):
        """One step at sampled nodes only: returns (f(t+1) [n, 9], phi(t) [n])."""
        xs = np.ascontiguousarray(xs, dtype=np.int32)
        ys = np.ascontiguousarray(ys, dtype=np.int32)
        fn = np.zeros((len(xs), 9))
        ph = np.zeros(len(xs))
        cp = self.p.c()
        rc = lib().oracle_step_cells(ctypes.byref(cp), _dp(self.f), _dp(self.phi_prev), self.t,
                                     len(xs), xs.ctypes.data_as(_I), ys.ctypes.data_as(_I),
                                     _dp(fn), _dp(ph))
        if rc != 0:
            raise ValueError("oracle_step_cells: node outside the lattice")
        return fn, ph


def threads_available() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:  # pragma: no cover
        return os.cpu_count() or 1
