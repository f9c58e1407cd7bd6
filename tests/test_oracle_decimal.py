"""Whole-step pin of the FP64 oracle against an independent 40-digit computation (CPU).

The per-function pins check each piece of the oracle; this one checks the composed step.
It re-implements the method here in Python's `decimal` arithmetic at 40 significant
digits, from the paper's statement and not from the oracle's code: the moment phi =
sum_i f_i (Eq. 12); the clipped, regularised signed distance psi (Eq. 13, reading R1);
its isotropic gradient (reading R2) and the unit normal (Eq. 13); the sharpening
magnitude (1/(4 eps)) (1 - tanh^2(psi / (2 eps))) (Eqs. 6, 11, R1); the backward
Euler time derivative of phi u, zero at t = 0 (reading R3); the forcing (Eq. 11); the
equilibrium (Eq. 10); the BGK update (Eq. 9) and streaming along c_i; the single-vortex
velocity of Eq. 14 (sign and sampling per readings R4, R5) and the initial state f_eq(phi0,
u(0)) (reading R7). sin, cos, tanh are evaluated from their series and exp at 40 digits,
ln and sqrt by the decimal module.

Three steps on an 8 x 8 periodic lattice, from a smooth field with a few values
outside [0, 1] so the clip acts, must agree with the oracle to 1e-14 of max |f|: the
oracle's FP64 rounding (about 1e-16 per operation) is the only difference left.
"""
import math
from decimal import Decimal, getcontext

import numpy as np
import pytest

import oracle as O

getcontext().prec = 40
D0, D1, D2 = Decimal(0), Decimal(1), Decimal(2)

# D2Q9 (reading R11): c_0 = (0, 0); c_1..4 axis; c_5..8 diagonals; weights after Eq. 10
CX = (0, 1, 0, -1, 0, 1, -1, -1, 1)
CY = (0, 0, 1, 0, -1, 1, 1, -1, -1)
WT = (Decimal(4) / 9,) + (D1 / 9,) * 4 + (D1 / 36,) * 4
CS2 = D1 / 3


def _pi():
    """pi by Machin's formula, 16 x arctan(1/5) - 4 x arctan(1/239), at working precision."""
    def atan_inv(n):
        x = D1 / n
        x2 = x * x
        s, term, k = x, x, 1
        while True:
            term *= -x2
            t = term / (2 * k + 1)
            if abs(t) < Decimal(10) ** (-45):
                return s
            s += t
            k += 1
    return 16 * atan_inv(5) - 4 * atan_inv(239)


PI = _pi()


def dsin(x):
    x = x % (2 * PI)
    s, term, k = x, x, 1
    while abs(term) > Decimal(10) ** (-45):
        term *= -x * x / ((2 * k) * (2 * k + 1))
        s += term
        k += 1
    return s


def dcos(x):
    return dsin(x + PI / 2)


def dtanh(x):
    e = (2 * x).exp()
    return (e - 1) / (e + 1)


def velocity(x, y, t, nx, ny, U0, T, sign):
    """Eq. 14 with the sign factor of reading R5, nodes at integer coordinates (R4)."""
    ct = dcos(PI * t / T)
    sx, sy = dsin(PI * x / nx), dsin(PI * y / ny)
    u = sign * U0 * sx * sx * dsin(2 * PI * y / ny) * ct
    v = -sign * U0 * sy * sy * dsin(2 * PI * x / nx) * ct
    return u, v


def feq(ph, u, v):
    return [WT[i] * ph * (1 + (CX[i] * u + CY[i] * v) / CS2) for i in range(9)]


def dec_init(phi0, vel):
    ny, nx = len(phi0), len(phi0[0])
    f = [[[None] * nx for _ in range(ny)] for _ in range(9)]
    for y in range(ny):
        for x in range(nx):
            u, v = vel(x, y, D0)
            e = feq(phi0[y][x], u, v)
            for i in range(9):
                f[i][y][x] = e[i]
    return f, [row[:] for row in phi0]


def dec_step(f, phi_prev, t, tau, eps, delta, vel, conservative=False):
    ny, nx = len(f[0]), len(f[0][0])
    phi = [[sum(f[i][y][x] for i in range(9)) for x in range(nx)] for y in range(ny)]

    def psi(p):
        pc = min(max(p, D0), D1)
        return eps * ((pc + delta) / (1 - pc + delta)).ln()

    chi = [[phi[y][x] if conservative else psi(phi[y][x]) for x in range(nx)] for y in range(ny)]
    out = [[[None] * nx for _ in range(ny)] for _ in range(9)]
    for y in range(ny):
        for x in range(nx):
            ph = phi[y][x]
            gx = sum(WT[i] * CX[i] * chi[(y + CY[i]) % ny][(x + CX[i]) % nx] for i in range(1, 9)) / CS2
            gy = sum(WT[i] * CY[i] * chi[(y + CY[i]) % ny][(x + CX[i]) % nx] for i in range(1, 9)) / CS2
            norm = (gx * gx + gy * gy).sqrt()
            nxv, nyv = gx / (norm + delta), gy / (norm + delta)
            if conservative:
                S = ph * (1 - ph) / eps
            else:
                th = dtanh(chi[y][x] / (2 * eps))
                S = (1 - th * th) / (4 * eps)
            u, v = vel(x, y, Decimal(t))
            up, vp = vel(x, y, Decimal(t - 1))
            dx = dy = D0
            if t > 0:
                dx = ph * u - phi_prev[y][x] * up
                dy = ph * v - phi_prev[y][x] * vp
            Gx, Gy = dx + CS2 * S * nxv, dy + CS2 * S * nyv
            e = feq(ph, u, v)
            for i in range(9):
                F = WT[i] * (CX[i] * Gx + CY[i] * Gy) / CS2
                fi = f[i][y][x]
                fs = fi - (fi - e[i]) / tau + (1 - 1 / (2 * tau)) * F
                out[i][(y + CY[i]) % ny][(x + CX[i]) % nx] = fs
    return out, phi


def _phi0(n, seed):
    rng = np.random.default_rng(seed)
    y, x = np.mgrid[0:n, 0:n].astype(float)
    p = 0.5 + 0.45 * np.sin(2 * np.pi * x / n + 0.3) * np.cos(2 * np.pi * y / n - 0.2) + 0.05 * rng.standard_normal((n, n))
    p[1, 2], p[5, 6], p[6, 1] = 1.03, -0.02, 1.0005  # a few values the clip acts on
    return p


@pytest.mark.parametrize("model", [O.MODIFIED, O.CONSERVATIVE])
def test_three_whole_steps_match_a_40_digit_computation(model):
    n, steps = 8, 3
    tau, eps, U0, T, sign = 0.8, 1.0, 0.04, 20.0, -1.0
    phi0 = _phi0(n, seed=3 + model)
    Dd = lambda a: Decimal(float(a))  # the oracle's FP64 inputs, exactly
    vel = lambda x, y, t: velocity(Decimal(x), Decimal(y), t, n, n, Dd(U0), Dd(T), Dd(sign))
    f, pp = dec_init([[Dd(v) for v in row] for row in phi0], vel)
    for t in range(steps):
        f, pp = dec_step(f, pp, t, Dd(tau), Dd(eps), Dd(O.DELTA), vel, conservative=model == O.CONSERVATIVE)
    ref = np.array([[[float(v) for v in row] for row in plane] for plane in f])
    ref_pp = np.array([[float(v) for v in row] for row in pp])
    s = O.Sim(O.Params(nx=n, ny=n, tau=tau, eps=eps, U0=U0, T=T, sign=sign, model=model), phi0).step(steps)
    assert np.abs(s.f - ref).max() <= 1e-14 * np.abs(ref).max()
    assert np.abs(s.phi_prev - ref_pp).max() <= 1e-14
    # the check has teeth: the first step alone (t = 0, no time derivative) already
    # differs from three steps by far more than the tolerance
    assert np.abs(s.f - O.Sim(O.Params(nx=n, ny=n, tau=tau, eps=eps, U0=U0, T=T, sign=sign, model=model),
                              phi0).step(1).f).max() > 1e-6


def test_decimal_series_against_libm():
    """The series used above agree with libm to FP64 precision at sample points."""
    for xv in (0.0, 0.3, 1.0, 2.5, -4.0, 7.0):
        x = Decimal(xv)
        assert float(dsin(x)) == pytest.approx(math.sin(xv), abs=1e-16)
        assert float(dcos(x)) == pytest.approx(math.cos(xv), abs=1e-16)
        assert float(dtanh(x)) == pytest.approx(math.tanh(xv), abs=1e-16)
    assert float(PI) == math.pi
