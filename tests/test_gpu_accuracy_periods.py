"""FP32 accuracy over full single-vortex periods (Section 3, Eq. 14), through the C ABI.

The FP32 workloads: radius 0.15 L at (0.5 L, 0.75 L), tau 0.8, U0 0.04, T = 16 L steps,
eps in {0.5, 1, 2}. The FP32 path must stay within 1e-5 phi-L2 of the FP64 reference
after one full period: the FP64 oracle at 256^2, the FP64 GPU path (itself pinned to the
oracle per step at 1e-12) at 1024^2 and 2048^2.

At eps = 0.5 that bound is not reachable by any FP32 computation, and the test below
pins why on the method rather than on the kernel: the FP64 GPU run, with its initial
populations perturbed once by relative noise of FP32's unit roundoff (2^-24), departs by
more than 1e-3 by t = T, four orders of magnitude more than the same perturbation
causes at eps = 1. The FP32 kernel's own error at eps = 0.5 stays within a small factor
of that response.
"""
import math

import numpy as np
import pytest

import oracle as O
from paper_2203_05230_gb300 import lbm_ace as A
from paper_2203_05230_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def e2(a, b):
    return math.sqrt(((a - b) ** 2).sum() / (b ** 2).sum())


def _kw(v):
    return dict(nx=v.L, ny=v.L, tau=v.tau, eps=v.eps, U0=v.U0, T_period=float(v.T), vortex_sign=v.sign,
                phi0=v.phi0())


def _period(v, precision, perturb=None, seed=0):
    with A.Lattice(precision=precision, **_kw(v)) as g:
        if perturb:
            f, pp = g.get_state()
            rng = np.random.default_rng(seed)
            g.set_state(f * (1.0 + perturb * rng.choice([-1.0, 1.0], size=f.shape)), pp, 0)
        m0 = g.mass()
        g.step(v.T)
        return g.phi(), (g.mass() - m0) / m0


@pytest.mark.parametrize("eps", [2.0])  # eps = 1: test_gpu_parity.py
def test_fp32_full_period_256_against_the_oracle(eps):
    v = W.vortex_fp32(256, eps=eps)
    op = O.Params(nx=256, ny=256, tau=v.tau, eps=v.eps, U0=v.U0, T=v.T, sign=v.sign)
    ref = O.Sim(op, v.phi0()).step(v.T, threads=O.threads_available()).phi()
    phi, drift = _period(v, A.F32)
    assert e2(phi, ref) <= 1e-5
    assert abs(drift) <= 1e-5


@pytest.mark.parametrize("L,eps", [(1024, 1.0), (1024, 2.0), (2048, 1.0)])
def test_fp32_full_period_against_the_fp64_gpu_path(L, eps):
    """The full-size FP32 workloads over one period (T = 16384 at 1024^2, 32768 at
    2048^2) against the FP64 GPU path on the same lattice."""
    v = W.vortex_fp32(L, eps=eps)
    p64, d64 = _period(v, A.F64)
    p32, d32 = _period(v, A.F32)
    assert e2(p32, p64) <= 1e-5
    assert abs(d64) <= 1e-12 and abs(d32) <= 1e-5


def test_thin_interface_conditioning_sets_the_fp32_error():
    """eps = 0.5 at 256^2: the method amplifies an FP32-sized perturbation of its initial
    state (FP64 arithmetic throughout) into a phi-L2 departure of order 1e-3 by t = T,
    more than 10^4 times what the same perturbation does at eps = 1 (about 1e-8); the
    FP32 kernel's error there is of that size, not larger."""
    u32 = 2.0 ** -24
    resp, ref = {}, {}
    for eps in (0.5, 1.0):
        v = W.vortex_fp32(256, eps=eps)
        ref[eps], _ = _period(v, A.F64)
        resp[eps] = [e2(_period(v, A.F64, perturb=u32, seed=k)[0], ref[eps]) for k in (1, 2, 3)]
    v = W.vortex_fp32(256, eps=0.5)
    p32, _ = _period(v, A.F32)
    err32 = e2(p32, ref[0.5])
    print(f"eps 0.5: FP32 error {err32:.3e}; FP64 responses to 2^-24 perturbations {resp[0.5]}; "
          f"at eps 1: {resp[1.0]}")
    assert min(resp[0.5]) > 2e-4
    assert min(resp[0.5]) > 1e4 * max(resp[1.0])
    assert err32 <= 10.0 * max(resp[0.5])
