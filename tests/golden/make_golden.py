"""Writes tests/golden/oracle_vortex64.json from the CPU oracle alone.

The stored numbers are the oracle's own result for the 64^2 FP64 single-vortex
run (disk R = 9.6 at (32, 48), eps 1, tau 0.8, U0 0.04, T 2000, u = -U0...,
v = +U0...): the relative L1 and L2 errors of phi(T) against phi(0) (the
single-vortex benchmark of Section 3) and the relative mass drift. They guard
the oracle against unintended changes; they are not the paper's numbers (it
prints none). Run: python tests/golden/make_golden.py
"""
import json
import math
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import oracle as O  # noqa: E402
from paper_2203_05230_gb300 import workloads as W  # noqa: E402


def vortex64():
    v = W.VORTEX_64_F64
    p = O.Params(nx=v.L, ny=v.L, tau=v.tau, eps=v.eps, U0=v.U0, T=v.T, sign=v.sign)
    phi0 = v.phi0()
    s = O.Sim(p, phi0)
    m0 = s.mass()
    s.step(v.T, threads=O.threads_available())
    phi = s.phi()
    return {
        "config": "64x64 single vortex, FP64, R 9.6 at (32, 48), eps 1, tau 0.8, U0 0.04, T 2000",
        "E1": float(np.abs(phi - phi0).sum() / np.abs(phi0).sum()),
        "E2": float(math.sqrt(((phi - phi0) ** 2).sum() / (phi0 ** 2).sum())),
        "mass_drift_rel": float((s.mass() - m0) / m0),
        "phi_min": float(phi.min()),
        "phi_max": float(phi.max()),
    }


if __name__ == "__main__":
    out = os.path.join(os.path.dirname(os.path.abspath(__file__)), "oracle_vortex64.json")
    with open(out, "w") as fh:
        json.dump(vortex64(), fh, indent=1)
    print(open(out).read())
