"""Both paths of the FP32 and 16-bit mass sums, through the C ABI (a13 and the global
mass of the stored state, Eq. 12 summed over the lattice).

The fused reductions and the step kernels add FP32 values in split parts whose rounded
part is an exact integer sum; that path assumes every value is below 2 in magnitude. A
thread that meets a larger value sums its values again in FP64. Lattice states never
hold such values in practice, so these tests plant them in one region of the state:
the threads there take the FP64 path, the others the split path, and the totals must
still equal the FP64 sums of what the lattice holds.
"""
import math

import numpy as np
import pytest

from paper_2203_05230_gb300 import lbm_ace as A
from paper_2203_05230_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def fsum(a):
    return math.fsum(np.asarray(a, dtype=np.float64).ravel())


def state_with_large_values(nx, ny, big, seed=0):
    """Equilibrium populations of a smooth field at rest, with phi scaled to `big` in a
    block of rows and columns (so some threads see values of 2 or more)."""
    phi = W.random_smooth_phi(nx, ny, seed=seed)
    phi[ny // 4:ny // 2, nx // 3:nx // 2] *= big
    w = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)
    f = w[:, None, None] * phi[None]
    return f, phi


@pytest.mark.parametrize("variant", [A.KERNEL_QUAD, A.KERNEL_PAIR])
@pytest.mark.parametrize("big", [1.0, 20.0])
def test_fp32_mass_paths(variant, big):
    nx, ny = 136, 44
    f, phi = state_with_large_values(nx, ny, big, seed=3)
    with A.Lattice(nx=nx, ny=ny, precision=A.F32, kernel_variant=variant, velocity_kind=A.VEL_UNIFORM,
                   ux=0.01, uy=0.0) as g:
        assert g.launch_shape()[4] == variant
        g.set_state(f, phi, 1)
        fs, _ = g.get_state()
        if big > 1.0:
            assert np.abs(fs).max() >= 2.0
        assert g.mass() == pytest.approx(fsum(fs.astype(np.float32)), rel=1e-13, abs=0.0)
        g.step(1)
        f1, p1 = g.get_state()
        assert g.step_mass() == pytest.approx(fsum(p1.astype(np.float32)), rel=1e-13, abs=0.0)
        assert g.mass() == pytest.approx(fsum(f1.astype(np.float32)), rel=1e-13, abs=0.0)


@pytest.mark.parametrize("precision", [A.F16DEV, A.BF16DEV])
@pytest.mark.parametrize("big", [1.0, 20.0])
def test_16bit_mass_paths(precision, big):
    nx, ny = 136, 44
    f, phi = state_with_large_values(nx, ny, big, seed=5)
    with A.Lattice(nx=nx, ny=ny, precision=precision, velocity_kind=A.VEL_UNIFORM, ux=0.01, uy=0.0) as g:
        assert g.launch_shape()[4] == A.KERNEL_DEV4
        g.set_state(f, phi, 1)
        fs, _ = g.get_state()
        # the mass is the sum of the stored 16-bit deviations and the FP32 phi plane; the
        # read-back expands g_i + s_i phi per population, equal to it up to the rounding
        # of that expansion
        assert g.mass() == pytest.approx(fsum(fs), rel=1e-6)
        g.step(1)
        _, p1 = g.get_state()
        assert g.step_mass() == pytest.approx(fsum(p1.astype(np.float32)), rel=1e-13, abs=0.0)

