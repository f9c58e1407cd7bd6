"""Host input and output of the C ABI: phi0 and phi in page-locked host memory.

lbm_ace_init uploads a page-locked phi0 without waiting for the copy, and
lbm_ace_get_phi writes a page-locked out through its mapped address; pageable memory
goes through synchronous staging and device buffers. Both routes must give the same
state and the same phi, bit for bit, and the check of phi0 for non-finite values must
hold on both.
"""
import numpy as np
import pytest

from paper_2203_05230_gb300 import lbm_ace as A
from paper_2203_05230_gb300 import workloads as W

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

PRECISIONS = [A.F64, A.F32, A.BF16DEV, A.F16DEV]


def pinned_like(a, offset=0):
    """A page-locked copy of a (FP64), starting `offset` values into its pinned block."""
    buf = torch.empty(a.size + offset + 5, dtype=torch.float64).pin_memory()
    view = buf.numpy()[offset:offset + a.size].reshape(a.shape)
    view[...] = a
    return buf, view


@pytest.mark.parametrize("precision", PRECISIONS)
@pytest.mark.parametrize("nx,ny", [(64, 40), (300, 304)])
def test_pinned_phi0_gives_the_same_state(precision, nx, ny):
    phi0 = W.random_smooth_phi(nx, ny, seed=nx + precision)
    keep, phi0_pinned = pinned_like(phi0, offset=3)
    out = []
    for src in (phi0, phi0_pinned):
        with A.Lattice(nx=nx, ny=ny, precision=precision, phi0=src, T_period=300.0) as g:
            init_phi = g.phi()
            g.step(5)
            out.append((init_phi, *g.get_state(), g.mass()))
    for a, b in zip(*out):
        assert np.array_equal(a, b)
    del keep


@pytest.mark.parametrize("precision", PRECISIONS)
@pytest.mark.parametrize("offset", [0, 3])
def test_pinned_out_gives_the_same_phi(precision, offset):
    nx, ny = 256, 264
    with A.Lattice(nx=nx, ny=ny, precision=precision, phi0=W.random_smooth_phi(nx, ny, seed=7),
                   T_period=300.0) as g:
        g.step(9)
        pageable = g.phi()
        buf = torch.full((nx * ny + offset + 5,), -1.0, dtype=torch.float64).pin_memory()
        view = buf.numpy()[offset:offset + nx * ny].reshape(ny, nx)
        g.phi(view)
        assert np.array_equal(view, pageable)
        # the values around the window are untouched
        whole = buf.numpy()
        assert np.all(whole[:offset] == -1.0) and np.all(whole[offset + nx * ny:] == -1.0)
        # the state read back after the direct write is unchanged by it
        g.step(1)
        assert np.isfinite(g.mass())


@pytest.mark.parametrize("precision", PRECISIONS)
@pytest.mark.parametrize("k", [0, 40321, 300 * 300 - 1])
def test_non_finite_pinned_phi0_is_rejected(precision, k):
    phi0 = np.full((300, 300), 0.5)
    phi0.flat[k] = np.nan if k % 2 == 0 else -np.inf
    phi0.flat[min(k + 11, phi0.size - 1)] = np.nan
    keep, src = pinned_like(phi0)
    with pytest.raises(A.LbmAceError) as e:
        A.Lattice(nx=300, ny=300, phi0=src, precision=precision)
    assert e.value.status == A.EINVAL and f"phi0[{k}]" in str(e.value)
    del keep


@pytest.mark.parametrize("pin", [False, True])
@pytest.mark.parametrize("precision", [A.F32, A.BF16DEV])
def test_phi0_beyond_fp32_range_is_rejected_for_fp32_storage(pin, precision):
    """A value that is finite in FP64 but rounds to infinity in FP32 is rejected by the
    FP32-based forms (here a large field, checked on the device), and accepted by FP64."""
    phi0 = np.full((300, 300), 0.5)
    phi0.flat[1234] = 1e39
    keep, src = pinned_like(phi0) if pin else (None, phi0)
    with pytest.raises(A.LbmAceError) as e:
        A.Lattice(nx=300, ny=300, phi0=src, precision=precision)
    assert e.value.status == A.EINVAL and "phi0[1234] is not finite as FP32" in str(e.value)
    with A.Lattice(nx=300, ny=300, phi0=src, precision=A.F64) as g:
        assert g.lbm_ace_steps_done() == 0
    src.flat[1234] = 3.4028234663852886e38  # FLT_MAX: finite in FP32
    with A.Lattice(nx=300, ny=300, phi0=src, precision=precision) as g:
        assert g.lbm_ace_steps_done() == 0
    del keep
