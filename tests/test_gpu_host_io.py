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


@pytest.mark.parametrize("precision", [A.F32, A.F64])
@pytest.mark.parametrize("pin", [True, False])
def test_chunked_creation_equals_the_whole_upload(precision, pin):
    """From 2^20 nodes, FP64 and FP32 lattices upload phi0 in row chunks on a second
    stream and initialise each chunk as it lands. The state must equal, bit for bit, the
    one the whole-plane init gives (reached here through a restart at t = 0 from the same
    values, which FP32 holds exactly)."""
    L = 1024
    phi0 = W.random_smooth_phi(L, L, seed=11).astype(np.float32).astype(np.float64)
    keep, src = pinned_like(phi0) if pin else (None, phi0)
    with A.Lattice(nx=L, ny=L, precision=precision, phi0=src, T_period=16384.0) as a, \
         A.Lattice(nx=L, ny=L, precision=precision, T_period=16384.0) as b:
        b.lbm_ace_reset_device(torch.tensor(phi0.astype(np.float32), device="cuda").data_ptr(), 0)
        b.synchronize()
        fa, pa = a.get_state()
        fb, pb = b.get_state()
        assert np.array_equal(fa, fb) and np.array_equal(pa, pb)
        a.step(3)
        b.step(3)
        assert np.array_equal(a.phi(), b.phi())
    del keep


@pytest.mark.parametrize("k", [7, 1024 * 1000 + 5])
def test_chunked_creation_rejects_non_finite_phi0(k):
    phi0 = np.full((1024, 1024), 0.5)
    phi0.flat[k] = np.nan
    phi0.flat[1024 * 1023] = np.inf
    keep, src = pinned_like(phi0)
    with pytest.raises(A.LbmAceError) as e:
        A.Lattice(nx=1024, ny=1024, phi0=src, precision=A.F32)
    assert e.value.status == A.EINVAL and f"phi0[{k}]" in str(e.value)
    with A.Lattice(nx=1024, ny=1024, phi0=np.full((1024, 1024), 0.5), precision=A.F32) as g:
        g.step(2)
        assert g.mass() == pytest.approx(0.5 * 1024 * 1024, rel=1e-6)
    del keep
