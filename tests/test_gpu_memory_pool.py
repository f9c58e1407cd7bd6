"""The contexts' device memory pool and result slots, through the C ABI.

Lattices take their device buffers from a per-device pool that keeps what destroyed
lattices free, and their mapped result blocks from shared pinned pages. A lattice that
reuses another's memory must compute exactly what a lattice on fresh memory computes
(every buffer the step reads is written by init or by the step before), and
lbm_ace_release_cached_memory must hand the cached blocks back to the driver.
"""
import numpy as np
import pytest

from paper_2203_05230_gb300 import lbm_ace as A
from paper_2203_05230_gb300 import workloads as W

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def run(precision, nx, ny, steps, seed):
    phi0 = W.random_smooth_phi(nx, ny, seed=seed)
    with A.Lattice(nx=nx, ny=ny, precision=precision, phi0=phi0, T_period=200.0) as g:
        g.step(steps)
        f, pp = g.get_state()
        return f, pp, g.mass(), g.step_mass()


def test_reused_memory_gives_identical_results():
    A.release_cached_memory(0)
    # fresh memory for every lattice: the pool is empty after the release
    ref = [run(p, 200, 72, 7, seed=k) for k, p in enumerate((A.F32, A.F64, A.BF16DEV, A.F16DEV))]
    A.release_cached_memory(0)
    # a large lattice first, so that the smaller ones reuse its (stale) blocks
    with A.Lattice(nx=512, ny=512, precision=A.F32) as big:
        big.step(3)
    for k, p in enumerate((A.F32, A.F64, A.BF16DEV, A.F16DEV)):
        got = run(p, 200, 72, 7, seed=k)
        for a, b in zip(got, ref[k]):
            assert np.array_equal(a, b)


def test_release_returns_cached_memory_to_the_driver():
    A.release_cached_memory(0)
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info(0)
    with A.Lattice(nx=4096, ny=4096, precision=A.F32) as g:  # 1.2 GB of populations
        g.step(1)
        free_live, _ = torch.cuda.mem_get_info(0)
    free_cached, _ = torch.cuda.mem_get_info(0)
    A.release_cached_memory(0)
    free_released, _ = torch.cuda.mem_get_info(0)
    gb = 1 << 30
    assert free0 - free_live > gb                 # the lattice's buffers
    assert free0 - free_cached > gb               # kept by the pool after destroy
    assert free_released - free_cached > gb       # handed back by the release
    # a lattice created after the release allocates afresh and still works
    with A.Lattice(nx=64, ny=32, precision=A.F32) as g:
        g.step(2)
        assert np.isfinite(g.mass())


def test_many_contexts_share_result_slots():
    """More lattices alive at once than one pinned page has slots (32): each keeps its
    own result block."""
    lats = [A.Lattice(nx=32, ny=16, precision=A.F32, phi0=np.full((16, 32), 0.01 * (k + 1)))
            for k in range(40)]
    try:
        masses = [g.mass() for g in lats]
        for k, m in enumerate(masses):
            assert m == pytest.approx(0.01 * (k + 1) * 32 * 16, rel=1e-6)
    finally:
        for g in lats:
            g.close()


def test_release_rejects_bad_ordinals():
    with pytest.raises(A.LbmAceError):
        A.release_cached_memory(-1)
    with pytest.raises(A.LbmAceError):
        A.release_cached_memory(64)
