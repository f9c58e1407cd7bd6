"""GPU test of lbm_ace_mass_noalloc, the allocation-free global-mass entry point.

Some callers cannot allocate device memory: their memory is already handed out by
their own pool or caching allocator, or their loop cannot take the implicit device
synchronisation of cudaMalloc/cudaFree. They keep the populations in buffers of
their own and ask the library for the compensated global mass, which then keeps its
partial sums in a fixed static device array. This test plays such a caller: it holds
a lattice's populations in device memory it allocated itself, calls the entry point
twice in a row through the C ABI, and checks both results against lbm_ace_mass on
the same populations within the 1e-12 relative bound of the other mass checks. It
also drives the edges of the fixed array (exact multiples of a chunk, more partial
sums than one warp's lanes, the largest count) on values whose sum is known exactly,
and checks that host pointers are refused before any device work.

The file is named so that pytest collects it last.
"""
import math

import numpy as np
import pytest

from paper_2203_05230_gb300 import lbm_ace as A
from paper_2203_05230_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("precision,dtype", [(A.F64, np.float64), (A.F32, np.float32)])
def test_mass_noalloc_matches_mass_on_two_calls(precision, dtype):
    torch = pytest.importorskip("torch")
    L = 300
    phi0 = W.random_smooth_phi(L, L, seed=21)
    with A.Lattice(nx=L, ny=L, precision=precision, phi0=phi0, velocity_kind=A.VEL_UNIFORM,
                   ux=0.02, uy=0.01) as g:
        g.step(17)
        ref = g.mass()
        f, _ = g.get_state()  # the stored values, exactly representable in `dtype`
    dev = torch.device("cuda", 0)
    vals = torch.from_numpy(np.ascontiguousarray(f.astype(dtype))).to(dev)
    out = torch.full((3,), float("nan"), dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream(dev)
    for k in range(2):
        rc = A.lbm_ace_mass_noalloc(vals.data_ptr(), precision, vals.numel(),
                                    out.data_ptr() + 8 * k, stream.cuda_stream)
        assert rc == A.OK
    # a short prefix afterwards: every call starts from its own partials
    n = 70_001
    rc = A.lbm_ace_mass_noalloc(vals.data_ptr(), precision, n, out.data_ptr() + 16, stream.cuda_stream)
    assert rc == A.OK
    torch.cuda.synchronize()
    got = out.cpu().numpy()
    assert got[0] == pytest.approx(ref, rel=1e-12)
    assert got[1] == pytest.approx(ref, rel=1e-12)
    assert got[2] == pytest.approx(math.fsum(f.astype(dtype).ravel()[:n].astype(np.float64)), rel=1e-12)


@pytest.mark.parametrize("count", [2 * A.NOALLOC_CHUNK, 100 * A.NOALLOC_CHUNK + 123, A.NOALLOC_MAX_COUNT])
def test_mass_noalloc_edges_of_the_scratch_array(count):
    """Values k mod 1021 times 2^-10 are exact in FP32 and so are all their partial sums
    in FP64 (at most 2^38 units of 2^-10), so the sum is known exactly from integer
    arithmetic. Counts: an exact multiple of the chunk, more partial sums than the 32
    lanes of the final warp, and the largest count (4096 partial sums, 1 GiB of FP32)."""
    torch = pytest.importorskip("torch")
    dev = torch.device("cuda", 0)
    k = torch.arange(count, dtype=torch.int64, device=dev)
    vals = ((k % 1021).to(torch.float32) * (1.0 / 1024.0)).contiguous()
    del k
    q, r = divmod(count, 1021)
    exact_units = q * (1020 * 1021 // 2) + r * (r - 1) // 2
    expect = exact_units / 1024.0
    out = torch.full((2,), float("nan"), dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream(dev)
    for j in range(2):
        assert A.lbm_ace_mass_noalloc(vals.data_ptr(), A.F32, count, out.data_ptr() + 8 * j,
                                      stream.cuda_stream) == A.OK
    torch.cuda.synchronize()
    got = out.cpu().numpy()
    assert got[0] == expect and got[1] == expect
    del vals
    torch.cuda.empty_cache()


def test_mass_noalloc_rejects_bad_arguments_without_device_work():
    pytest.importorskip("torch")
    import torch
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    vals = torch.zeros(16, dtype=torch.float64, device="cuda")
    assert A.lbm_ace_mass_noalloc(vals.data_ptr(), A.F64, A.NOALLOC_MAX_COUNT + 1, out.data_ptr()) == A.EINVAL
    assert A.lbm_ace_mass_noalloc(vals.data_ptr(), A.F64, -1, out.data_ptr()) == A.EINVAL
    assert A.lbm_ace_mass_noalloc(0, A.F64, 16, out.data_ptr()) == A.EINVAL
    assert A.lbm_ace_mass_noalloc(vals.data_ptr(), A.F64, 16, 0) == A.EINVAL
    assert A.lbm_ace_mass_noalloc(vals.data_ptr(), A.F16DEV, 16, out.data_ptr()) == A.EINVAL
    # host memory, pageable and pinned, for either pointer
    host_vals = np.ones(16)
    host_out = np.zeros(1)
    pinned = torch.zeros(16, dtype=torch.float64).pin_memory()
    assert A.lbm_ace_mass_noalloc(host_vals.ctypes.data, A.F64, 16, out.data_ptr()) == A.EINVAL
    assert A.lbm_ace_mass_noalloc(vals.data_ptr(), A.F64, 16, host_out.ctypes.data) == A.EINVAL
    assert A.lbm_ace_mass_noalloc(pinned.data_ptr(), A.F64, 16, out.data_ptr()) == A.EINVAL
    assert A.lbm_ace_mass_noalloc(vals.data_ptr(), A.F64, 16, pinned.data_ptr()) == A.EINVAL
    assert host_out[0] == 0.0
    torch.cuda.synchronize()
    assert out.item() == 0.0
    # a count of zero writes 0 without reading `values`
    out.fill_(float("nan"))
    assert A.lbm_ace_mass_noalloc(vals.data_ptr(), A.F64, 0, out.data_ptr()) == A.OK
    torch.cuda.synchronize()
    assert out.item() == 0.0
    # the context is still usable: a valid call after all the refusals
    vals.fill_(0.25)
    assert A.lbm_ace_mass_noalloc(vals.data_ptr(), A.F64, 16, out.data_ptr()) == A.OK
    torch.cuda.synchronize()
    assert out.item() == 4.0
