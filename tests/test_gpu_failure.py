"""Failure detection without a GPU fault: a device-side wait that nothing completes gives
up after its limit, the kernel reports that through the context's device error flag,
the host call returns LBM_ACE_ETIMEOUT, and the context keeps working (the lattice
steps on and matches a lattice that never saw the failure)."""
import numpy as np
import pytest

from paper_2203_05230_gb300 import lbm_ace as A

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("limit", [1, 2_000_000])
def test_bounded_wait_gives_up_and_the_context_survives(limit):
    with A.vortex_lattice(64, T=640, precision=A.F32) as g, A.vortex_lattice(64, T=640, precision=A.F32) as h:
        g.step(3)
        with pytest.raises(A.LbmAceError) as e:
            g.lbm_ace_wait_selftest(limit)
        assert e.value.status == A.ETIMEOUT
        g.synchronize()                      # the flag was cleared by the report
        g.step(5)
        h.step(8)
        assert g.t == h.t == 8
        assert np.array_equal(g.phi(), h.phi())
        assert g.mass() == h.mass()


def test_wait_selftest_rejects_a_bad_limit():
    with A.vortex_lattice(32, T=320, precision=A.F32) as g:
        for bad in (0, -5, 4_000_000_001):
            with pytest.raises(A.LbmAceError) as e:
                g.lbm_ace_wait_selftest(bad)
            assert e.value.status == A.EINVAL
