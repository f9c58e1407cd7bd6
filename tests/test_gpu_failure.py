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


def _small_forward_case():
    """A 16 x 20 image with the fixed parameters the smoke check uses (scaled output
    layer so the increment is not negligible), and the oracle's emulated result."""
    import oracle.surrogate as S
    from paper_2203_05230_gb300 import workloads as W
    flat = np.asarray(W.surrogate_init_params(seed=0), dtype=np.float32)
    flat[-289:] *= 20.0
    rng = np.random.default_rng(0)
    phi = W.circles_phi0(20, np.random.Generator(np.random.PCG64(1)))[:16].astype(np.float32)
    u, v = rng.uniform(-0.05, 0.05, (2, 16, 20)).astype(np.float32)
    ref, _ = S.forward(flat.astype(np.float64), phi, u, v, emulate=True)
    return flat, phi, u, v, ref[0]


@pytest.mark.parametrize("limit", [1, 2_000_000])
def test_surrogate_bounded_wait_gives_up_and_the_net_survives(limit):
    """The tensor-core kernels' bounded mbarrier wait, run on a barrier nothing arrives
    on, gives up; the net reports LBM_ACE_ETIMEOUT once, and its forward pass then
    matches the oracle exactly as before the failure."""
    torch = pytest.importorskip("torch")
    flat, phi, u, v, ref = _small_forward_case()
    dev = {k: torch.tensor(a[None], device="cuda") for k, a in (("phi", phi), ("u", u), ("v", v))}
    with A.Net(0, torch.cuda.current_stream()) as net:
        net.set_params(flat)
        outs = []
        for fail in (False, True):
            if fail:
                with pytest.raises(A.LbmAceError) as e:
                    net.wait_selftest(limit)
                assert e.value.status == A.ETIMEOUT
                net.synchronize()  # the report cleared the flag
            out = torch.empty_like(dev["phi"])
            net.forward(dev["phi"], dev["u"], dev["v"], out, 1, 16, 20)
            net.synchronize()
            outs.append(out.cpu().numpy()[0].astype(np.float64))
    assert np.array_equal(outs[0], outs[1])
    inc = np.linalg.norm(outs[1] - ref) / np.linalg.norm(ref - phi)
    assert inc < 2e-3, inc


def test_surrogate_wait_selftest_rejects_a_bad_limit():
    torch = pytest.importorskip("torch")
    with A.Net(0, torch.cuda.current_stream()) as net:
        for bad in (0, -1, 2_000_000_001):
            with pytest.raises(A.LbmAceError) as e:
                net.wait_selftest(bad)
            assert e.value.status == A.EINVAL
