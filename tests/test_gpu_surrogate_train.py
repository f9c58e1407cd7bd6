"""What the trained surrogate gains over the method without it (GPU).

A short training run (the library's own forward, backward and Adam kernels on pairs
that the GPU lattice Boltzmann solver generates, 128^2 tiles) must
  * cut the held-out error of a 16-step prediction far below persistence (the answer
    the method gives without a learned model: phi unchanged over the window) and far
    below the untrained network, and
  * carry the single vortex through half a period by surrogate windows that the
    fallback checks accept, ending much closer to the lattice Boltzmann field than
    persistence does.
"""
import math

import numpy as np
import pytest

from paper_2203_05230_gb300 import lbm_ace as A
from paper_2203_05230_gb300 import surrogate as SG
from paper_2203_05230_gb300 import workloads as W

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def trained():
    s = torch.cuda.current_stream()
    data = SG.generate(n_traj=42, pairs=16, L=128, seed=123, stream=s)
    net = A.Net(0, s)
    net.set_params(W.surrogate_init_params(seed=1))
    tr = SG.Trainer(net, data, batch=8, seed=2)
    n_train = 40 * 16
    test_idx = np.arange(n_train, data.n_pairs)
    before = tr.evaluate(test_idx)
    hist = tr.train(1200, lr_max=2e-3, train_pairs=np.arange(n_train), log_every=100)
    after = tr.evaluate(test_idx)
    yield net, before, after, hist
    net.close()


def test_training_reduces_the_loss(trained):
    _, _, _, hist = trained
    assert hist[-1][1] < 0.05 * hist[0][1]


def test_trained_network_beats_persistence_and_the_untrained_network(trained):
    _, before, after, _ = trained
    assert after["E2_net"] < 0.2 * after["E2_persistence"], after
    assert after["E2_net"] < 0.1 * before["E2_net"], (before, after)
    assert after["increment_rel_err"] < 0.25, after


def test_hybrid_vortex_half_period(trained):
    net = trained[0]
    s = torch.cuda.current_stream()
    L, T = 128, 2048
    v = W.Vortex(L=L, eps=1.0, tau=0.8, U0=0.04, T=T)
    phi0 = v.phi0()
    kw = dict(nx=L, ny=L, tau=0.8, eps=1.0, U0=0.04, T_period=float(T), vortex_sign=-1.0, precision=A.F32,
              phi0=phi0, stream=s)
    half = T // 2
    with A.Lattice(**kw) as ref, A.Lattice(**kw) as hy:
        ref.step(half)
        st = net.hybrid_advance(hy, half // A.NET_K, mass_tol=1e-6, width_tol=0.1)
        p_ref, p_hy = ref.phi(), hy.phi()
        m0 = float(phi0.sum())
        assert hy.t == half
        assert abs(hy.mass() - m0) < 1e-5 * m0

    def e2(a, b):
        return math.sqrt(((a - b) ** 2).sum() / (b ** 2).sum())

    assert st["surrogate_windows"] >= 0.9 * st["windows"], st
    assert e2(p_hy, p_ref) < 0.25 * e2(phi0, p_ref), (e2(p_hy, p_ref), e2(phi0, p_ref))
