"""Batches of single-vortex lattices (persistent kernel, CUDA graph, autotuner).

Every lattice of a batch must evolve exactly as the same lattice would alone: the
batched kernel runs the single-lattice kernels' own tile code (quad32_strip on 128-column
strips when every nx is a multiple of 4, pair_tile on 256-column tiles otherwise); the
only difference is where the phase cos(pi t / T) of Eq. 14 is computed (on the device in
the graph, on the host for single lattices), which can move its last FP32 bit, hence the
1e-6 bound. The tests that take `specs` run both forms: SPECS holds a lattice with
nx = 130, which keeps the batch on column-pair tiles; SPECS_Q has nx = 132 there.
"""
import numpy as np
import pytest

import oracle as O
from paper_2203_05230_gb300 import lbm_ace as A
from paper_2203_05230_gb300 import workloads as W

pytestmark = pytest.mark.gpu

SPECS = [dict(nx=128, ny=128, tau=0.7, eps=0.8, U0=0.03, T_period=1500.0, xc=60.0, yc=70.0, R=20.0),
         dict(nx=192, ny=160, tau=0.9, eps=1.5, U0=0.05, T_period=2200.0, xc=90.0, yc=100.0, R=30.0),
         dict(nx=256, ny=256, tau=0.65, eps=1.0, U0=0.02, T_period=3000.0, xc=120.0, yc=140.0, R=40.0),
         dict(nx=384, ny=96, tau=0.8, eps=2.0, U0=0.04, T_period=3100.0, xc=200.0, yc=50.0, R=25.0),
         dict(nx=130, ny=41, tau=1.0, eps=0.6, U0=0.045, T_period=900.0, xc=60.0, yc=20.0, R=10.0)]
SPECS_Q = SPECS[:4] + [dict(SPECS[4], nx=132)]
FORMS = {"pair": SPECS, "quad": SPECS_Q}


@pytest.fixture(params=["pair", "quad"])
def form(request):
    return request.param


def expected_items(b, specs, form):
    """Work items per step: 128-column strips (quad) or 256-column tiles (pair) of each
    lattice's rows-tall bands."""
    cols = 128 if form == "quad" else 256
    return sum(-(-s["nx"] // cols) * -(-s["ny"] // b.info(i)["rows"]) for i, s in enumerate(specs))


def standalone(spec, steps):
    with A.Lattice(precision=A.F32, velocity_kind=A.VEL_SINGLE_VORTEX, vortex_sign=-1.0, **spec) as g:
        m0 = g.mass()
        g.step(steps)
        return g.phi(), m0, g.mass()


@pytest.mark.parametrize("rows", [0, 8, 33])
def test_batch_lattices_evolve_as_alone(rows, form):
    base = FORMS[form]
    specs = [dict(s, rows_per_cta=rows, vortex_sign=-1.0) for s in base]
    with A.Batch(specs) as b:
        assert b.info(0)["tiles"] == expected_items(b, base, form)  # the work-item form in use
        b.step(57)
        assert b.t == 57
        for i, s in enumerate(base):
            ref, m0, m1 = standalone(s, 57)
            assert np.abs(b.phi(i) - ref).max() <= 1e-6
            assert b.mass(i) == pytest.approx(m1, rel=1e-6)
            assert abs(b.mass(i) - m0) <= 1e-5 * m0


def test_graph_steps_match_sequential_launches(form):
    specs = [dict(s, vortex_sign=-1.0) for s in FORMS[form]]
    with A.Batch(specs) as a, A.Batch(specs) as b:
        a.step(40)
        b.step_sequential(25)
        b.step(15)  # mixing the two modes keeps the device time in step
        assert a.t == b.t == 40
        for i in range(len(specs)):
            assert np.abs(a.phi(i) - b.phi(i)).max() <= 1e-6


def test_autotune_keeps_the_state_and_picks_candidate_heights(form):
    base = FORMS[form]
    specs = [dict(s, vortex_sign=-1.0) for s in base]
    with A.Batch(specs) as b:
        b.step(10)
        before = [b.phi(i) for i in range(len(base))]
        rows = b.autotune(steps_per_trial=2)
        assert b.t == 10
        for i, s in enumerate(base):
            assert rows[i] in (8, 16, 32, 64, 128, 256) or rows[i] == s["ny"]
            assert np.array_equal(b.phi(i), before[i])
        b.step(20)
        for i, s in enumerate(base):
            ref, _, _ = standalone(s, 30)
            assert np.abs(b.phi(i) - ref).max() <= 1e-6


def test_batch_lattice_close_to_oracle():
    """One lattice of a batch against the FP64 oracle over 40 steps (FP32 storage)."""
    s = SPECS[0]
    phi0 = W.disk_phi0(s["nx"], s["ny"], s["xc"], s["yc"], s["R"], s["eps"])
    p = O.Params(nx=s["nx"], ny=s["ny"], tau=s["tau"], eps=s["eps"], U0=s["U0"], T=s["T_period"], sign=-1.0)
    ref = O.Sim(p, phi0).step(40).phi()
    with A.Batch([dict(x, vortex_sign=-1.0) for x in SPECS]) as b:
        b.step(40)
        assert np.abs(b.phi(0) - ref).max() <= 2e-5


def test_batch_rejects_unsupported_lattices():
    with pytest.raises(A.LbmAceError):
        A.Batch([dict(nx=65, ny=64)])
    with pytest.raises(A.LbmAceError):
        A.Batch([dict(nx=64, ny=64), dict(nx=64, ny=64, model=A.MODEL_CONSERVATIVE)])


def test_full_batch_of_256_lattices_at_sampled_lattices():
    """The 256-lattice workload of the batch study (73.65M nodes, seeded draws of size,
    disk, eps, tau, U0 and T), autotuned and stepped as the study runs it; the smallest,
    the largest and six random lattices are checked against the same lattice alone."""
    from paper_2203_05230_gb300 import experiments as E
    specs = E.batch_specs(256)
    sides = np.array([s["nx"] for s in specs])
    picks = sorted({int(np.argmin(sides)), int(np.argmax(sides)), 0, 255,
                    *[int(i) for i in np.random.default_rng(3).choice(256, 4, replace=False)]})
    with A.Batch(specs) as b:
        b.autotune(steps_per_trial=1)
        assert b.t == 0
        b.step(5)
        for i in picks:
            with A.Lattice(precision=A.F32, velocity_kind=A.VEL_SINGLE_VORTEX, **specs[i]) as g:
                m0 = g.mass()
                g.step(5)
                assert np.abs(b.phi(i) - g.phi()).max() <= 1e-6
                assert b.mass(i) == pytest.approx(g.mass(), rel=1e-6)
                assert abs(b.mass(i) - m0) <= 1e-5 * m0


def test_lattices_retire_at_their_own_end_step(form):
    """Uneven runs: each lattice advances until its own end step and then keeps its
    state, while the others go on; every lattice equals the same lattice run alone for
    exactly its own number of steps."""
    ends = [37, 60, 12, 60, 45]
    base = FORMS[form]
    specs = [dict(s, vortex_sign=-1.0) for s in base]
    with A.Batch(specs) as b:
        b.set_ends(ends)
        b.step(20)
        assert b.active()[0] == sum(e > 20 for e in ends)
        b.step(50)
        assert b.t == 70 and b.active() == (0, 0)
        for i, s in enumerate(base):
            assert b.lattice_steps(i) == ends[i]
            ref, m0, m1 = standalone(s, ends[i])
            assert np.abs(b.phi(i) - ref).max() <= 1e-6
            assert b.mass(i) == pytest.approx(m1, rel=1e-6)


def test_per_lattice_graph_and_host_launches_match_the_persistent_batch(form):
    """The two baselines -- one launch per lattice per step, captured in a graph or issued
    from the host -- give the batch's states, with retirement applied the same way."""
    ends = [30, 18, 41, 25, 9]
    specs = [dict(s, vortex_sign=-1.0) for s in FORMS[form]]
    with A.Batch(specs) as a, A.Batch(specs) as b, A.Batch(specs) as c:
        for x in (a, b, c):
            x.set_ends(ends)
        a.step(45)
        b.step_per_lattice(45)
        c.step_sequential(45)
        for i in range(len(specs)):
            assert b.lattice_steps(i) == c.lattice_steps(i) == ends[i]
            assert np.array_equal(a.phi(i), b.phi(i))
            assert np.abs(a.phi(i) - c.phi(i)).max() <= 1e-6


def test_default_ends_are_the_periods_and_the_shape_returns():
    """set_ends() without a list ends each lattice at its period T (rounded), the time at
    which the single-vortex benchmark compares the shape with the initial one; one
    lattice is checked against the FP64 oracle at its T."""
    specs = [dict(nx=64, ny=64, tau=0.8, eps=1.0, U0=0.04, T_period=T, xc=32.0, yc=44.0, R=9.6, vortex_sign=-1.0)
             for T in (96.0, 140.4, 201.0)]
    with A.Batch(specs) as b:
        b.set_ends()
        b.step(250)
        assert [b.lattice_steps(i) for i in range(3)] == [96, 140, 201]
        s = specs[1]
        phi0 = W.disk_phi0(64, 64, s["xc"], s["yc"], s["R"], s["eps"])
        p = O.Params(nx=64, ny=64, tau=s["tau"], eps=s["eps"], U0=s["U0"], T=s["T_period"], sign=-1.0)
        ref = O.Sim(p, phi0).step(140).phi()
        assert np.abs(b.phi(1) - ref).max() <= 2e-5
        for i, sp in enumerate(specs):
            e2 = np.sqrt(((b.phi(i) - phi0) ** 2).sum() / (phi0 ** 2).sum())
            assert e2 < 0.05  # the disk is back near its start at t = T


def test_set_ends_rejects_an_end_in_the_past():
    with A.Batch([dict(s, vortex_sign=-1.0) for s in SPECS[:2]]) as b:
        b.step(10)
        with pytest.raises(A.LbmAceError) as e:
            b.set_ends([5, 20])
        assert e.value.status == A.EINVAL
        b.set_ends([10, -1])
        b.step(5)
        assert b.lattice_steps(0) == 10 and b.lattice_steps(1) == 15


def test_autotune_sweeps_the_persistent_grid(form):
    """The autotuner also picks the persistent grid: a whole number of CTAs per SM, at
    most the occupancy limit the batch starts with; the state is unaffected."""
    torch = pytest.importorskip("torch")
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    base = FORMS[form]
    specs = [dict(s, vortex_sign=-1.0) for s in base]
    with A.Batch(specs) as b:
        g0 = b.info()["grid"]
        b.autotune(steps_per_trial=2)
        g = b.info()["grid"]
        assert g % sms == 0 and sms <= g <= g0
        b.step(12)
        for i, s in enumerate(base):
            ref, _, _ = standalone(s, 12)
            assert np.abs(b.phi(i) - ref).max() <= 1e-6


def test_strip_batch_with_tiny_and_ragged_lattices():
    """Four-column strips on lattices narrower than a strip (4, 8 columns), ragged last
    strips (132, 260 = 2 x 128 + 4), and bands shorter than the default height, each
    against the same lattice alone."""
    sizes = [(4, 3), (8, 5), (132, 17), (260, 65), (16, 64)]
    specs = [dict(nx=nx, ny=ny, tau=0.8, eps=1.0, U0=0.03, T_period=400.0, xc=0.5 * nx, yc=0.6 * ny,
                  R=0.25 * min(nx, ny) + 1.0, vortex_sign=-1.0) for nx, ny in sizes]
    with A.Batch(specs) as b:
        assert b.info(0)["tiles"] == expected_items(b, specs, "quad")
        b.step(23)
        for i, s in enumerate(specs):
            ref, m0, m1 = standalone({k: v for k, v in s.items() if k != "vortex_sign"}, 23)
            assert np.abs(b.phi(i) - ref).max() <= 1e-6, (i, s["nx"], s["ny"])
            assert b.mass(i) == pytest.approx(m1, rel=1e-6)
