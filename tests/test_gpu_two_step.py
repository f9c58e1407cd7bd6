"""Two steps per launch (kernel variant 6, temporal blocking in shared memory): the
same arithmetic on the same values as two launches of the column-pair kernel, so
states, phi and the state mass must agree bit for bit with variant 4 (the step mass up
to its summation order) for any step count
(odd counts end with one pair step), strip widths that do not fill the 256-column tile,
lattices smaller than a tile, every velocity source and both models."""
import numpy as np
import pytest

from paper_2203_05230_gb300 import lbm_ace as A
from paper_2203_05230_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def run(variant, nx, ny, steps, **kw):
    with A.Lattice(nx=nx, ny=ny, precision=A.F32, kernel_variant=variant,
                   phi0=W.random_smooth_phi(nx, ny, seed=nx + 7 * ny), **kw) as g:
        assert g.launch_shape()[4] == variant
        out = []
        for s in steps:
            g.step(s)
            f, pp = g.get_state()
            out.append((f, pp, g.step_mass() if g.t > 0 else None, g.mass(), g.t))
        return out


def same(a, b):
    for (fa, pa, ma, ga, ta), (fb, pb, mb, gb, tb) in zip(a, b):
        assert ta == tb
        assert np.array_equal(fa, fb) and np.array_equal(pa, pb)
        # the pair kernel alternates the bands' march direction, so its FP64 step-mass
        # partials are summed in another order than the two-step kernel's
        assert ga == gb and (ma == mb or abs(ma - mb) <= 1e-14 * abs(mb))


VORTEX = dict(velocity_kind=A.VEL_SINGLE_VORTEX, U0=0.04, T_period=400.0, vortex_sign=-1.0)


@pytest.mark.parametrize("nx,ny", [(256, 64), (512, 200), (258, 41), (300, 33), (8, 8), (24, 5), (1024, 96)])
def test_two_step_equals_pair_steps(nx, ny):
    steps = [1, 2, 3, 10, 4]
    same(run(A.KERNEL_PAIR, nx, ny, steps, **VORTEX), run(A.KERNEL_TWO_STEP, nx, ny, steps, **VORTEX))


@pytest.mark.parametrize("model", [A.MODEL_MODIFIED, A.MODEL_CONSERVATIVE])
@pytest.mark.parametrize("vel", ["uniform", "field"])
def test_two_step_velocity_sources_and_models(vel, model):
    nx, ny = 264, 70
    if vel == "uniform":
        kw = dict(velocity_kind=A.VEL_UNIFORM, ux=0.03, uy=-0.02)
    else:
        u, v = W.stream_function_field(nx, 3)
        u, v = u[:ny], v[:ny]
        kw = dict(velocity_kind=A.VEL_FIELD, u_field=np.ascontiguousarray(u), v_field=np.ascontiguousarray(v))
    same(run(A.KERNEL_PAIR, nx, ny, [6, 5], model=model, **kw),
         run(A.KERNEL_TWO_STEP, nx, ny, [6, 5], model=model, **kw))


def test_two_step_after_restart_and_checkpoint():
    nx, ny = 256, 48
    with A.Lattice(nx=nx, ny=ny, precision=A.F32, kernel_variant=A.KERNEL_TWO_STEP, **VORTEX) as g, \
         A.Lattice(nx=nx, ny=ny, precision=A.F32, kernel_variant=A.KERNEL_PAIR, **VORTEX) as h:
        g.step(7)
        h.step(7)
        f, pp = g.get_state()
        g.set_state(f, pp, g.t)
        g.step(8)
        h.step(8)
        assert np.array_equal(g.get_state()[0], h.get_state()[0])


def test_two_step_rejects_what_it_cannot_do():
    for kw in (dict(precision=A.F64), dict(precision=A.F32, nx=63), dict(precision=A.F32, vel_fn=lambda t, nx, ny: (np.zeros((ny, nx)), np.zeros((ny, nx))))):
        args = dict(nx=64, ny=64, kernel_variant=A.KERNEL_TWO_STEP)
        args.update(kw)
        with pytest.raises(A.LbmAceError) as e:
            A.Lattice(**args)
        assert e.value.status == A.EINVAL
