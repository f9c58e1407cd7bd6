"""16-bit deviation storage (FP16 / BF16) against the FP64 oracle, through the C ABI.

The library stores g_i = f*_i - s_i phi in 16 bits (s: dyadic split weights summing
to 1) and does all arithmetic in FP32. Tolerances follow from the storage rounding:
the deviations are at most ~0.02 in these states, so one rounding costs ~1e-5 (FP16,
11-bit significand) or ~8e-5 (BF16, 8-bit) absolute; one step is checked against
5e-5 (FP16) and 4e-4 (BF16) of max|f|. Over the full 256^2 single-vortex period the
phi-L2 error against the oracle is bounded and printed.
"""
import math

import numpy as np
import pytest

import oracle as O
from paper_2203_05230_gb300 import lbm_ace as A
from paper_2203_05230_gb300 import workloads as W

pytestmark = pytest.mark.gpu

DEV = [(A.F16DEV, 5e-5), (A.BF16DEV, 4e-4)]


def rel_max(a, b):
    return np.abs(a - b).max() / np.abs(b).max()


@pytest.mark.parametrize("precision,tol", DEV)
@pytest.mark.parametrize("nx,ny,model", [(64, 64, 0), (258, 37, 0), (514, 21, 1), (4, 9, 0), (516, 37, 1),
                                         (1032, 11, 0)])
def test_dev_one_step_close_to_oracle(precision, tol, nx, ny, model):
    op = O.Params(nx=nx, ny=ny, tau=0.8, eps=1.0, U0=0.05, T=100.0, sign=-1.0, model=model)
    s = O.Sim(op, W.random_smooth_phi(nx, ny, seed=nx + ny)).step(3)
    with A.Lattice(nx=nx, ny=ny, tau=0.8, eps=1.0, U0=0.05, T_period=100.0, vortex_sign=-1.0,
                   model=model, precision=precision) as g:
        g.set_state(s.f, s.phi_prev, s.t)
        f_in, pp_in = g.get_state()          # the state as stored (rounded to 16 bits)
        assert rel_max(f_in, s.f) <= tol and np.array_equal(pp_in, s.phi_prev.astype(np.float32))
        g.step(1)
        f, pp = g.get_state()
    ref = O.Sim.from_state(op, f_in, pp_in, s.t).step(1)  # oracle from the stored state
    assert rel_max(f, ref.f) <= tol
    assert rel_max(pp, ref.phi_prev) <= 1e-6  # phi(t) itself is FP32


@pytest.mark.parametrize("precision,bound,mbound", [(A.F16DEV, 2e-4, 5e-5), (A.BF16DEV, 5e-3, 1e-3)])
def test_dev_full_period_256_phi_l2_and_mass(precision, bound, mbound):
    """Single vortex on 256^2 (T = 4096, eps 1) against the FP64 oracle: phi-L2 after the
    full period (printed; measured 3.8e-5 FP16, 1.0e-3 BF16), and the mass drift left by
    rounding the deviations to 16 bits (unbiased, so it grows like a random walk:
    measured 5.6e-6 FP16, 2.2e-4 BF16 over the period)."""
    v = W.vortex_fp32(256)
    phi0 = v.phi0()
    op = O.Params(nx=256, ny=256, tau=v.tau, eps=v.eps, U0=v.U0, T=v.T, sign=v.sign)
    ref = O.Sim(op, phi0).step(v.T, threads=O.threads_available()).phi()
    with A.Lattice(nx=256, ny=256, tau=v.tau, eps=v.eps, U0=v.U0, T_period=float(v.T),
                   vortex_sign=v.sign, precision=precision, phi0=phi0) as g:
        m0 = g.mass()
        g.step(v.T)
        phi = g.phi()
        m1 = g.mass()
        ms = g.step_mass()
    e2 = math.sqrt(((phi - ref) ** 2).sum() / (ref ** 2).sum())
    drift = (m1 - m0) / m0
    print(f"precision {precision}: phi-L2 vs FP64 oracle after one period = {e2:.3e}, "
          f"mass drift = {drift:.3e}")
    assert e2 <= bound
    assert abs(drift) <= mbound
    assert ms == pytest.approx(m1, rel=1e-5)


@pytest.mark.parametrize("precision,tol", DEV)
def test_dev_full_size_4096_sampled_nodes(precision, tol):
    """The 4096^2 lattice of the 16-bit storage study, in the benchmark's launch shape: one
    step from the stored (16-bit) form of an oracle-made state, checked at 512 sampled
    nodes plus the corners and the tile seams against the oracle's per-node step of that
    same stored state, and the mass bookkeeping of the step."""
    L = 4096
    v = W.vortex_fp32(L)
    op = O.Params(nx=L, ny=L, tau=v.tau, eps=v.eps, U0=v.U0, T=float(v.T), sign=v.sign)
    s = O.Sim(op, v.phi0()).step(2, threads=O.threads_available())
    rng = np.random.default_rng(4096)
    xs = np.concatenate([rng.integers(0, L, 512), [0, L - 1, 0, L - 1, 255, 256, 511, 512]])
    ys = np.concatenate([rng.integers(0, L, 512), [0, 0, L - 1, L - 1, 87, 88, 175, 176]])
    with A.Lattice(nx=L, ny=L, tau=v.tau, eps=v.eps, U0=v.U0, T_period=float(v.T), vortex_sign=v.sign,
                   precision=precision) as g:
        g.set_state(s.f, s.phi_prev, s.t)
        f_in, pp_in = g.get_state()
        del s
        ref = O.Sim.from_state(op, f_in, pp_in, 2)
        del f_in
        fn, ph = ref.step_cells(xs, ys)
        scale = np.abs(ref.f).max()
        del ref
        g.step(1)
        f, pp = g.get_state()
        m_state = g.mass()
        m_step = g.step_mass()
    got = f[:, ys, xs].T
    assert np.abs(got - fn).max() <= tol * scale
    assert np.abs(pp[ys, xs] - ph).max() <= 1e-6       # phi(t) itself is FP32
    assert m_step == pytest.approx(pp.astype(np.float64).sum(), rel=1e-12)
    assert m_state == pytest.approx(f.sum(), rel=1e-6)  # f as read back: 16-bit g + FP32 phi


@pytest.mark.parametrize("precision", [A.F16DEV, A.BF16DEV])
def test_dev_phi_readout_matches_state(precision):
    """get_phi returns the moment of the populations get_state returns."""
    with A.vortex_lattice(128, precision=precision) as g:
        g.step(37)
        f, _ = g.get_state()
        phi = g.phi()
    assert np.abs(f.sum(0) - phi).max() <= 2e-6


@pytest.mark.parametrize("precision", [A.F16DEV, A.BF16DEV])
def test_dev_resume_from_checkpoint(precision):
    """A run resumed from get_state / set_state follows the uninterrupted run to the
    storage rounding (the checkpoint goes through FP64 populations)."""
    with A.vortex_lattice(128, precision=precision) as a:
        a.step(30)
        f, pp = a.get_state()
        a.step(30)
        pa = a.phi()
    with A.vortex_lattice(128, precision=precision) as b:
        b.set_state(f, pp, 30)
        b.step(30)
        pb = b.phi()
    assert np.abs(pa - pb).max() <= (2e-5 if precision == A.F16DEV else 2e-4)


def test_dev_rejects_odd_nx_and_variants():
    with pytest.raises(A.LbmAceError):
        A.Lattice(nx=65, ny=64, precision=A.F16DEV)
    with pytest.raises(A.LbmAceError):
        A.Lattice(nx=64, ny=64, precision=A.BF16DEV, kernel_variant=1)
    with pytest.raises(A.LbmAceError):
        A.Lattice(nx=66, ny=64, precision=A.BF16DEV, kernel_variant=A.KERNEL_DEV4)
    with pytest.raises(A.LbmAceError):
        A.Lattice(nx=64, ny=64, precision=A.F32, kernel_variant=A.KERNEL_DEV4)


def _vel_kw(kind, nx, ny):
    if kind == "vortex":
        return dict(U0=0.05, T_period=60.0, vortex_sign=-1.0)
    if kind == "uniform":
        return dict(velocity_kind=A.VEL_UNIFORM, ux=0.03, uy=-0.02)
    rng = np.random.default_rng(nx * 7 + ny)
    return dict(velocity_kind=A.VEL_FIELD, u_field=0.04 * rng.uniform(-1, 1, (ny, nx)),
                v_field=0.04 * rng.uniform(-1, 1, (ny, nx)))


@pytest.mark.parametrize("precision", [A.F16DEV, A.BF16DEV])
@pytest.mark.parametrize("nx,ny,model,vel", [(512, 40, 0, "vortex"), (516, 37, 0, "vortex"), (1028, 19, 1, "uniform"),
                                             (4, 9, 0, "field"), (8, 3, 0, "vortex"), (264, 130, 0, "field"),
                                             (2048, 64, 0, "vortex")])
def test_dev_quad_kernel_is_bit_identical_to_pair_kernel(precision, nx, ny, model, vel):
    """The four-columns-per-thread kernel (7) and the column-pair kernel (5) do the same
    arithmetic on the same values: 13 steps from t = 0 (the first step has no time
    derivative) agree bit for bit, on full and ragged strips, lattices narrower than one
    quad's strip, every velocity source and both models. The quad kernel's FP64 step
    mass (summed exactly in FP32 parts) matches the FP64 sum of the phi it wrote."""
    phi0 = W.random_smooth_phi(nx, ny, seed=nx + 3 * ny)
    out = []
    for variant in (A.KERNEL_DEV, A.KERNEL_DEV4):
        with A.Lattice(nx=nx, ny=ny, model=model, precision=precision, phi0=phi0, kernel_variant=variant,
                       **_vel_kw(vel, nx, ny)) as g:
            assert g.launch_shape()[4] == variant
            g.step(13)
            f, pp = g.get_state()
            out.append((f, pp, g.step_mass()))
    (fa, ppa, ma), (fb, ppb, mb) = out
    assert np.array_equal(fa, fb) and np.array_equal(ppa, ppb)
    assert mb == pytest.approx(ppb.astype(np.float64).sum(), rel=1e-13, abs=1e-300)
    assert ma == pytest.approx(mb, rel=1e-12)


@pytest.mark.parametrize("precision", [A.F16DEV, A.BF16DEV])
def test_dev_default_kernel_choice(precision):
    with A.Lattice(nx=64, ny=16, precision=precision) as g:
        assert g.launch_shape()[4] == A.KERNEL_DEV4
    with A.Lattice(nx=66, ny=16, precision=precision) as g:
        assert g.launch_shape()[4] == A.KERNEL_DEV


@pytest.mark.parametrize("precision,variant,other", [(A.F32, A.KERNEL_QUAD, A.KERNEL_PAIR),
                                                    (A.BF16DEV, A.KERNEL_DEV4, A.KERNEL_DEV)])
def test_quad_kernels_take_at_most_4095_rows_per_band(precision, variant, other):
    """The integer part of the quad kernels' step mass is exact for bands of at most 4095
    rows: an explicit taller band is refused, the automatic shape never exceeds it, and a
    4095-row band gives the column-pair kernels' states and step mass."""
    nx, ny = 8, 4100
    with pytest.raises(A.LbmAceError) as e:
        A.Lattice(nx=nx, ny=ny, precision=precision, kernel_variant=variant, rows_per_cta=4096)
    assert e.value.status == A.EINVAL
    phi0 = W.random_smooth_phi(nx, ny, seed=5)
    out = []
    for v, rows in ((variant, 4095), (variant, 0), (other, 4095)):
        with A.Lattice(nx=nx, ny=ny, precision=precision, kernel_variant=v, rows_per_cta=rows, phi0=phi0,
                       T_period=900.0) as g:
            shape = g.launch_shape()
            assert shape[4] == v and shape[1] <= 4095
            g.step(3)
            f, pp = g.get_state()
            out.append((f, pp, g.step_mass()))
    # the step masses: a 4095-row band of this 8-wide lattice gives each of its two
    # threads 4 x 4095 values, whose FP32 remainder sum (terms below 2^-17, a random walk
    # of ~5e-4) rounds by ~1e-10 of the total; default launch shapes give a thread at
    # most a few hundred values (~1e-14)
    for f, pp, m in out[1:]:
        assert np.array_equal(f, out[0][0]) and np.array_equal(pp, out[0][1])
        assert m == pytest.approx(out[0][2], rel=1e-9)
    assert out[0][2] == pytest.approx(float(out[0][1].astype(np.float32).astype(np.float64).sum()), rel=1e-9)
