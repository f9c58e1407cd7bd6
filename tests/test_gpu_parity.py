"""CUDA path against the FP64 CPU oracle, element by element, through the C ABI.

Tolerances, FP64 storage and arithmetic:
* one step from an identical state: |f_gpu - f_oracle| <= 1e-12 max|f_oracle| for
  every population of every node. The two sides differ only in rounding order and in
  libm vs CUDA log/sqrt (each below 1e-15 relative); the bound is on the field's max
  norm because in the bulk the regularised normal of Eq. 13 turns rounding of psi
  into O(1) relative noise of values that are themselves ~1e-12 of the field.
* several steps: 2e-9 max|phi|. The method itself sets this bound. Where phi
  saturates at exactly 1 (the initial disk), the clip and the regulariser of Eq. 13
  leave a force floor of ~delta/eps (2e-9) whose direction comes from rounding noise
  in psi; an oracle run whose initial populations are perturbed by one ulp differs
  from the unperturbed run by 5e-10 after one step (decaying to ~1e-11 after 20), so
  no two correct implementations agree better than that over several steps.
FP32: one step within 2e-6 max|f| (a few float ulps); phi-L2 within 1e-5 after a
full single-vortex period.

All oracle inputs come from the seeded generators in workloads.py or from the
oracle itself; none comes from the CUDA path.
"""
import math

import numpy as np
import pytest

import oracle as O
from paper_2203_05230_gb300 import lbm_ace as A
from paper_2203_05230_gb300 import workloads as W

pytestmark = pytest.mark.gpu

VEL = {"vortex": (O.VORTEX, A.VEL_SINGLE_VORTEX), "uniform": (O.UNIFORM, A.VEL_UNIFORM),
       "field": (O.FIELD, A.VEL_FIELD)}


def pair(nx, ny, *, tau=0.8, eps=1.0, model=0, vel="vortex", T=100.0, U0=0.05, sign=-1.0,
         ux=0.02, uy=-0.015, precision=A.F64, rows=0, phi0=None, seed=0, variant=0):
    """Matching oracle parameters and library keyword arguments."""
    ok, ak = VEL[vel]
    uf = vf = None
    if vel == "field":
        rng = np.random.default_rng(seed + 100)
        uf = 0.05 * rng.uniform(-1, 1, (ny, nx))
        vf = 0.05 * rng.uniform(-1, 1, (ny, nx))
    op = O.Params(nx=nx, ny=ny, tau=tau, eps=eps, model=model, vel_kind=ok, U0=U0, T=T, sign=sign,
                  ux=ux, uy=uy, ufield=uf, vfield=vf)
    kw = dict(nx=nx, ny=ny, tau=tau, eps=eps, model=model, velocity_kind=ak, U0=U0, T_period=T,
              vortex_sign=sign, ux=ux, uy=uy, precision=precision, rows_per_cta=rows,
              kernel_variant=variant)
    if uf is not None:
        kw["u_field"], kw["v_field"] = uf, vf
    if phi0 is not None:
        kw["phi0"] = phi0
    return op, kw


def oracle_state(op, seed=0, steps=3):
    """A non-equilibrium state at t = steps, made by the oracle from a seeded field."""
    phi0 = W.random_smooth_phi(op.nx, op.ny, seed=seed, eps=op.eps)
    return O.Sim(op, phi0).step(steps)


ONE_STEP = 1e-12
MULTI_STEP = 2e-9


def rel_max(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


SHAPES = [(8, 8), (16, 16), (64, 64), (9, 7), (37, 53), (130, 20), (257, 70), (3, 3), (3, 5),
          (4, 9), (132, 40), (260, 33), (258, 11), (514, 21)]


def variants(nx, precision):
    """Kernel variants valid for this width: direct loads and independent warps always,
    the bulk-copy pipeline when a row is a multiple of 16 bytes."""
    elem = 8 if precision == A.F64 else 4
    return ([A.KERNEL_DIRECT, A.KERNEL_WARP] + ([A.KERNEL_BULK] if (nx * elem) % 16 == 0 else [])
            + ([A.KERNEL_PAIR] if nx % 2 == 0 else []))


CASES = [(nx, ny, v) for nx, ny in SHAPES for v in variants(nx, A.F64)]


@pytest.mark.parametrize("nx,ny,variant", CASES)
@pytest.mark.parametrize("model", [A.MODEL_MODIFIED, A.MODEL_CONSERVATIVE])
def test_f64_one_step_matches_oracle(nx, ny, variant, model):
    op, kw = pair(nx, ny, model=model, variant=variant)
    s = oracle_state(op, seed=nx * 1000 + ny)
    with A.Lattice(**kw) as g:
        g.set_state(s.f, s.phi_prev, s.t)
        g.step(1)
        f, pp = g.get_state()
    s.step(1)
    assert rel_max(f, s.f) <= ONE_STEP
    assert rel_max(pp, s.phi_prev) <= ONE_STEP


QUAD_SHAPES = [(8, 8), (16, 16), (64, 64), (4, 9), (132, 40), (260, 33), (516, 37), (1028, 19), (384, 3)]


@pytest.mark.parametrize("nx,ny", QUAD_SHAPES)
@pytest.mark.parametrize("model", [A.MODEL_MODIFIED, A.MODEL_CONSERVATIVE])
@pytest.mark.parametrize("vel", ["vortex", "field"])
def test_f32_quad_kernel_one_step_matches_oracle(nx, ny, model, vel):
    """The four-columns-per-thread FP32 kernel (warp strips of 128 columns, ragged and
    dead strips, lattices narrower than a quad's strip) one step from an oracle state,
    and bit for bit the column-pair kernel over 10 steps from that state."""
    op, kw = pair(nx, ny, model=model, vel=vel, precision=A.F32, variant=A.KERNEL_QUAD, seed=nx + ny)
    s = oracle_state(op, seed=nx * 1000 + ny)
    out = []
    for variant in (A.KERNEL_QUAD, A.KERNEL_PAIR):
        kw["kernel_variant"] = variant
        with A.Lattice(**kw) as g:
            assert g.launch_shape()[4] == variant
            g.set_state(s.f, s.phi_prev, s.t)
            g.step(1)
            out.append(g.get_state())
            g.step(9)
            out.append(g.get_state() + (g.step_mass(),))
    f, pp = out[0]
    nxt = s.copy().step(1)
    assert rel_max(f, nxt.f) <= 2e-6
    assert rel_max(pp, nxt.phi_prev) <= 2e-6
    fq, ppq, mq = out[1]
    fp_, ppp, _ = out[3]
    assert np.array_equal(out[0][0], out[2][0]) and np.array_equal(fq, fp_) and np.array_equal(ppq, ppp)
    assert mq == pytest.approx(ppq.sum(), rel=1e-12)


@pytest.mark.parametrize("vel", ["vortex", "uniform", "field"])
@pytest.mark.parametrize("t0", [0, 1, 57])
def test_f64_velocity_sources_and_first_step(vel, t0):
    op, kw = pair(33, 29, vel=vel, T=80.0)
    s = oracle_state(op, seed=5, steps=0)
    s.t = t0
    with A.Lattice(**kw) as g:
        g.set_state(s.f, s.phi_prev, t0)
        g.step(1)
        f1, pp1 = g.get_state()
        g.step(2)
        f, pp = g.get_state()
        assert g.t == t0 + 3
    s.step(1)
    assert rel_max(f1, s.f) <= ONE_STEP and rel_max(pp1, s.phi_prev) <= ONE_STEP
    s.step(2)
    assert rel_max(f, s.f) <= MULTI_STEP and rel_max(pp, s.phi_prev) <= MULTI_STEP


@pytest.mark.parametrize("rows", [1, 2, 3, 7, 64])
@pytest.mark.parametrize("variant", [A.KERNEL_DIRECT, A.KERNEL_BULK, A.KERNEL_WARP, A.KERNEL_PAIR])
def test_f64_launch_shapes_agree(rows, variant):
    """Rows per CTA and the kernel variant change only the tiling and how rows reach
    the SM: one step matches the oracle, and ten steps are bit-for-bit those of the
    default launch (the halo recomputation sums the populations in the same order as
    the interior, and both variants share the collision code)."""
    op, kw = pair(150, 53, rows=rows, variant=variant)
    s = oracle_state(op, seed=11)
    with A.Lattice(**kw) as g:
        assert g.launch_shape()[1] == min(rows, 53)  # clamped to ny
        g.set_state(s.f, s.phi_prev, s.t)
        g.step(1)
        f, _ = g.get_state()
        g.step(9)
        f10, pp10 = g.get_state()
    with A.Lattice(**{**kw, "rows_per_cta": 0, "kernel_variant": A.KERNEL_DIRECT}) as d:
        d.set_state(s.f, s.phi_prev, s.t)
        d.step(10)
        fd, ppd = d.get_state()
    s.step(1)
    assert rel_max(f, s.f) <= ONE_STEP
    assert np.array_equal(f10, fd) and np.array_equal(pp10, ppd)


def test_f64_init_matches_oracle_init_and_phi_and_mass():
    v = W.VORTEX_64_F64
    op, kw = pair(64, 64, T=v.T, U0=v.U0, phi0=v.phi0())
    s = O.Sim(op, v.phi0())
    with A.Lattice(**kw) as g:
        f, pp = g.get_state()
        assert rel_max(f, s.f) <= 1e-15 and np.array_equal(pp, s.phi_prev)
        assert rel_max(g.phi(), s.phi()) <= 1e-15
        assert g.mass() == pytest.approx(s.mass(), rel=1e-14)
        # built-in disk equals the host-built disk
    with A.Lattice(**{k: x for k, x in kw.items() if k != "phi0"}, xc=v.xc, yc=v.yc, R=v.R) as g2:
        assert rel_max(g2.phi(), s.phi()) <= 1e-15


def test_f64_full_vortex_period_64():
    """The 64^2 FP64 single vortex (R 9.6 at (32, 48), eps 1, tau 0.8, U0 0.04, T 2000)
    over a full period: phi matches the oracle within the multi-step bound, the
    shape-return errors agree, and the GPU conserves mass to 1e-12."""
    v = W.VORTEX_64_F64
    op, kw = pair(64, 64, T=v.T, U0=v.U0, sign=v.sign, tau=v.tau, eps=v.eps, phi0=v.phi0())
    s = O.Sim(op, v.phi0())
    s.step(v.T, threads=O.threads_available())
    with A.Lattice(**kw) as g:
        m0 = g.mass()
        for _ in range(4):
            g.step(v.T // 4)
        phi = g.phi()
        m1 = g.mass()
    assert rel_max(phi, s.phi()) <= MULTI_STEP
    assert abs(m1 - m0) / m0 <= 1e-12
    phi0 = v.phi0()
    e1g = np.abs(phi - phi0).sum() / phi0.sum()
    e1o = np.abs(s.phi() - phi0).sum() / phi0.sum()
    assert e1g == pytest.approx(e1o, rel=1e-7)


@pytest.mark.parametrize("nx,ny,variant", [(nx, ny, v) for nx, ny in [(64, 64), (37, 53), (257, 70), (260, 33)]
                                            for v in variants(nx, A.F32)])
def test_f32_one_step_close_to_oracle(nx, ny, variant):
    op, kw = pair(nx, ny, precision=A.F32, variant=variant)
    s = oracle_state(op, seed=3)
    with A.Lattice(**kw) as g:
        g.set_state(s.f, s.phi_prev, s.t)
        g.step(1)
        f, pp = g.get_state()
    s.step(1)
    assert rel_max(f, s.f) <= 2e-6 and rel_max(pp, s.phi_prev) <= 2e-6


def test_f32_full_period_256_phi_l2():
    """FP32 single vortex on 256^2 (T = 16 L = 4096, eps 1): phi-L2 against the FP64
    oracle within 1e-5 after the full period."""
    v = W.vortex_fp32(256)
    phi0 = v.phi0()
    op, kw = pair(256, 256, T=v.T, U0=v.U0, sign=v.sign, tau=v.tau, eps=v.eps, phi0=phi0,
                  precision=A.F32)
    s = O.Sim(op, phi0).step(v.T, threads=O.threads_available())
    with A.Lattice(**kw) as g:
        m0 = g.mass()
        g.step(v.T)
        phi = g.phi()
        m1 = g.mass()
    ref = s.phi()
    e2 = math.sqrt(((phi - ref) ** 2).sum() / (ref ** 2).sum())
    assert e2 <= 1e-5, e2
    assert abs(m1 - m0) / m0 <= 1e-5


@pytest.mark.parametrize("precision,tol", [(A.F32, 2e-6), (A.F64, ONE_STEP)])
def test_full_size_2048_sampled_nodes(precision, tol):
    # default launch: the kernel variant and shape the benchmark uses
    """The 2048^2 lattice in the benchmark's launch shape: one step from an oracle-made
    state, checked at 512 sampled nodes (plus the four corners and the tile seams)
    against the oracle's per-node evaluation, and exact global mass bookkeeping."""
    L = 2048
    v = W.vortex_fp32(L)
    op, kw = pair(L, L, T=v.T, U0=v.U0, sign=v.sign, tau=v.tau, eps=v.eps, precision=precision)
    s = O.Sim(op, v.phi0()).step(2, threads=O.threads_available())
    rng = np.random.default_rng(2048)
    xs = np.concatenate([rng.integers(0, L, 512), [0, L - 1, 0, L - 1, 127, 128, 255, 256]])
    ys = np.concatenate([rng.integers(0, L, 512), [0, 0, L - 1, L - 1, 31, 32, 63, 64]])
    fn, ph = s.step_cells(xs, ys)
    with A.Lattice(**kw) as g:
        g.set_state(s.f, s.phi_prev, s.t)
        g.step(1)
        f, pp = g.get_state()
        m_state = g.mass()
        m_step = g.step_mass()
    scale = np.abs(s.f).max()
    got = f[:, ys, xs].T
    assert np.abs(got - fn).max() <= tol * scale
    assert np.abs(pp[ys, xs] - ph).max() <= tol
    assert m_step == pytest.approx(pp.sum(), rel=1e-12)
    assert m_state == pytest.approx(f.sum(), rel=1e-12)


def test_checkpoint_resume_is_bitwise():
    op, kw = pair(96, 80, T=500.0)
    s = oracle_state(op, seed=9, steps=0)
    with A.Lattice(**kw, phi0=s.phi()) as a:
        a.step(40)
        f, pp = a.get_state()
        t = a.t
        a.step(60)
        fa, ppa = a.get_state()
    with A.Lattice(**kw, phi0=s.phi()) as b:
        b.set_state(f, pp, t)
        b.step(60)
        fb, ppb = b.get_state()
    assert np.array_equal(fa, fb) and np.array_equal(ppa, ppb)


def test_uniform_phi_is_a_fixed_point():
    """Degenerate case: constant phi has grad psi = 0, so n = 0 and no sharpening;
    with a uniform velocity the equilibrium state stays put."""
    for val in (0.0, 0.3, 1.0):
        with A.Lattice(nx=20, ny=12, velocity_kind=A.VEL_UNIFORM, ux=0.03, uy=0.01,
                       phi0=np.full((12, 20), val)) as g:
            g.step(50)
            assert np.abs(g.phi() - val).max() <= 1e-14


def test_zero_steps_and_repeated_calls():
    with A.Lattice(nx=16, ny=16) as g:
        f0, _ = g.get_state()
        g.step(0)
        f1, _ = g.get_state()
        assert np.array_equal(f0, f1) and g.t == 0
        with pytest.raises(A.LbmAceError):
            g.step_mass()
        with pytest.raises(A.LbmAceError):
            g.step(-1)


def test_callback_velocity_equals_field_velocity_and_reports_errors():
    nx, ny = 40, 24
    rng = np.random.default_rng(1)
    u = 0.03 * rng.uniform(-1, 1, (ny, nx))
    v = 0.03 * rng.uniform(-1, 1, (ny, nx))
    phi0 = W.random_smooth_phi(nx, ny, seed=2)
    with A.Lattice(nx=nx, ny=ny, velocity_kind=A.VEL_FIELD, u_field=u, v_field=v, phi0=phi0) as a:
        a.step(25)
        pa = a.phi()
    with A.Lattice(nx=nx, ny=ny, vel_fn=lambda t, nx_, ny_: (u, v), phi0=phi0) as b:
        b.step(25)
        pb = b.phi()
    assert np.array_equal(pa, pb)

    def bad(t, nx_, ny_):
        if t >= 3:
            raise ValueError("no velocity")
        return u, v
    with A.Lattice(nx=nx, ny=ny, vel_fn=bad, phi0=phi0) as c:
        with pytest.raises(A.LbmAceError) as e:
            c.step(10)
        assert e.value.status == A.ECALLBACK


def test_callback_time_dependent_matches_oracle_vortex():
    """A host callback that evaluates Eq. 14 reproduces the built-in vortex."""
    L, T = 48, 300.0
    phi0 = W.disk_phi0(L, L, 24, 36, 7.2, 1.0)
    y, x = np.mgrid[0:L, 0:L].astype(float)

    def vortex(t, nx_, ny_):
        c = math.cos(math.pi * t / T)
        return (-0.04 * np.sin(np.pi * x / L) ** 2 * np.sin(2 * np.pi * y / L) * c,
                0.04 * np.sin(np.pi * y / L) ** 2 * np.sin(2 * np.pi * x / L) * c)
    op, kw = pair(L, L, T=T, U0=0.04, sign=-1.0, phi0=phi0)
    s = O.Sim(op, phi0).step(30)
    with A.Lattice(nx=L, ny=L, vel_fn=vortex, phi0=phi0) as g:
        g.step(30)
        assert rel_max(g.phi(), s.phi()) <= MULTI_STEP


@pytest.mark.parametrize("L,precision", [(2048, A.F32), (512, A.F64), (260, A.F32), (132, A.F64)])
def test_kernel_variants_are_bit_identical(L, precision):
    """The kernel variants do the same arithmetic on the same values: 12 steps of the
    single vortex agree bit for bit."""
    out = []
    quad = [A.KERNEL_QUAD] if precision == A.F32 and L % 4 == 0 else []
    for variant in [A.KERNEL_DIRECT, A.KERNEL_BULK, A.KERNEL_WARP, A.KERNEL_PAIR] + quad:
        with A.vortex_lattice(L, precision=precision, kernel_variant=variant) as g:
            assert g.launch_shape()[4] == variant
            g.step(12)
            out.append(g.get_state())
    for o in out[1:]:
        assert np.array_equal(out[0][0], o[0]) and np.array_equal(out[0][1], o[1])


@pytest.mark.parametrize("k", [0, 12345, 300 * 300 - 1])
def test_large_non_finite_phi0_is_rejected_after_upload(k):
    """phi0 fields above 65,536 values are checked on the device right after their
    upload (small ones on the host): the smallest bad index is reported as EINVAL, and a
    valid field then builds a working lattice."""
    phi0 = np.full((300, 300), 0.5)
    phi0.flat[k] = np.inf if k % 2 else np.nan
    phi0.flat[min(k + 7, phi0.size - 1)] = np.nan
    with pytest.raises(A.LbmAceError) as e:
        A.Lattice(nx=300, ny=300, phi0=phi0, precision=A.F32)
    assert e.value.status == A.EINVAL and f"phi0[{k}]" in str(e.value)
    with A.Lattice(nx=300, ny=300, phi0=np.full((300, 300), 0.5), precision=A.F32) as g:
        g.step(3)
        assert g.mass() == pytest.approx(0.5 * 300 * 300, rel=1e-6)  # FP32 populations
