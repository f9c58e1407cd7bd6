"""Mutation check of the oracles' pins (CPU).

A pin is only worth something if a plausible mistake in the oracle fails it. Each case
below plants one such mistake -- a dropped or sign-flipped term, a wrong prefactor, a
transposed index, a mis-read formula -- in a copy of the oracle's source (the C step of
Eqs. 9-14 or the numpy surrogate network), runs the unchanged pin suite against that
copy in a fresh process, and requires at least one pin to fail. An unmutated copy run
the same way must pass, so a broken harness cannot pass for a caught mutant.

The copies live in a temporary tree (oracle/, tests/ with the pin file, its conftest
and golden values); the library package is reached through PYTHONPATH. Nothing here
touches the CUDA path.
"""
import concurrent.futures as cf
import os
import shutil
import subprocess
import sys
import tempfile

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

# (name, file in oracle/, text to replace, replacement, which occurrence)
C_MUTANTS = [
    ("time derivative dropped (Sec. 2.2)", "if (t > 0) {", "if (0) {", 0),
    ("time derivative applied at t = 0 (R3)", "if (t > 0) {", "if (t >= 0) {", 0),
    ("time derivative with flipped sign", "dx = phi_c * u - phi_prev[k] * up;", "dx = phi_prev[k] * up - phi_c * u;", 0),
    ("u(t) used for u(t - 1)", "oracle_velocity(p, x, y, (double)(t - 1), &up, &vp);",
     "oracle_velocity(p, x, y, (double)t, &up, &vp);", 0),
    ("sharpening flux with flipped sign (Eq. 11)", "double gx = dx + CS2 * S * nxv, gy = dy + CS2 * S * nyv;",
     "double gx = dx - CS2 * S * nxv, gy = dy - CS2 * S * nyv;", 0),
    ("forcing prefactor 1 - 1/tau (Eq. 9)", "(1.0 - 1.0 / (2.0 * p->tau)) * F[i]", "(1.0 - 1.0 / p->tau) * F[i]", 0),
    ("forcing components transposed (Eq. 11)", "out[i] = W[i] * (CX[i] * gx + CY[i] * gy) / CS2;",
     "out[i] = W[i] * (CX[i] * gy + CY[i] * gx) / CS2;", 0),
    ("clip of phi missing (Eq. 13)", "    if (phic < 0.0) phic = 0.0;\n    if (phic > 1.0) phic = 1.0;\n", "", 0),
    ("literal tanh(2 psi / eps) of Eq. 11 with Eq. 13's psi (R1)", "double th = tanh(psi / (2.0 * eps));",
     "double th = tanh(2.0 * psi / eps);", 0),
    ("sharpening magnitude 1/eps for 1/(4 eps) (R1)", "return (1.0 - th * th) / (4.0 * eps);",
     "return (1.0 - th * th) / eps;", 0),
    ("wrong diagonal velocity c_6", "static const int CY[9] = {0, 0, 1, 0, -1, 1, 1, -1, -1};",
     "static const int CY[9] = {0, 0, 1, 0, -1, 1, -1, -1, -1};", 0),
    ("equilibrium without 1/c_s^2 (Eq. 10)", "(1.0 + cu / CS2)", "(1.0 + cu)", 0),
    ("gradient without 1/c_s^2 (R2)", "    out[0] = gx / CS2;\n    out[1] = gy / CS2;", "    out[0] = gx;\n    out[1] = gy;", 0),
    ("gradient window transposed (R2)", "double c = win[(CY[i] + 1) * 3 + (CX[i] + 1)];",
     "double c = win[(CX[i] + 1) * 3 + (CY[i] + 1)];", 0),
    ("normal not normalised (Eq. 13)", "double nxv = g[0] / (norm + p->delta), nyv = g[1] / (norm + p->delta);",
     "double nxv = g[0], nyv = g[1];", 0),
    ("psi without its eps factor (Eq. 13)", "return eps * log((phic + delta) / (1.0 - phic + delta));",
     "return log((phic + delta) / (1.0 - phic + delta));", 0),
    ("BGK relaxation with flipped sign (Eq. 9)", "fi - (fi - feq[i]) / p->tau", "fi + (fi - feq[i]) / p->tau", 0),
    ("streaming against c_i (Eq. 9, left side)",
     "size_t dst = (size_t)wrap(y + CY[i], p->ny) * p->nx + wrap(x + CX[i], p->nx);",
     "size_t dst = (size_t)wrap(y - CY[i], p->ny) * p->nx + wrap(x - CX[i], p->nx);", 0),
    ("vortex v with the sign of u (Eq. 14)", "*v = -p->sign * p->U0 * sy * sy", "*v = p->sign * p->U0 * sy * sy", 0),
    ("vortex period factor 2 (Eq. 14)", "double ct = cos(PI * t / p->T);", "double ct = cos(2.0 * PI * t / p->T);", 0),
    ("phi(t - 1) never updated", "        memcpy(phi_prev, phi, n * sizeof(double));\n", "", 0),
    ("initial populations at rest (R7)", "oracle_feq(phi0[k], u, v, feq);", "oracle_feq(phi0[k], 0.0, 0.0, feq);", 0),
    ("sampled step pulls from x + c_i", "int sx = wrap(x - CX[i], p->nx), sy = wrap(y - CY[i], p->ny);",
     "int sx = wrap(x + CX[i], p->nx), sy = wrap(y + CY[i], p->ny);", 0),
    ("conservative ablation with 4 phi(1 - phi)/eps (R8)", "S = phi_c * (1.0 - phi_c) / p->eps;",
     "S = 4.0 * phi_c * (1.0 - phi_c) / p->eps;", 0),
]

S_MUTANTS = [
    ("GELU' without the density term", "    return 0.5 * (1.0 + erf(z / math.sqrt(2.0))) + z * np.exp(-0.5 * z * z) / math.sqrt(2.0 * math.pi)",
     "    return 0.5 * (1.0 + erf(z / math.sqrt(2.0)))", 0),
    ("GELU with erf(z / 2)", "    return 0.5 * z * (1.0 + _erf(z / math.sqrt(2.0)))", "    return 0.5 * z * (1.0 + _erf(z / 2.0))", 0),
    ("forward shift with flipped sign", "shifted = np.roll(x, shift=(1 - j, 1 - i), axis=(2, 3))",
     "shifted = np.roll(x, shift=(j - 1, i - 1), axis=(2, 3))", 0),
    ("taps transposed", 'out += np.einsum("oc,bchw->bohw", W[:, :, j, i], shifted)',
     'out += np.einsum("oc,bchw->bohw", W[:, :, i, j], shifted)', 0),
    ("convolution for cross-correlation", 'out += np.einsum("oc,bchw->bohw", W[:, :, j, i], shifted)',
     'out += np.einsum("oc,bchw->bohw", W[:, :, 2 - j, 2 - i], shifted)', 0),
    ("input gradient shift with flipped sign", "W[:, :, j, i], g), shift=(j - 1, i - 1), axis=(2, 3))",
     "W[:, :, j, i], g), shift=(1 - j, 1 - i), axis=(2, 3))", 0),
    ("weight gradient shift with flipped sign", "shifted = np.roll(x, shift=(1 - j, 1 - i), axis=(2, 3))",
     "shifted = np.roll(x, shift=(j - 1, i - 1), axis=(2, 3))", 1),
    ("bias gradient as a mean", "return dW, g.sum(axis=(0, 2, 3))", "return dW, g.mean(axis=(0, 2, 3))", 0),
    ("Adam without bias correction", "    mh = m / (1.0 - beta1 ** step)\n    vh = v / (1.0 - beta2 ** step)",
     "    mh = m\n    vh = v", 0),
    ("BF16 ties away from even", "r = ((bits + np.uint64(0x7FFF) + lsb) >> np.uint64(16)) << np.uint64(16)",
     "r = ((bits + np.uint64(0x8000)) >> np.uint64(16)) << np.uint64(16)", 0),
    ("mass-conserving mean removal dropped", "    delta = z5 - z5.mean(axis=(1, 2), keepdims=True)", "    delta = z5", 0),
    ("adjoint of the mean removal dropped", "    g5 = (g - g.mean(axis=(1, 2), keepdims=True))[:, None]",
     "    g5 = g[:, None]", 0),
]


def _replace_nth(text, old, new, nth):
    pos = -1
    for _ in range(nth + 1):
        pos = text.find(old, pos + 1)
        if pos < 0:
            raise AssertionError(f"mutation target not found (occurrence {nth}): {old!r}")
    return text[:pos] + new + text[pos + len(old):]


def _tree(tmp, pin_file, mutate=None):
    """Copy of oracle/ (sources only) and of the pin file with its conftest and golden
    values; `mutate` = (file, old, new, nth) is applied to the oracle copy."""
    src = os.path.join(ROOT, "oracle")
    dst = os.path.join(tmp, "oracle")
    os.makedirs(dst)
    for name in os.listdir(src):
        if name.endswith((".py", ".c")):
            shutil.copy(os.path.join(src, name), dst)
    if mutate:
        fname, old, new, nth = mutate
        p = os.path.join(dst, fname)
        text = open(p).read()
        open(p, "w").write(_replace_nth(text, old, new, nth))
    tdir = os.path.join(tmp, "tests")
    shutil.copytree(os.path.join(ROOT, "tests", "golden"), os.path.join(tdir, "golden"),
                    ignore=shutil.ignore_patterns("__pycache__"))
    for name in ("__init__.py", "conftest.py", pin_file):
        shutil.copy(os.path.join(ROOT, "tests", name), tdir)
    return os.path.join(tdir, pin_file)


def _run(pin_file, mutate=None):
    with tempfile.TemporaryDirectory(prefix="oracle_mut_") as tmp:
        test = _tree(tmp, pin_file, mutate)
        # one OpenMP thread per copy: several copies run at once, and spinning OpenMP
        # threads on oversubscribed cores slow a run by orders of magnitude
        env = dict(os.environ, PYTHONPATH=ROOT, OMP_NUM_THREADS="1", OMP_WAIT_POLICY="passive",
                   PYTHONDONTWRITEBYTECODE="1")
        r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider", "-m", "not gpu",
                            test], cwd=tmp, env=env, capture_output=True, text=True, timeout=600)
        return r.returncode, r.stdout[-3000:] + r.stderr[-2000:]


def _check(pin_file, fname, mutants):
    with cf.ThreadPoolExecutor(max_workers=max(2, min(8, os.cpu_count() or 2))) as ex:
        control = ex.submit(_run, pin_file)
        runs = {m[0]: ex.submit(_run, pin_file, (fname, m[1], m[2], m[3])) for m in mutants}
        rc, out = control.result()
        assert rc == 0, f"unmutated copy of the oracle fails its pins:\n{out}"
        survivors = []
        for name, fut in runs.items():
            rc, out = fut.result()
            if rc != 1 or " failed" not in out:
                survivors.append(f"{name}: exit {rc}\n{out[-1500:]}")
    assert not survivors, "mutants not caught by any pin:\n\n" + "\n\n".join(survivors)


def test_every_planted_mistake_in_the_step_oracle_fails_a_pin():
    pytest.importorskip("numpy")
    if shutil.which("gcc") is None:
        pytest.skip("gcc is needed to build the oracle copies")
    _check("test_oracle_pins.py", "lbm_ace_oracle.c", C_MUTANTS)


def test_every_planted_mistake_in_the_surrogate_oracle_fails_a_pin():
    _check("test_surrogate_oracle.py", "surrogate.py", S_MUTANTS)
