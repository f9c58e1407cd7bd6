"""Pins of the surrogate oracle (CPU): each check rests on something other than the
oracle itself - brute-force loops, closed forms, published values of the normal
distribution, finite differences, the Adam update's closed form on its first step."""
import math

import numpy as np
import pytest

from oracle import surrogate as S
from paper_2203_05230_gb300 import workloads as W


def brute_conv(x, Wt, b):
    B, ci, H, Wd = x.shape
    co = Wt.shape[0]
    out = np.zeros((B, co, H, Wd))
    for n in range(B):
        for o in range(co):
            for y in range(H):
                for xx in range(Wd):
                    s = b[o]
                    for c in range(ci):
                        for j in range(3):
                            for i in range(3):
                                s += Wt[o, c, j, i] * x[n, c, (y + j - 1) % H, (xx + i - 1) % Wd]
                    out[n, o, y, xx] = s
    return out


def test_conv_matches_brute_force():
    rng = np.random.default_rng(1)
    x = rng.standard_normal((2, 3, 4, 5))
    Wt = rng.standard_normal((2, 3, 3, 3))
    b = rng.standard_normal(2)
    assert np.allclose(S.conv3x3(x, Wt, b), brute_conv(x, Wt, b), rtol=0, atol=1e-12)


@pytest.mark.parametrize("j,i", [(0, 0), (0, 2), (1, 2), (2, 1), (2, 2)])
def test_conv_delta_kernel_is_a_shift(j, i):
    rng = np.random.default_rng(2)
    x = rng.standard_normal((1, 1, 6, 7))
    Wt = np.zeros((1, 1, 3, 3))
    Wt[0, 0, j, i] = 1.0
    # out[y, x] = in[y + j - 1, x + i - 1]
    ref = np.roll(x, shift=(1 - j, 1 - i), axis=(2, 3))
    assert np.array_equal(S.conv3x3(x, Wt, np.zeros(1)), ref)
    assert S.conv3x3(x, Wt, np.zeros(1))[0, 0, 0, 0] == x[0, 0, (j - 1) % 6, (i - 1) % 7]


def test_conv_input_grad_is_the_adjoint():
    rng = np.random.default_rng(3)
    x = rng.standard_normal((2, 3, 5, 4))
    g = rng.standard_normal((2, 4, 5, 4))
    Wt = rng.standard_normal((4, 3, 3, 3))
    lhs = (S.conv3x3(x, Wt, np.zeros(4)) * g).sum()
    rhs = (x * S.conv3x3_input_grad(g, Wt)).sum()
    assert abs(lhs - rhs) < 1e-11 * abs(lhs)


def test_gelu_values():
    # Phi(1) = 0.8413447460685429, Phi(-1) = 0.15865525393145707 (standard normal CDF)
    assert S.gelu(np.array([0.0]))[0] == 0.0
    assert abs(S.gelu(np.array([1.0]))[0] - 0.8413447460685429) < 1e-15
    assert abs(S.gelu(np.array([-1.0]))[0] + 0.15865525393145707) < 1e-15
    z = np.linspace(-6, 6, 101)
    assert np.allclose(S.gelu(z) - S.gelu(-z), z, rtol=0, atol=1e-14)   # z Phi(z) + z Phi(-z) = z
    assert abs(S.gelu_grad(np.array([0.0]))[0] - 0.5) < 1e-16
    h = 1e-6
    fd = (S.gelu(z + h) - S.gelu(z - h)) / (2 * h)
    assert np.allclose(S.gelu_grad(z), fd, rtol=0, atol=1e-8)


def test_bf16_rounding():
    one = 1.0
    assert S.bf16(np.array([one]))[0] == 1.0
    assert S.bf16(np.array([1 + 2 ** -7]))[0] == 1 + 2 ** -7          # representable
    assert S.bf16(np.array([1 + 2 ** -8]))[0] == 1.0                  # tie -> even (mantissa 0)
    assert S.bf16(np.array([1 + 3 * 2 ** -8]))[0] == 1 + 2 ** -6      # tie -> even (mantissa 2)
    assert S.bf16(np.array([1 + 2 ** -8 + 2 ** -12]))[0] == 1 + 2 ** -7
    assert S.bf16(np.array([-3.5]))[0] == -3.5
    x = np.random.default_rng(4).standard_normal(10000) * 100
    r = S.bf16(x)
    assert np.all(np.abs(r - x) <= 2 ** -8 * np.abs(x) * (1 + 1e-6))   # unit roundoff of an 8-bit significand
    assert np.array_equal(S.bf16(r), r)


def small_problem(widths, B=2, H=5, Wd=6, seed=5):
    rng = np.random.default_rng(seed)
    flat = rng.standard_normal(S.param_count(widths)) * 0.4
    phi = rng.uniform(0, 1, (B, H, Wd))
    u = rng.uniform(-0.05, 0.05, (B, H, Wd))
    v = rng.uniform(-0.05, 0.05, (B, H, Wd))
    tgt = phi + rng.standard_normal((B, H, Wd)) * 0.1
    return flat, phi, u, v, tgt


def test_mass_is_conserved():
    flat, phi, u, v, _ = small_problem(S.WIDTHS, B=3, H=8, Wd=8)
    out, _ = S.forward(flat, phi, u, v)
    assert np.allclose(out.sum(axis=(1, 2)), phi.sum(axis=(1, 2)), rtol=1e-13, atol=0)


def test_translation_equivariance():
    flat, phi, u, v, _ = small_problem(S.WIDTHS, B=1, H=7, Wd=9)
    out, _ = S.forward(flat, phi, u, v)
    r = lambda a: np.roll(a, shift=(2, -3), axis=(1, 2))
    out2, _ = S.forward(flat, r(phi), r(u), r(v))
    assert np.abs(out2 - r(out)).max() < 1e-13 * np.abs(out).max()


def test_gradient_matches_finite_differences_all_parameters():
    widths = (3, 4, 4, 4, 4, 1)
    flat, phi, u, v, tgt = small_problem(widths)
    L0, g, _ = S.loss_and_grad(flat, phi, u, v, tgt, widths)
    h = 1e-6
    fd = np.empty_like(flat)
    for k in range(flat.size):
        e = np.zeros_like(flat)
        e[k] = h
        lp = S.loss_value(S.forward(flat + e, phi, u, v, widths)[0], tgt)
        lm = S.loss_value(S.forward(flat - e, phi, u, v, widths)[0], tgt)
        fd[k] = (lp - lm) / (2 * h)
    scale = np.abs(g).max()
    assert np.abs(g - fd).max() < 1e-6 * scale, np.abs(g - fd).max() / scale


def test_gradient_matches_finite_differences_full_width():
    flat, phi, u, v, tgt = small_problem(S.WIDTHS, B=1, H=4, Wd=5, seed=6)
    flat = W.surrogate_init_params(seed=3) * 3.0
    _, g, _ = S.loss_and_grad(flat, phi, u, v, tgt)
    rng = np.random.default_rng(7)
    # sample every layer's weights and biases
    offs, k = [], 0
    for shp in S.param_shapes():
        n = int(np.prod(shp))
        offs.extend(k + rng.choice(n, size=min(n, 6), replace=False))
        k += n
    h = 1e-6
    for k in offs:
        e = np.zeros_like(flat)
        e[k] = h
        lp = S.loss_value(S.forward(flat + e, phi, u, v)[0], tgt)
        lm = S.loss_value(S.forward(flat - e, phi, u, v)[0], tgt)
        fd = (lp - lm) / (2 * h)
        assert abs(g[k] - fd) < 1e-6 * np.abs(g).max() + 1e-7 * abs(fd), (k, g[k], fd)


def test_emulated_storage_error_is_bf16_sized():
    flat = W.surrogate_init_params(seed=1)
    flat[-289:] *= 30.0  # make the output layer matter
    _, phi, u, v, tgt = small_problem(S.WIDTHS, B=1, H=8, Wd=8)
    a, _ = S.forward(flat, phi, u, v)
    b, _ = S.forward(flat, phi, u, v, emulate=True)
    d, db = a - phi, b - phi
    rel = np.sqrt(((d - db) ** 2).sum() / (d ** 2).sum())
    assert 1e-3 < rel < 1e-2
    _, ga, _ = S.loss_and_grad(flat, phi, u, v, tgt)
    _, gb, _ = S.loss_and_grad(flat, phi, u, v, tgt, emulate=True)
    # BF16 storage at about eight points of the pass: 5.5e-3 (forward) and 6.7e-3
    # (gradient) measured here, sqrt(8) x 2^-9 / sqrt(3) = 3.2e-3 before amplification
    assert np.linalg.norm(ga - gb) < 1.5e-2 * np.linalg.norm(ga)


def test_adam_first_step_closed_form():
    rng = np.random.default_rng(8)
    p = rng.standard_normal(50)
    g = rng.standard_normal(50)
    lr, eps = 1e-3, 1e-8
    p1, m, v = S.adam(p, g, np.zeros(50), np.zeros(50), 1, lr, eps=eps)
    # bias-corrected m = g and v = g^2 on the first step: update lr g / (|g| + eps)
    assert np.allclose(p1, p - lr * g / (np.abs(g) + eps), rtol=0, atol=1e-15)
    assert np.allclose(m, 0.1 * g) and np.allclose(v, 0.001 * g * g)
    p2, _, _ = S.adam(p, np.zeros(50), np.zeros(50), np.zeros(50), 1, lr)
    assert np.array_equal(p2, p)


def test_adam_minimises_a_quadratic():
    p, m, v = np.array([0.0, 10.0]), np.zeros(2), np.zeros(2)
    for t in range(1, 3001):
        p, m, v = S.adam(p, p - np.array([3.0, -2.0]), m, v, t, 0.05)
    assert np.allclose(p, [3.0, -2.0], atol=1e-3)


def test_width_estimator_on_the_profile():
    for eps in (1.0, 2.0):
        phi = W.disk_phi0(128, 128, 64.0, 64.0, 30.0, eps)
        assert abs(S.interface_width(phi) / eps - 1) < 0.015 / eps ** 2


def test_surrogate_inputs_are_divergence_free_and_bounded():
    rng = np.random.Generator(np.random.PCG64(0))
    u, v = W.mode_field(64, rng)
    assert np.sqrt(u * u + v * v).max() <= 0.05 + 1e-15
    # spectral divergence of an exact sum of Fourier modes vanishes
    k = np.fft.fftfreq(64) * 2 * math.pi
    div = np.fft.ifft2(1j * k[None, :] * np.fft.fft2(u) + 1j * k[:, None] * np.fft.fft2(v)).real
    assert np.abs(div).max() < 1e-14
    phi = W.circles_phi0(64, rng)
    assert phi.min() >= 0 and phi.max() <= 1
