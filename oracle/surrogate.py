"""FP64 CPU oracle of the learned surrogate (TEST INFRASTRUCTURE ONLY).

Plain numpy, written from the definitions, for checking the CUDA surrogate kernels.
Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU legs may import it;
it shares no code with the CUDA library.

The paper has no learned component. The surrogate advances the phase field of
the single-vortex problem (Section 3) by K = 16 lattice Boltzmann steps in one
application:

    x0  = (phi, 20 u, 20 v)                                 three input channels
    z_l = conv3x3(a_{l-1}, W_l) + b_l,  a_l = GELU(z_l)     l = 1 .. 4, width 32
    z_5 = conv3x3(a_4, W_5) + b_5                           one channel
    phi_out = phi + z_5 - mean(z_5)                         per tile

* conv3x3 is the cross-correlation of deep-learning practice on a periodic
  lattice: out[co, y, x] = b[co] + sum_{ci, j, i} W[co, ci, j, i] in[ci, y+j-1, x+i-1],
  indices taken modulo the tile (the lattices are periodic, Section 3).
* GELU(z) = z Phi(z) with Phi the standard normal CDF (Hendrycks and Gimpel, 2016),
  written with erf.
* Subtracting the tile mean of z_5 keeps sum(phi) unchanged, the global mass
  conservation of the conservative ACE (Eq. 8 is in divergence form).
* The loss is the mean squared error over all nodes of the batch; its gradient
  is taken analytically, layer by layer (chain rule), and pinned against
  central finite differences.
* Adam follows Kingma and Ba (2015), Algorithm 1, with bias correction.

Parameters travel as one flat vector in the order W_1, b_1, ..., W_5, b_5, each W in
[co][ci][j][i] order (j the row offset, i the column offset, both 0..2); this is the
interchange format of the C library's ``lbm_ace_net_set_params``.

``emulate=True`` rounds to BF16 (round to nearest even, through FP32) exactly where the
CUDA path stores BF16: the weights of layers 2-5 (tensor-core operands), the stored z_l
and a_l of layers 1-4 and the back-propagated dL/dz_l of layers 1-4. Layer 1, which the
CUDA path runs on FP32 units, keeps FP32 weights. This makes the comparison with the
GPU a test of the arithmetic, not of the storage precision; the pure FP64 mode gives
the storage error.
"""
from __future__ import annotations

import math

import numpy as np

WIDTHS = (3, 32, 32, 32, 32, 1)
U_SCALE = 20.0        # velocity input scale: 1 / 0.05, the largest |u| of the training fields
K_STEPS = 16          # LB steps per application


# --- parameters --------------------------------------------------------------

def param_shapes(widths=WIDTHS):
    out = []
    for ci, co in zip(widths[:-1], widths[1:]):
        out.append((co, ci, 3, 3))
        out.append((co,))
    return out


def param_count(widths=WIDTHS) -> int:
    return int(sum(np.prod(s) for s in param_shapes(widths)))


def unpack(flat, widths=WIDTHS):
    """Flat vector -> list of (W, b) per layer (views, float64)."""
    flat = np.asarray(flat, dtype=np.float64)
    assert flat.size == param_count(widths), (flat.size, param_count(widths))
    layers, k = [], 0
    shapes = param_shapes(widths)
    for w_s, b_s in zip(shapes[0::2], shapes[1::2]):
        nw, nb = int(np.prod(w_s)), int(np.prod(b_s))
        layers.append((flat[k:k + nw].reshape(w_s), flat[k + nw:k + nw + nb].reshape(b_s)))
        k += nw + nb
    return layers


def pack(layers) -> np.ndarray:
    return np.concatenate([np.concatenate([W.ravel(), b.ravel()]) for W, b in layers])


# --- elementary operations -----------------------------------------------------

def bf16(x):
    """Round to the nearest BF16 value (ties to even) via FP32; returns float64."""
    f = np.asarray(x, dtype=np.float32)
    bits = f.view(np.uint32).astype(np.uint64)
    lsb = (bits >> np.uint64(16)) & np.uint64(1)
    r = ((bits + np.uint64(0x7FFF) + lsb) >> np.uint64(16)) << np.uint64(16)
    return (r.astype(np.uint32).view(np.float32)).astype(np.float64)


def f32(x):
    return np.asarray(x, dtype=np.float32).astype(np.float64)


def conv3x3(x, W, b):
    """Periodic 3x3 cross-correlation. x [B, ci, H, W], W [co, ci, 3, 3], b [co]."""
    B, ci, H, Wd = x.shape
    co = W.shape[0]
    out = np.broadcast_to(b.reshape(1, co, 1, 1), (B, co, H, Wd)).astype(np.float64).copy()
    for j in range(3):
        for i in range(3):
            # shifted[..., y, x] = x[..., y + j - 1, x + i - 1]
            shifted = np.roll(x, shift=(1 - j, 1 - i), axis=(2, 3))
            out += np.einsum("oc,bchw->bohw", W[:, :, j, i], shifted)
    return out


def conv3x3_input_grad(g, W):
    """Adjoint of conv3x3 with respect to its input: d/dx of sum(g * conv3x3(x, W, 0))."""
    B, co, H, Wd = g.shape
    ci = W.shape[1]
    out = np.zeros((B, ci, H, Wd))
    for j in range(3):
        for i in range(3):
            # x[y', x'] meets g[y' - j + 1, x' - i + 1]
            out += np.roll(np.einsum("oc,bohw->bchw", W[:, :, j, i], g), shift=(j - 1, i - 1), axis=(2, 3))
    return out


def conv3x3_weight_grad(g, x):
    """d/dW of sum(g * conv3x3(x, W, b)): [co, ci, 3, 3]; and d/db: [co]."""
    co, ci = g.shape[1], x.shape[1]
    dW = np.zeros((co, ci, 3, 3))
    for j in range(3):
        for i in range(3):
            shifted = np.roll(x, shift=(1 - j, 1 - i), axis=(2, 3))
            dW[:, :, j, i] = np.einsum("bohw,bchw->oc", g, shifted)
    return dW, g.sum(axis=(0, 2, 3))


try:
    from scipy.special import erf as _erf
except ImportError:  # pragma: no cover - scipy is present on both machines
    _erf = np.vectorize(math.erf, otypes=[np.float64])


def gelu(z):
    z = np.asarray(z, dtype=np.float64)
    return 0.5 * z * (1.0 + _erf(z / math.sqrt(2.0)))


def gelu_grad(z):
    """d GELU / dz = Phi(z) + z phi(z), phi the standard normal density."""
    z = np.asarray(z, dtype=np.float64)
    erf = _erf
    return 0.5 * (1.0 + erf(z / math.sqrt(2.0))) + z * np.exp(-0.5 * z * z) / math.sqrt(2.0 * math.pi)


# --- network -------------------------------------------------------------------

def _inputs(phi, u, v):
    phi = np.asarray(phi, dtype=np.float64)
    if phi.ndim == 2:
        phi, u, v = phi[None], np.asarray(u)[None], np.asarray(v)[None]
    return np.stack([phi, np.asarray(u, np.float64) * U_SCALE, np.asarray(v, np.float64) * U_SCALE], axis=1)


def _weights(flat, widths, emulate):
    layers = unpack(flat, widths)
    if not emulate:
        return layers
    out = []
    for l, (W, b) in enumerate(layers):
        rw = f32 if l == 0 else bf16
        out.append((rw(W), f32(b)))
    return out


def forward(flat, phi, u, v, widths=WIDTHS, emulate=False):
    """phi_out [B, H, W] and the cache for ``backward``. phi, u, v: [B, H, W] or [H, W]."""
    x0 = _inputs(phi, u, v)
    if emulate:
        x0 = f32(x0)
    layers = _weights(flat, widths, emulate)
    rnd = bf16 if emulate else (lambda a: a)
    a = x0
    zs, acts = [], [x0]
    for W, b in layers[:-1]:
        z = conv3x3(a, W, b)
        zr = rnd(z)
        a = rnd(gelu(z))
        zs.append(zr)
        acts.append(a)
    W5, b5 = layers[-1]
    z5 = conv3x3(a, W5, b5)[:, 0]
    delta = z5 - z5.mean(axis=(1, 2), keepdims=True)
    out = x0[:, 0] + delta
    return out, {"layers": layers, "zs": zs, "acts": acts, "emulate": emulate}


def loss_value(phi_out, target) -> float:
    d = phi_out - np.asarray(target, dtype=np.float64).reshape(phi_out.shape)
    return float((d * d).mean())


def backward(cache, phi_out, target):
    """Gradient of the mean squared error with respect to the flat parameter vector."""
    layers, zs, acts, emulate = cache["layers"], cache["zs"], cache["acts"], cache["emulate"]
    rnd = bf16 if emulate else (lambda a: a)
    target = np.asarray(target, dtype=np.float64).reshape(phi_out.shape)
    N = phi_out.size
    g = 2.0 * (phi_out - target) / N                                   # dL/dphi_out
    g5 = (g - g.mean(axis=(1, 2), keepdims=True))[:, None]            # through the mean removal
    grads = [None] * len(layers)
    grads[-1] = conv3x3_weight_grad(g5, acts[-1])
    gz = g5
    for l in range(len(layers) - 1, 0, -1):                          # layer l+1 -> dL/dz_l
        da = conv3x3_input_grad(gz, layers[l][0])
        gz = rnd(da * gelu_grad(zs[l - 1]))
        grads[l - 1] = conv3x3_weight_grad(gz, acts[l - 1])
    return pack(grads)


def loss_and_grad(flat, phi, u, v, target, widths=WIDTHS, emulate=False):
    out, cache = forward(flat, phi, u, v, widths, emulate)
    return loss_value(out, target), backward(cache, out, target), out


def adam(flat, grad, m, v, step, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update (Kingma and Ba, 2015, Algorithm 1); step counts from 1.
    Returns (new parameters, m, v)."""
    m = beta1 * m + (1.0 - beta1) * grad
    v = beta2 * v + (1.0 - beta2) * grad * grad
    mh = m / (1.0 - beta1 ** step)
    vh = v / (1.0 - beta2 ** step)
    return flat - lr * mh / (np.sqrt(vh) + eps), m, v


# --- fallback checks -------------------------------------------------------------

def mass(phi) -> float:
    return float(np.asarray(phi, dtype=np.float64).sum())


def interface_width(phi, band=(0.05, 0.95)) -> float:
    """sum phi(1 - phi) / sum |grad phi| over the band nodes (central differences,
    periodic). For the equilibrium profile 1/2 + 1/2 tanh(s / (2 eps)) of Eq. 2 (with
    the thickness convention of the library) phi(1 - phi) = eps |dphi/ds|, so the ratio
    estimates eps."""
    phi = np.asarray(phi, dtype=np.float64)
    gx = 0.5 * (np.roll(phi, -1, axis=-1) - np.roll(phi, 1, axis=-1))
    gy = 0.5 * (np.roll(phi, -1, axis=-2) - np.roll(phi, 1, axis=-2))
    m = (phi > band[0]) & (phi < band[1])
    return float((phi * (1 - phi))[m].sum() / np.sqrt(gx * gx + gy * gy)[m].sum())
