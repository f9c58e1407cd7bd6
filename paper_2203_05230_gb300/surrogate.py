"""Learned surrogate of K = 16 lattice Boltzmann steps: data, training, hybrid rollout.

Everything that computes runs in the library's kernels through the C ABI
(include/lbm_ace_surrogate.h): the training pairs come from the GPU lattice Boltzmann
solver (``Lattice`` with a static divergence-free field), the network is trained by the
library's own forward, backward and Adam kernels, and the rollout is the library's
hybrid advance with the lattice Boltzmann fallback. PyTorch only provides device memory
and the stream; numpy computes the error measures of results copied to the host.

Training workload (seeded): trajectories on 256 x 256 periodic tiles start from 1-4
circles (radius 0.05-0.2 L, eps 1, tau 0.8) in a frozen field built from 4 random
stream-function modes with max |u| <= 0.05; phi is recorded every K = 16 steps, and
consecutive snapshots form the (input, target) pairs.
"""
from __future__ import annotations

import math
import time

import numpy as np

from . import lbm_ace as A
from . import workloads as W

K = A.NET_K


def _torch():
    import torch
    if not torch.cuda.is_available():
        raise A.LbmAceError(A.ECUDA, "the surrogate needs a CUDA device")
    return torch


class Dataset:
    """Snapshots phi[traj, k] (k = 0..pairs) and fields u[traj], v[traj] on the device."""

    def __init__(self, snaps, u, v, pairs):
        self.snaps, self.u, self.v, self.pairs = snaps, u, v, pairs
        self.n_traj, self.L = snaps.shape[0], snaps.shape[-1]

    @property
    def n_pairs(self):
        return self.n_traj * self.pairs


def generate(n_traj: int, pairs: int, L: int = W.SURROGATE_TILE, seed: int = 0, tau: float = 0.8,
             eps: float = 1.0, stream=None) -> Dataset:
    """Run the GPU lattice Boltzmann solver (FP32) for `pairs` windows of K steps on each
    of `n_traj` seeded trajectory starts; returns the device dataset."""
    torch = _torch()
    dev = torch.device("cuda")
    snaps = torch.empty((n_traj, pairs + 1, L, L), dtype=torch.float32, device=dev)
    u = torch.empty((n_traj, L, L), dtype=torch.float32, device=dev)
    v = torch.empty((n_traj, L, L), dtype=torch.float32, device=dev)
    s = stream if stream is not None else torch.cuda.current_stream()
    for t, (phi0, uu, vv) in enumerate(W.surrogate_trajectories(n_traj, L, seed)):
        with A.Lattice(nx=L, ny=L, tau=tau, eps=eps, precision=A.F32, velocity_kind=A.VEL_FIELD,
                       u_field=uu, v_field=vv, phi0=phi0, stream=s) as g:
            g.lbm_ace_velocity_device(0.0, u[t].data_ptr(), v[t].data_ptr())
            for k in range(pairs + 1):
                if k:
                    g.step(K)
                g.lbm_ace_get_phi_device(snaps[t, k].data_ptr())
            g.synchronize()
    return Dataset(snaps, u, v, pairs)


class Trainer:
    """Minibatch Adam on (snapshot k, snapshot k + 1) pairs of a Dataset."""

    def __init__(self, net: A.Net, data: Dataset, batch: int = 16, seed: int = 0):
        torch = _torch()
        self.net, self.data, self.batch = net, data, batch
        L = data.L
        dev = torch.device("cuda")
        self.buf = {k: torch.empty((batch, L, L), dtype=torch.float32, device=dev) for k in ("phi", "tgt", "u", "v")}
        self.rng = np.random.Generator(np.random.PCG64(seed))

    def _load(self, pairs_idx):
        d, L = self.data, self.data.L
        traj, k = pairs_idx // d.pairs, pairs_idx % d.pairs
        snap_idx = traj * (d.pairs + 1) + k
        n = self.net
        n.gather(self.buf["phi"], d.snaps, snap_idx, L * L)
        n.gather(self.buf["tgt"], d.snaps, snap_idx + 1, L * L)
        n.gather(self.buf["u"], d.u, traj, L * L)
        n.gather(self.buf["v"], d.v, traj, L * L)

    def step(self, pairs_idx, lr: float, want_loss: bool = False):
        b = self.buf
        self._load(pairs_idx)
        loss, _ = self.net.loss_grad(b["phi"], b["u"], b["v"], b["tgt"], len(pairs_idx), self.data.L, self.data.L,
                                     want_loss=want_loss)
        self.net.adam(lr)
        return loss

    def train(self, steps: int, lr_max: float = 2e-3, lr_min: float = 2e-5, train_pairs=None, log_every: int = 0):
        """Cosine-decayed learning rate; minibatches drawn from train_pairs (default all)."""
        pool = np.arange(self.data.n_pairs) if train_pairs is None else np.asarray(train_pairs)
        hist = []
        for s in range(steps):
            lr = lr_min + 0.5 * (lr_max - lr_min) * (1 + math.cos(math.pi * s / max(1, steps)))
            idx = self.rng.choice(pool, size=self.batch, replace=False)
            want = bool(log_every) and (s % log_every == 0 or s == steps - 1)
            loss = self.step(idx, lr, want_loss=want)
            if want:
                hist.append((s, loss))
        self.net.synchronize()
        return hist

    def evaluate(self, pairs_idx):
        """Relative L2 error of the network and of persistence (phi(t + K) ~ phi(t))
        against the lattice Boltzmann targets, and of the predicted increment."""
        torch = _torch()
        b, L = self.buf, self.data.L
        err_n = err_p = ref = inc = 0.0
        out = torch.empty((self.batch, L, L), dtype=torch.float32, device="cuda")
        idx = np.asarray(pairs_idx)
        for s in range(0, len(idx), self.batch):
            chunk = idx[s:s + self.batch]
            self._load(chunk)
            self.net.forward(b["phi"], b["u"], b["v"], out, len(chunk), L, L)
            self.net.synchronize()
            o = out[:len(chunk)].cpu().numpy().astype(np.float64)
            p = b["phi"][:len(chunk)].cpu().numpy().astype(np.float64)
            t = b["tgt"][:len(chunk)].cpu().numpy().astype(np.float64)
            err_n += ((o - t) ** 2).sum()
            err_p += ((p - t) ** 2).sum()
            ref += (t ** 2).sum()
            inc += ((t - p) ** 2).sum()
        return {"E2_net": math.sqrt(err_n / ref), "E2_persistence": math.sqrt(err_p / ref),
                "increment_rel_err": math.sqrt(err_n / inc)}


def vortex_rollout(net: A.Net, L: int = 256, eps: float = 1.0, tau: float = 0.8, U0: float = 0.04, T=None,
                   mass_tol: float = 1e-6, width_tol: float = 0.1, stream=None):
    """One period of the single vortex (Section 3) on L x L: the plain FP32 lattice
    Boltzmann run against the hybrid advance (surrogate windows, LB fallback); returns
    phi-L2 between the two at t = T and at T/2, mass drift, widths and wall times."""
    torch = _torch()
    T = int(T if T else 16 * L)
    windows = T // K
    s = stream if stream is not None else torch.cuda.current_stream()
    v = W.Vortex(L=L, eps=eps, tau=tau, U0=U0, T=T)
    phi0 = v.phi0()
    kw = dict(nx=L, ny=L, tau=tau, eps=eps, U0=U0, T_period=float(T), vortex_sign=-1.0, precision=A.F32,
              phi0=phi0, stream=s)
    res = {}
    half = windows // 2 * K
    with A.Lattice(**kw) as ref:
        m0 = ref.mass()
        ref.step(half)
        half_ref = ref.phi()
        ref.step(T - half)
        phi_ref = ref.phi()
    with A.Lattice(**kw) as hy:
        st1 = net.hybrid_advance(hy, windows // 2, mass_tol, width_tol)
        half_hy = hy.phi()
        st2 = net.hybrid_advance(hy, windows - windows // 2, mass_tol, width_tol)
        phi_hy = hy.phi()
        m1 = hy.mass()
    # wall time of one period, each on a fresh lattice
    with A.Lattice(**kw) as g:
        g.synchronize()
        t0 = time.perf_counter()
        g.step(T)
        g.synchronize()
        res["lbm_seconds"] = time.perf_counter() - t0
    with A.Lattice(**kw) as g:
        g.synchronize()
        t0 = time.perf_counter()
        net.hybrid_advance(g, windows, mass_tol, width_tol)
        g.synchronize()
        res["hybrid_seconds"] = time.perf_counter() - t0
    res["speedup"] = res["lbm_seconds"] / res["hybrid_seconds"]
    # end to end through the public API: lattice built from the host phi0, the period,
    # phi read back to the host
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    with A.Lattice(**kw) as g:
        net.hybrid_advance(g, windows, mass_tol, width_tol)
        g.phi()
    res["hybrid_e2e_seconds"] = time.perf_counter() - t0

    def e2(a, b):
        return math.sqrt(((a - b) ** 2).sum() / (b ** 2).sum())

    res.update({
        "L": L, "T": T, "windows": windows,
        "E2_vs_lbm_T": e2(phi_hy, phi_ref), "E2_vs_lbm_half": e2(half_hy, half_ref),
        "E2_lbm_shape_return": e2(phi_ref, phi0), "E2_hybrid_shape_return": e2(phi_hy, phi0),
        "mass_drift_hybrid": (m1 - m0) / m0,
        "surrogate_windows": st1["surrogate_windows"] + st2["surrogate_windows"],
        "fallback_windows": st1["fallback_windows"] + st2["fallback_windows"],
        "max_width_dev": max(st1["max_width_dev"], st2["max_width_dev"]),
    })
    return res
