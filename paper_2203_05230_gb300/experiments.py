"""Accuracy studies on the GPU library (single-vortex benchmark of Section 3).

Everything here runs through the C ABI; numpy only computes the error measures of
the results (phi-L1/L2 against a reference field, mass drift, interface width).

* ``paper_ablation``: the paper's own run (Section 3: L = 200, R = 0.2 L at
  (0.5 L, 0.75 L), U0 = 0.04, M = 0.001, T = 6 L / U0 = 30000 steps, the sign of
  Eq. 14) for the modified ACE (Eq. 8) and the conservative-ACE ablation (Eq. 1),
  over several interface thicknesses: the relative L1 error of phi(T) against phi(0)
  (the quantity of Fig. 2, whose data the paper does not include).
* ``fp32_study``: FP32 against the FP64 GPU path over one period on the FP32
  workloads (1024^2 and 2048^2, eps in {0.5, 1, 2}, T = 16 L).
* ``precision_study``: FP64, FP32, FP16- and BF16-deviation storage on 4096^2
  (eps 1, T = 16384): phi-L2 against FP64, mass drift, interface width, speed.

* ``batch_study``: 256 lattices of uneven size in one persistent, graph-replayed
  launch per step (tiles from the autotuner) against one launch per lattice per step.
* ``surrogate_study``: the learned surrogate of 16 steps trained on 20,000 pairs that the
  GPU solver generates (625 trajectories x 32 windows on 256^2 tiles), evaluated on
  held-out trajectories against persistence, then rolled out over one period of the
  256^2 vortex with the lattice Boltzmann fallback, against the plain FP32 run.

* ``surrogate_sweep``: the rollout's error and speed against the fallback's width
  tolerance, for two training lengths.

Run: python -m paper_2203_05230_gb300.experiments
{ablation,fp32,precision,batch,surrogate,surrogate_sweep} (one GPU).
The paper's eps is 4x the eps used here (psi = eps ln(phi / (1 - phi)) as printed
in Eq. 13); tables give both.
"""
from __future__ import annotations

import json
import math
import sys
import time

import numpy as np

from . import lbm_ace as A
from . import workloads as W


def errors(phi: np.ndarray, ref: np.ndarray) -> dict:
    """Relative L1 and L2 errors of phi against ref."""
    d = phi - ref
    return {"E1": float(np.abs(d).sum() / np.abs(ref).sum()),
            "E2": float(math.sqrt((d * d).sum() / (ref * ref).sum()))}


def interface_width(phi: np.ndarray, band=(0.05, 0.95)) -> float:
    """sum phi(1 - phi) / sum |grad phi| over the nodes of the interface band (central
    differences, periodic). For the equilibrium profile 1/2 + 1/2 tanh(s / (2 eps)),
    phi(1 - phi) = eps |dphi/ds|, so the ratio is eps over any band; restricting it to
    the band keeps rounding noise in the bulk (where both sums would otherwise gather
    small contributions from millions of nodes) out of the estimate."""
    gx = 0.5 * (np.roll(phi, -1, axis=1) - np.roll(phi, 1, axis=1))
    gy = 0.5 * (np.roll(phi, -1, axis=0) - np.roll(phi, 1, axis=0))
    m = (phi > band[0]) & (phi < band[1])
    return float((phi * (1 - phi))[m].sum() / np.sqrt(gx * gx + gy * gy)[m].sum())


def run_vortex(L, *, eps, tau, U0, T, steps=None, precision=A.F64, model=A.MODEL_MODIFIED, sign=-1.0,
               R_frac=0.15, yc_frac=0.75):
    """Run the single vortex for `steps` (default T) steps; returns (phi0, phi, mass0, mass,
    seconds of the stepping)."""
    v = W.Vortex(L=L, eps=eps, tau=tau, U0=U0, T=int(T), R_frac=R_frac, yc_frac=yc_frac, sign=sign)
    phi0 = v.phi0()
    with A.Lattice(nx=L, ny=L, tau=tau, eps=eps, U0=U0, T_period=float(T), vortex_sign=sign,
                   precision=precision, model=model, phi0=phi0) as g:
        m0 = g.mass()
        g.synchronize()
        t0 = time.perf_counter()
        g.step(int(steps if steps is not None else T))
        g.synchronize()
        dt = time.perf_counter() - t0
        phi = g.phi()
        m1 = g.mass()
    return phi0, phi, m0, m1, dt


def paper_ablation(eps_paper=(1.5, 2.0, 3.0, 4.0), precision=A.F64):
    L, U0, M = 200, 0.04, 0.001
    tau = 0.5 + 3.0 * M
    T = int(round(6 * L / U0))
    rows = []
    for ep in eps_paper:
        row = {"eps_paper": ep, "eps": ep / 4}
        for name, model in (("modified", A.MODEL_MODIFIED), ("conservative", A.MODEL_CONSERVATIVE)):
            phi0, phi, m0, m1, _ = run_vortex(L, eps=ep / 4, tau=tau, U0=U0, T=T, precision=precision,
                                              model=model, sign=1.0, R_frac=0.2, yc_frac=0.75)
            e = errors(phi, phi0)
            row[name] = {"E1": e["E1"], "E2": e["E2"], "mass_drift": (m1 - m0) / m0,
                         "phi_min": float(phi.min()), "phi_max": float(phi.max())}
        rows.append(row)
    return {"study": "paper single vortex, L 200, R 40 at (100, 150), U0 0.04, M 0.001 (tau 0.503), "
                     "T 30000 steps, Eq. 14 sign; relative L1/L2 of phi(T) against phi(0)",
            "precision": int(precision), "rows": rows}


def fp32_study(sizes=(1024, 2048), eps_list=(0.5, 1.0, 2.0)):
    rows = []
    for L in sizes:
        for eps in eps_list:
            v = W.vortex_fp32(L, eps)
            kw = dict(eps=eps, tau=v.tau, U0=v.U0, T=v.T)
            phi0, p64, a0, a1, t64 = run_vortex(L, precision=A.F64, **kw)
            _, p32, b0, b1, t32 = run_vortex(L, precision=A.F32, **kw)
            rows.append({"L": L, "eps": eps, "T": v.T,
                         "fp32_vs_fp64": errors(p32, p64),
                         "shape_return_fp64": errors(p64, phi0), "shape_return_fp32": errors(p32, phi0),
                         "mass_drift_fp64": (a1 - a0) / a0, "mass_drift_fp32": (b1 - b0) / b0,
                         "mlups_fp64": L * L * v.T / t64 / 1e6, "mlups_fp32": L * L * v.T / t32 / 1e6})
    return {"study": "FP32 against the FP64 GPU path over one single-vortex period (T = 16 L)", "rows": rows}


def precision_study(L=4096, T=16384, eps=1.0):
    kw = dict(eps=eps, tau=0.8, U0=0.04, T=T)
    out = {}
    phi0 = ref = None
    for name, prec in (("f64", A.F64), ("f32", A.F32), ("f16dev", A.F16DEV), ("bf16dev", A.BF16DEV)):
        p0, phi, m0, m1, dt = run_vortex(L, precision=prec, **kw)
        if ref is None:
            phi0, ref = p0, phi
        out[name] = {"vs_fp64": errors(phi, ref), "shape_return": errors(phi, phi0),
                     "mass_drift": (m1 - m0) / m0, "width_t0": interface_width(phi0),
                     "width_T": interface_width(phi), "mlups": L * L * T / dt / 1e6}
    return {"study": f"single vortex {L}x{L}, eps {eps}, tau 0.8, U0 0.04, T {T}: storage forms against "
                     "the FP64 GPU run", "forms": out}


def _events_seconds(fn, stream):
    """Run fn() between two CUDA events on `stream` (synchronised on both sides)."""
    import torch
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    fn()
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / 1e3


def storage_forms(L=4096, T=16384, eps=1.0, speed_steps=300, accuracy=True, stream=None):
    """The 16-bit deviation forms against plain FP32 on the same lattice (the precision
    workload: single vortex, eps 1, tau 0.8, U0 0.04, period T): speed by CUDA events over
    `speed_steps` steps after a warm-up, each form in its own lattice on `stream`; with
    `accuracy`, one full period of FP64, FP32, FP16 and BF16 storage and the errors at T
    (phi-L2 against the FP64 and the FP32 runs, mass drift, interface width)."""
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    v = W.Vortex(L=L, eps=eps, T=T)
    kw = dict(nx=L, ny=L, tau=v.tau, eps=eps, U0=v.U0, T_period=float(T), vortex_sign=v.sign, phi0=v.phi0(),
              stream=s.cuda_stream)
    out = {"workload": f"single vortex {L}x{L}, eps {eps}, tau {v.tau}, U0 {v.U0}, T {T}", "speed": {}}
    for name, prec in (("f32", A.F32), ("f16dev", A.F16DEV), ("bf16dev", A.BF16DEV)):
        with A.Lattice(precision=prec, **kw) as g:
            g.step(20)
            sec = _events_seconds(lambda: g.step(speed_steps), s)
            shape = g.launch_shape()
        out["speed"][name] = {"mlups": L * L * speed_steps / sec / 1e6, "us_per_step": sec / speed_steps * 1e6,
                              "bytes_per_lup": 80 if prec == A.F32 else 44, "kernel_variant": shape[4],
                              "rows_per_cta": shape[1]}
    f32 = out["speed"]["f32"]["mlups"]
    for name in ("f16dev", "bf16dev"):
        out["speed"][name]["speedup_vs_f32"] = out["speed"][name]["mlups"] / f32
    if accuracy:
        res, phi = {}, {}
        phi0 = v.phi0()
        for name, prec in (("f64", A.F64), ("f32", A.F32), ("f16dev", A.F16DEV), ("bf16dev", A.BF16DEV)):
            with A.Lattice(precision=prec, **kw) as g:
                m0 = g.mass()
                sec = _events_seconds(lambda: g.step(T), s)
                phi[name] = g.phi()
                res[name] = {"mass_drift": (g.mass() - m0) / m0, "width_T": interface_width(phi[name]),
                             "period_seconds": sec}
        for name in res:
            res[name]["phi_l2_vs_f64"] = errors(phi[name], phi["f64"])["E2"]
            res[name]["phi_l2_vs_f32"] = errors(phi[name], phi["f32"])["E2"]
            res[name]["shape_return_phi_l2"] = errors(phi[name], phi0)["E2"]
        out["accuracy_at_T"] = res
        out["width_t0"] = interface_width(phi0)
    return out


def batch_uneven(count=256, seed=0, window=200, seq_window=20, tune_steps=2, stream=None, check=8):
    """The batched workload run to each lattice's own period: autotuned, one persistent
    graph-replayed launch per step, lattices retiring at t = T_i; aggregate MLUPS by CUDA
    events over the whole run. Then, with the ends lifted, the same `window` steps of all
    lattices as the persistent batch, as one launch per lattice per step captured in a
    graph, and (`seq_window` steps) as host-issued launches in the single-lattice
    library's launch shape. `check` lattices are compared at their T_i with the same
    lattice run alone (phi-L2) and with their initial field (shape return)."""
    import torch
    # a stream of its own: a batch given the legacy default stream would make one
    # itself, and events on the default stream would not bracket its work
    s = stream if stream is not None and stream.cuda_stream != 0 else torch.cuda.Stream()
    specs = batch_specs(count, seed)
    ends = [int(round(sp["T_period"])) for sp in specs]
    nodes = [sp["nx"] * sp["ny"] for sp in specs]
    out = {"workload": f"{count} single-vortex lattices, sides {sorted({sp['nx'] for sp in specs})}, FP32, "
                       f"each to its own period T_i in [8 L, 16 L]",
           "nodes": int(sum(nodes)), "lattice_updates": int(sum(n * e for n, e in zip(nodes, ends))),
           "max_T": max(ends)}
    rng = np.random.default_rng(seed + 1)
    picks = sorted({int(np.argmin(nodes)), int(np.argmax(nodes)),
                    *[int(i) for i in rng.choice(count, max(0, check - 2), replace=False)]})
    with A.Batch(specs, stream=s) as b:
        t0 = time.perf_counter()
        b.autotune(steps_per_trial=tune_steps)
        out["autotune_seconds"] = time.perf_counter() - t0
        out["grid"] = b.info()["grid"]
        b.set_ends()
        sec = _events_seconds(lambda: b.step(max(ends)), s)
        out["run_seconds"] = sec
        out["mlups_uneven_run"] = out["lattice_updates"] / sec / 1e6
        assert all(b.lattice_steps(i) == ends[i] for i in range(count))
        checks = []
        for i in picks:
            sp = specs[i]
            phi_b = b.phi(i)
            with A.Lattice(precision=A.F32, velocity_kind=A.VEL_SINGLE_VORTEX, stream=s.cuda_stream, **sp) as g:
                phi0 = g.phi()
                g.step(ends[i])
                ref = g.phi()
            checks.append({"lattice": i, "L": sp["nx"], "T": ends[i], "phi_l2_vs_alone": errors(phi_b, ref)["E2"],
                           "shape_return_phi_l2": errors(phi_b, phi0)["E2"]})
        out["checked_lattices"] = checks
        b.set_ends([-1] * count)
        sec_p = _events_seconds(lambda: b.step(window), s)
        sec_g = _events_seconds(lambda: b.step_per_lattice(window), s)
        sec_h = _events_seconds(lambda: b.step_sequential(seq_window), s)
    n = out["nodes"]
    out["window"] = {"steps": window, "mlups_persistent": n * window / sec_p / 1e6,
                     "mlups_per_lattice_graph": n * window / sec_g / 1e6,
                     "mlups_host_launches": n * seq_window / sec_h / 1e6, "host_launch_steps": seq_window}
    out["speedup_vs_per_lattice_graph"] = out["window"]["mlups_persistent"] / out["window"]["mlups_per_lattice_graph"]
    out["speedup_vs_host_launches"] = out["window"]["mlups_persistent"] / out["window"]["mlups_host_launches"]
    return out


def plain_fp32_fastest(L=256, eps=1.0, tau=0.8, U0=0.04, T=None, stream=None):
    """One period of the plain FP32 lattice on L x L in four launch forms, timed by CUDA
    events: per-step launches (programmatic dependent launch), the whole period captured
    in one CUDA graph, a persistent batch of one lattice (graph replays), and the
    two-steps-per-launch kernel. Returns the seconds of each and the fastest."""
    import torch
    s = torch.cuda.Stream()
    T = int(T if T else 16 * L)
    v = W.Vortex(L=L, eps=eps, tau=tau, U0=U0, T=T)
    kw = dict(nx=L, ny=L, tau=tau, eps=eps, U0=U0, T_period=float(T), vortex_sign=v.sign, phi0=v.phi0(),
              precision=A.F32, stream=s.cuda_stream)
    res = {}
    with torch.cuda.stream(s):
        with A.Lattice(**kw) as g:
            g.step(8)
            res["launches"] = _events_seconds(lambda: g.step(T), s)
        with A.Lattice(**kw) as g:
            graph = torch.cuda.CUDAGraph()
            with torch.cuda.graph(graph, stream=s):
                g.step(T)
            res["graph"] = _events_seconds(graph.replay, s)
            phi_graph = g.phi()
        with A.Lattice(**kw) as g:
            g.step(T)
            assert np.array_equal(g.phi(), phi_graph)  # the captured period is the same run
        spec = {k: kw[k] for k in ("nx", "ny", "tau", "eps", "U0", "T_period", "vortex_sign")}
        spec.update(xc=v.xc, yc=v.yc, R=v.R)
        with A.Batch([spec], stream=s) as b:
            b.autotune(steps_per_trial=8)
            b.step(8)
            res["batch_of_one"] = _events_seconds(lambda: b.step(T), s)
        with A.Lattice(kernel_variant=A.KERNEL_TWO_STEP, **kw) as g:
            g.step(8)
            res["two_steps_per_launch"] = _events_seconds(lambda: g.step(T), s)
    best = min(res, key=res.get)
    return {"L": L, "T": T, "seconds": res, "mlups": {k: L * L * T / x / 1e6 for k, x in res.items()},
            "fastest": best}


def batch_specs(count=256, seed=0):
    """The batched workload: `count` single-vortex lattices with seeded draws (sides
    from {128, ..., 1024}, centre in [0.3, 0.7] L, radius in [0.1, 0.2] L, eps in
    [0.5, 2], tau in [0.6, 1.0], U0 in [0.02, 0.05], T in [8 L, 16 L])."""
    return [dict(nx=q.L, ny=q.L, xc=q.xc, yc=q.yc, R=q.R, eps=q.eps, tau=q.tau, U0=q.U0,
                 T_period=float(q.T), vortex_sign=-1.0) for q in W.batched_instances(count, seed)]


def batch_study(count=256, steps=20, tune_steps=3):
    """Aggregate MLUPS of the persistent graph-replayed batch (after autotuning) against
    one launch per lattice per step, on the same lattices."""
    specs = batch_specs(count)
    with A.Batch(specs) as b:
        nodes = b.info()["nodes"]
        t0 = time.perf_counter()
        rows = b.autotune(steps_per_trial=tune_steps)
        tune_s = time.perf_counter() - t0
        b.step(3)
        b.synchronize()
        t0 = time.perf_counter()
        b.step(steps)
        b.synchronize()
        dt_g = time.perf_counter() - t0
        t0 = time.perf_counter()
        b.step_sequential(steps)
        dt_s = time.perf_counter() - t0
        info = b.info()
    sides = sorted({s["nx"] for s in specs})
    return {"study": f"{count} single-vortex lattices, sides {sides}, FP32", "nodes": nodes,
            "tiles": info["tiles"], "grid": info["grid"], "autotune_s": tune_s,
            "rows_by_side": {int(s["nx"]): r for s, r in zip(specs, rows)},
            "mlups_batched_graph": nodes * steps / dt_g / 1e6,
            "mlups_sequential_launches": nodes * steps / dt_s / 1e6,
            "speedup": dt_s / dt_g}


def surrogate_study(n_traj=625, pairs=32, steps=20000, batch=16, held_out=25, L=256, seed=0, lr_max=2e-3,
                    save_params=None):
    """Train the surrogate on trajectories 0 .. n_traj - held_out - 1 and report held-out
    errors, the untrained network's error, training throughput and the vortex rollout;
    the trained parameters go to the .npy file `save_params` if given."""
    import torch
    from . import surrogate as SG
    s = torch.cuda.current_stream()
    out = {"study": f"surrogate: {n_traj} trajectories x {pairs} windows of {SG.K} steps on {L}^2 "
                    f"(held out {held_out}), {steps} Adam steps of batch {batch}"}
    t0 = time.perf_counter()
    data = SG.generate(n_traj, pairs, L=L, seed=seed, stream=s)
    torch.cuda.synchronize()
    out["generate_seconds"] = time.perf_counter() - t0
    out["pairs"] = data.n_pairs
    n_train = (n_traj - held_out) * pairs
    train_idx, test_idx = np.arange(n_train), np.arange(n_train, data.n_pairs)
    with A.Net(0, s) as net:
        net.set_params(W.surrogate_init_params(seed=seed))
        tr = SG.Trainer(net, data, batch=batch, seed=seed)
        out["untrained"] = tr.evaluate(test_idx)
        t0 = time.perf_counter()
        hist = tr.train(steps, lr_max=lr_max, train_pairs=train_idx, log_every=max(1, steps // 20))
        out["train_seconds"] = time.perf_counter() - t0
        out["train_pairs_per_second"] = steps * batch / out["train_seconds"]
        out["loss_history"] = hist
        out["held_out"] = tr.evaluate(test_idx)
        out["train_subset"] = tr.evaluate(train_idx[:len(test_idx)])
        out["rollout_256"] = SG.vortex_rollout(net, L=256, stream=s)
        out["params_sha16"] = __import__("hashlib").sha256(net.get_params().tobytes()).hexdigest()[:16]
        if save_params:
            np.save(save_params, net.get_params())
    return out


def surrogate_sweep(n_traj=625, pairs=32, steps_list=(6000, 20000), batch=16, held_out=25, L=256, seed=0,
                    width_tols=(0.1, 0.05, 0.03, 0.02, 0.01)):
    """Accuracy against speed of the hybrid rollout: for each training length, the
    held-out error and one 256^2 vortex period at several interface-width tolerances of
    the fallback check (tighter tolerances send more windows to the LB solver)."""
    import torch
    from . import surrogate as SG
    s = torch.cuda.current_stream()
    data = SG.generate(n_traj, pairs, L=L, seed=seed, stream=s)
    n_train = (n_traj - held_out) * pairs
    train_idx, test_idx = np.arange(n_train), np.arange(n_train, data.n_pairs)
    out = {"study": f"hybrid rollout of the {L}^2 vortex period against the fallback's width tolerance",
           "runs": []}
    for steps in steps_list:
        with A.Net(0, s) as net:
            net.set_params(W.surrogate_init_params(seed=seed))
            tr = SG.Trainer(net, data, batch=batch, seed=seed)
            t0 = time.perf_counter()
            tr.train(steps, train_pairs=train_idx)
            run = {"adam_steps": steps, "train_seconds": time.perf_counter() - t0, "held_out": tr.evaluate(test_idx),
                   "rollouts": []}
            for wt in width_tols:
                ro = SG.vortex_rollout(net, L=L, width_tol=wt, stream=s)
                run["rollouts"].append({"width_tol": wt, **{k: ro[k] for k in (
                    "E2_vs_lbm_T", "E2_vs_lbm_half", "speedup", "surrogate_windows", "fallback_windows",
                    "max_width_dev", "mass_drift_hybrid")}})
            out["runs"].append(run)
    return out


def main(argv):
    which = argv[1] if len(argv) > 1 else "ablation"
    if which == "surrogate":
        res = surrogate_study(save_params=argv[2] if len(argv) > 2 else None)
    else:
        res = {"ablation": paper_ablation, "fp32": fp32_study, "precision": precision_study,
               "batch": batch_study, "surrogate_sweep": surrogate_sweep}[which]()
    print(json.dumps(res))


if __name__ == "__main__":
    main(sys.argv)
