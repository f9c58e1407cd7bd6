#!/usr/bin/env python3
"""Benchmark of the fused lattice Boltzmann step (modified conservative ACE, D2Q9).

Workload: the single-vortex benchmark (Section 3, Eq. 14) on a periodic
2048 x 2048 lattice, FP32 populations, eps 1, tau 0.8, U0 0.04, T = 16 L steps,
disk R = 0.15 L at (0.5 L, 0.75 L). One bench step is one lattice time step (one
launch of the fused step kernel). Its working set (2 x 151 MB population
buffers + a 16.8 MB phi plane) is larger than the 126 MB L2, so no flush is
needed between steps.

Prints one JSON line. ``--impl reference`` times the FP64 CPU oracle instead (on
the host cores, a bounded sample per step). Under torchrun each rank runs an
independent replica of the workload on its own GPU (no collective on the data
path); the line reports the aggregate over ranks.

``--surrogate`` measures the learned surrogate instead (one GPU): the forward pass on a
batch of 256 x 256 images (CUDA events, the tensor-core roofline of its algorithmic
FLOPs), and, after training it on GPU-generated pairs, one period of the 256 x 256
single vortex advanced by the hybrid (surrogate windows of 16 steps with the lattice
Boltzmann fallback) against the plain FP32 lattice Boltzmann run: wall-clock MLUPS of
both and the phi-L2 error between them.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "MLUPS"
KERNEL_NAME = {1: "ace_step", 2: "ace_step_bulk", 3: "ace_step_warp", 4: "ace_step_pair", 5: "ace_step_dev",
               6: "ace_step_tb2", 7: "ace_step_dev4", 8: "ace_step_quad"}
STEPS_PER_LAUNCH = {6: 2}   # the two-step kernel: one launch advances two steps
BYTES_PER_LUP = {"f64": 160, "f32": 80, "f16dev": 44, "bf16dev": 44}
HBM_NOMINAL_GBS = 7900.0  # GB300 HBM3e, nominal (context beside the measured copy peak)
# arithmetic type of each storage form: the 16-bit deviation forms compute in FP32
ARITH_DTYPE = {"f64": "f64", "f32": "f32", "f16dev": "f32", "bf16dev": "f32"}
# FP64 step: 204 FP64 FLOP per node update (55.5 DFMA counted twice, 53.4 DADD, 40.0 DMUL;
# ncu op counters of ace_step_pair<double>), bound by the FP64 pipe rather than by HBM.
# Peak: GB300's nominal FP64 rate, 152 SMs x 2.07 GHz x 4 FLOP per clock = 1.259 TFLOP/s
# (an FMA-chain probe measured 1.256).
F64_FLOP_PER_LUP = 204.0
F64_PEAK_TFLOPS = 152 * 2.07e9 * 4 / 1e12
L2_BYTES = 126e6  # GB300's L2 as the runtime reports it (cudaDevAttrL2CacheSize), about 126 MB


def l2_note(L: int, precision: str) -> str:
    """How the timed steps relate to the L2: the state's buffers and whether one population
    buffer (what a step streams in) is larger than the L2."""
    n = L * L
    if precision in ("f32", "f64"):
        e = 4 if precision == "f32" else 8
        pop, parts = 9 * n * e, f"2 x {9 * n * e / 1e6:.1f} MB {precision.upper()} population buffers + " \
                                 f"{n * e / 1e6:.1f} MB phi plane"
        total = 19 * n * e
    else:
        pop, parts = 18 * n, f"2 x {18 * n / 1e6:.1f} MB 16-bit deviation buffers + 2 x {4 * n / 1e6:.1f} MB phi planes"
        total = 44 * n
    if pop > L2_BYTES:
        return "inputs larger than L2: " + parts
    if total <= L2_BYTES:
        return f"state fits in L2 ({total / 1e6:.1f} MB: {parts}); no flush between steps: the L2-resident steady state"
    return (f"state larger than L2 ({total / 1e6:.1f} MB: {parts}) but one population buffer smaller; no flush "
            "between steps: part of a step's reads hit in L2")


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--L", type=int, default=2048)
    ap.add_argument("--precision", default="f32", choices=["f32", "f64", "f16dev", "bf16dev"])
    ap.add_argument("--rows", type=int, default=0, help="rows per CTA (0: library default)")
    ap.add_argument("--variant", type=int, default=0, help="step kernel: 0 auto, 1 direct loads, 2 bulk-copy pipeline, 3 independent warps, 4 column pairs, "
                    "6 two steps per launch; 16-bit storage: 5 column pairs, 7 column quads")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--surrogate", action="store_true", help="benchmark the learned surrogate instead")
    ap.add_argument("--surr-batch", type=int, default=16, help="images per timed forward (surrogate mode)")
    ap.add_argument("--surr-traj", type=int, default=625,
                    help="training trajectories of 32 windows (surrogate mode; 0: forward timing only)")
    ap.add_argument("--surr-train-steps", type=int, default=20000)
    ap.add_argument("--no-forms", action="store_true",
                    help="skip the record of the 16-bit, batched and surrogate forms against plain FP32")
    ap.add_argument("--forms-train-steps", type=int, default=20000,
                    help="Adam steps of the surrogate trained inside the forms record")
    return ap.parse_args()


def workload(args):
    from paper_2203_05230_gb300 import workloads as W
    v = W.vortex_fp32(args.L)
    return v, {
        "workload": f"single vortex {args.L}x{args.L} {args.precision.upper()} eps {v.eps} tau {v.tau} "
                    f"U0 {v.U0} T {v.T} steps, disk R {v.R:g} at ({v.xc:g}, {v.yc:g})",
        "lattice": [args.L, args.L], "T_period": v.T, "eps": v.eps, "tau": v.tau, "U0": v.U0,
        "l2": l2_note(args.L, args.precision),
    }


def dist_setup():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def max_over_ranks(secs: float, ws: int, device=None) -> float:
    """The job's time is the slowest replica's: MAX over the ranks of the process group
    (a no-op for one rank)."""
    if ws <= 1:
        return secs
    import torch
    import torch.distributed as dist
    t = torch.tensor([secs], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_mlups(ws: int, lups_per_rank: int, secs: float) -> float:
    """Whole-job throughput: every rank advances its own replica by lups_per_rank node
    updates in the (max-over-ranks) time secs."""
    return ws * lups_per_rank / secs / 1e6


class ClockSampler:
    """nvidia-smi samples during the timed region (SM clock, throttle reasons)."""
    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.lines = []
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits", "-lms", "100",
                 "-i", str(self.idx)], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None
        time.sleep(0.3)
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                mx = float(parts[1])
            except ValueError:
                continue
            for nm, val in zip(names, parts[3:7]):
                if val.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def rejected(clk):
    bad = {"hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown"}
    if bad & set(clk.get("reasons", [])):
        return True
    if clk.get("sm_mhz") and clk.get("sm_max_mhz") and clk["sm_mhz"] < 0.6 * clk["sm_max_mhz"] \
            and "sw_power_cap" not in clk["reasons"]:
        return True
    return False


def kernel_source_hash() -> str:
    """Hash of the step kernels' device sources (all variants; the mass reductions of
    ace_reduce.cuh are not part of a step)."""
    h = hashlib.sha256()
    for name in ("ace_kernels.cuh", "ace_step_bulk.cuh", "ace_step_warp.cuh", "ace_step_pair.cuh",
                 "ace_step_dev.cuh", "ace_step_dev4.cuh", "ace_step_quad.cuh", "ace_step_tb2.cuh"):
        h.update(open(os.path.join(ROOT, "paper_2203_05230_gb300", "csrc", name), "rb").read())
    return h.hexdigest()[:16]


def stored_traffic(kernel: str, precision: str, L: int):
    """DRAM bytes per launch of the fused step from the committed ncu summary, or None
    when the kernel source has changed since the counters were taken."""
    path = os.path.join(ROOT, "profiles", f"{kernel}_{precision}_{L}.json")
    if not os.path.exists(path):
        return None
    d = json.load(open(path))
    h = kernel_source_hash()
    if d.get("kernel_source_sha256_16") != h:
        return None
    return d.get("dram_bytes_per_launch")


def measured_peak():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        d = json.load(open(path))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def cpu_baseline(args, v, seconds):
    """The FP64 oracle, as it stands, on all host cores: whole-lattice steps of the
    same workload from t = 0 for about `seconds` of CPU work; then the same loop on one
    thread for about a third of that (reported beside it, not as the baseline)."""
    import oracle as O
    th = O.threads_available()
    p = O.Params(nx=args.L, ny=args.L, tau=v.tau, eps=v.eps, U0=v.U0, T=v.T, sign=v.sign)
    s = O.Sim(p, v.phi0())

    def timed(threads, budget):
        t0 = time.perf_counter()
        s.step(1, threads=threads)
        one = time.perf_counter() - t0
        n = max(1, min(2000, int(budget / max(one, 1e-6))))
        t0 = time.perf_counter()
        s.step(n, threads=threads)
        return n, time.perf_counter() - t0

    n, dt = timed(th, seconds)
    n1, dt1 = timed(1, seconds / 3)
    return {"value": args.L * args.L * n / dt / 1e6, "unit": METRIC, "cores": th, "kind": "oracle",
            "sample": f"{n} whole-lattice FP64 oracle steps of the {args.L}x{args.L} vortex from t=1, "
                      f"{th} OpenMP threads, {dt:.1f} s",
            "single_thread": {"value": args.L * args.L * n1 / dt1 / 1e6, "unit": METRIC, "cores": 1,
                              "sample": f"{n1} further steps of the same lattice on one thread, {dt1:.1f} s"}}


def run_reference(args):
    ws, rank, _ = dist_setup()
    if rank != 0:
        return 0
    import oracle as O
    v, cfg = workload(args)
    th = O.threads_available()
    budget = 100.0  # seconds for the whole --steps K --warmup W run
    # calibrate: rate of one step on a 64-row periodic strip of the lattice
    h = 64
    mk = lambda hh: O.Sim(O.Params(nx=args.L, ny=hh, tau=v.tau, eps=v.eps, U0=v.U0, T=v.T, sign=v.sign),
                          v.phi0()[:hh])
    s = mk(h)
    t0 = time.perf_counter()
    s.step(2, threads=th)
    rate = 2 * args.L * h / (time.perf_counter() - t0)
    per = budget / (args.steps + args.warmup)
    h = int(max(3, min(args.L, per * rate / args.L)))
    s = mk(h)
    s.step(args.warmup, threads=th)
    t0 = time.perf_counter()
    s.step(args.steps, threads=th)
    dt = time.perf_counter() - t0
    val = args.L * h * args.steps / dt / 1e6
    line = {"metric": METRIC, "value": val, "unit": METRIC, "impl": "reference", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": cfg,
            "cpu_baseline": {"value": val, "unit": METRIC, "cores": th, "kind": "oracle",
                             "sample": f"each step: one FP64 oracle step of a {args.L}x{h} periodic strip "
                                       f"of the vortex lattice (bounded sample), {th} OpenMP threads"},
            "e2e": {"value": val, "unit": METRIC, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def run_ours(args):
    import torch
    ws, rank, local = dist_setup()
    if ws > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    dev = torch.cuda.current_device()
    from paper_2203_05230_gb300 import lbm_ace as A
    v, cfg = workload(args)
    prec = {"f32": A.F32, "f64": A.F64, "f16dev": A.F16DEV, "bf16dev": A.BF16DEV}[args.precision]
    stream = torch.cuda.current_stream()
    lat = A.vortex_lattice(args.L, eps=v.eps, tau=v.tau, U0=v.U0, T=v.T, precision=prec,
                           stream=stream.cuda_stream, device=dev, rows_per_cta=args.rows,
                           kernel_variant=args.variant)
    shape = lat.launch_shape()

    def warm():
        # the W untimed steps run right before the timed region (inside the clock
        # sampler, after its start-up pause): a GPU left idle for 0.3 s runs the next
        # 20 steps about 1.5 % slower
        for _ in range(args.warmup):
            lat.step(1)
        torch.cuda.synchronize()
        return lat.mass()

    def timed():
        if ws > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        lat.step(args.steps)
        e1.record(stream)
        torch.cuda.synchronize()
        if ws > 1:
            torch.distributed.barrier()
        return e0.elapsed_time(e1) / 1e3

    with ClockSampler(dev) as cs:
        m0 = warm()
        secs = timed()
    clk = cs.summary()
    note = None
    if rejected(clk):
        with ClockSampler(dev) as cs:
            m0 = warm()
            secs = timed()
        note = f"first measurement rejected for clocks {clk}; re-measured"
        clk = cs.summary()
    m1 = lat.mass()
    secs = max_over_ranks(secs, ws, "cuda")
    lups = args.L * args.L * args.steps
    value = job_mlups(ws, lups, secs)
    spl = STEPS_PER_LAUNCH.get(shape[4], 1)
    launches = args.steps // spl + args.steps % spl
    per_launch = secs / launches
    # algorithmic bytes of one launch: the state (populations and phi) read and written
    # once, whether the launch advances one step or two
    bpl = BYTES_PER_LUP[args.precision] * args.L * args.L
    peak, peak_kind = measured_peak()
    achieved = bpl / per_launch / 1e9
    traffic = stored_traffic(KERNEL_NAME[shape[4]], args.precision, args.L)
    lat.close()
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak, "traffic": traffic,
                "peak_kind": f"{peak_kind} (MEASURED_PEAKS.json hbm_gbs)" if peak_kind == "measured"
                else "fallback",
                "algorithmic_bytes_per_launch": bpl, "lattice_updates_per_launch": spl * args.L * args.L,
                "frac_of_nominal": achieved / HBM_NOMINAL_GBS, "nominal_gbs": HBM_NOMINAL_GBS,
                "dram_gbs_moved": traffic / per_launch / 1e9 if traffic else None,
                "kernel": "lbmace::" + KERNEL_NAME[shape[4]]}
    if args.precision == "f64":  # bound by the FP64 pipe: FLOP/s against the FP64 rate
        tf = F64_FLOP_PER_LUP * spl * args.L * args.L / per_launch / 1e12
        roofline = {"bound": "alu", "achieved": tf, "peak": F64_PEAK_TFLOPS, "unit": "TFLOP/s",
                    "frac": tf / F64_PEAK_TFLOPS, "traffic": traffic,
                    "peak_kind": "derived: nominal FP64 rate, 152 SMs x 2.07 GHz x 4 FLOP/clk",
                    "flop_per_lattice_update": F64_FLOP_PER_LUP,
                    "hbm_frac_algorithmic": achieved / peak,
                    "kernel": "lbmace::" + KERNEL_NAME[shape[4]]}

    e2e = None
    if not args.no_e2e:
        e2e = run_e2e(args, v, prec, stream, dev, A, ws)

    line = {"metric": METRIC, "value": value, "unit": METRIC, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": secs / args.steps * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": ARITH_DTYPE[args.precision], "storage": args.precision,
            "data": "synthetic",
            "config": {**cfg, "launch": {"tile_x": shape[0], "rows_per_cta": shape[1],
                                         "grid": [shape[2], shape[3]],
                                         "kernel": {1: "ace_step (direct loads)",
                                                    2: "ace_step_bulk (bulk-copy pipeline)",
                                                    3: "ace_step_warp (independent warps)",
                                                    4: "ace_step_pair (two columns per thread)",
                                                    5: "ace_step_dev (16-bit deviations)",
                                                    6: "ace_step_tb2 (two steps per launch)",
                                                    7: "ace_step_dev4 (16-bit deviations, four columns per thread)",
                                                    8: "ace_step_quad (four columns per thread, warp strips)"}[shape[4]],
                                         "steps_per_launch": spl},
                       "parallelism": f"replicas x{ws}" if ws > 1 else "single GPU"},
            "roofline": roofline,
            "hbm_gbs_algorithmic": achieved,
            "mass_drift_rel_timed": (m1 - m0) / m0,
            "clocks": clk, "gpu_launches": launches, "e2e": e2e}
    if note:
        line["clock_note"] = note
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(args, v, args.cpu_seconds)
    if ws == 1 and not args.no_forms and args.precision == "f32" and args.L == 2048:
        line["forms"] = forms_record(args, stream)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if ws > 1:
        torch.distributed.destroy_process_group()
    return 0


def forms_record(args, stream):
    """The three extra forms against plain FP32 on the same GPU, in this process:
    16-bit deviation storage on the 4096^2 precision workload (speed by CUDA events and
    errors over its full period T = 16384 against FP64 and FP32 runs), the 256-lattice
    batch run to each lattice's own period (aggregate MLUPS by CUDA events; speedups
    over one launch per lattice per step, graph-captured and host-issued), and the
    learned surrogate (trained here for --forms-train-steps Adam steps; one 256^2
    vortex period by the hybrid against the fastest plain FP32 form of that lattice)."""
    import torch
    from paper_2203_05230_gb300 import experiments as E
    from paper_2203_05230_gb300 import lbm_ace as A
    from paper_2203_05230_gb300 import surrogate as SG
    from paper_2203_05230_gb300 import workloads as W
    rec = {}
    t0 = time.perf_counter()
    rec["storage_16bit"] = E.storage_forms(L=4096, T=16384, stream=stream)
    rec["storage_16bit"]["record_seconds"] = time.perf_counter() - t0
    t0 = time.perf_counter()
    rec["batch"] = E.batch_uneven(256, stream=stream)
    rec["batch"]["record_seconds"] = time.perf_counter() - t0
    t0 = time.perf_counter()
    L = W.SURROGATE_TILE
    data = SG.generate(625, 32, L=L, seed=0, stream=stream)
    n_train = (625 - 25) * 32
    sur = {}
    with A.Net(0, stream) as net:
        net.set_params(W.surrogate_init_params(seed=0))
        tr = SG.Trainer(net, data, batch=16, seed=0)
        t1 = time.perf_counter()
        tr.train(args.forms_train_steps, train_pairs=np.arange(n_train))
        sur["training"] = {"pairs": data.n_pairs, "held_out_pairs": data.n_pairs - n_train,
                           "adam_steps": args.forms_train_steps, "seconds": time.perf_counter() - t1,
                           **{k: v for k, v in tr.evaluate(np.arange(n_train, data.n_pairs)).items()}}
        del data
        ro = SG.vortex_rollout(net, L=L, stream=stream)
    plain = E.plain_fp32_fastest(L=L)
    best = plain["fastest"]
    sur["plain_fp32"] = plain
    sur["hybrid"] = {k: ro[k] for k in ("hybrid_seconds", "E2_vs_lbm_T", "E2_vs_lbm_half", "E2_lbm_shape_return",
                                        "E2_hybrid_shape_return", "mass_drift_hybrid", "surrogate_windows",
                                        "fallback_windows", "max_width_dev")}
    sur["hybrid"]["mlups_equivalent"] = L * L * ro["T"] / ro["hybrid_seconds"] / 1e6
    sur["speedup_vs_fastest_plain_fp32"] = plain["seconds"][best] / ro["hybrid_seconds"]
    sur["speedup_vs_plain_fp32_launches"] = plain["seconds"]["launches"] / ro["hybrid_seconds"]
    sur["phi_l2_vs_plain_fp32_at_T"] = ro["E2_vs_lbm_T"]
    sur["record_seconds"] = time.perf_counter() - t0
    rec["surrogate"] = sur
    return rec


def run_e2e(args, v, prec, stream, dev, A, ws=1, runs=3):
    """The same metric through the public API with host buffers: phi0 uploaded from
    pinned host memory, K steps, phi and the mass read back; wall clock. A run is about
    1.5 ms of host and device work, so host noise moves one sample by several per cent: the
    value is the median of `runs` complete runs (each creates, steps, reads back and
    destroys its own lattice), all listed. With ws > 1 ranks, each run's time is the
    slowest rank's and the value is whole-job."""
    import torch
    n = args.L * args.L
    phi0 = torch.from_numpy(v.phi0()).pin_memory()
    out = torch.empty(n, dtype=torch.float64).pin_memory()
    times = []
    for _ in range(runs):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        lat = A.Lattice(nx=args.L, ny=args.L, tau=v.tau, eps=v.eps, U0=v.U0, T_period=float(v.T),
                        vortex_sign=v.sign, precision=prec, stream=stream.cuda_stream, device=dev,
                        phi0=phi0.numpy(), rows_per_cta=args.rows, kernel_variant=args.variant)
        lat.step(args.steps)
        lat.phi(out.numpy().reshape(args.L, args.L))
        m = lat.mass()
        dt = time.perf_counter() - t0
        lat.close()
        assert math.isfinite(m)
        times.append(max_over_ranks(dt, ws, "cuda"))
    dt = statistics.median(times)
    return {"value": job_mlups(ws, n * args.steps, dt), "unit": METRIC,
            "runs": [job_mlups(ws, n * args.steps, t) for t in times],
            "h2d_bytes_per_step": ws * 8 * n / args.steps, "d2h_bytes_per_step": ws * (8 * n + 8) / args.steps,
            "what": "init from pinned host phi0 + K steps + phi and mass read back, wall clock (slowest "
                    "rank), median of the listed runs; bytes per step are the job's totals / K"}


SURR_FLOP_PER_PIXEL = 2 * 9 * (3 * 32 + 3 * 32 * 32 + 32)   # multiply-adds of the five layers x 2


def measured_bf16_peak():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        d = json.load(open(path))
        return float(d["bf16_tflops"]), "measured (MEASURED_PEAKS.json bf16_tflops, burst)"
    return 1900.0, "fallback"


def run_surrogate(args):
    """Forward throughput of the learned surrogate and the hybrid vortex rollout."""
    import torch
    torch.cuda.set_device(0)
    dev = torch.cuda.current_device()
    from paper_2203_05230_gb300 import lbm_ace as A
    from paper_2203_05230_gb300 import surrogate as SG
    from paper_2203_05230_gb300 import workloads as W
    stream = torch.cuda.current_stream()
    steps = 400 if args.steps == 20000 else args.steps
    L, B = W.SURROGATE_TILE, args.surr_batch
    net = A.Net(dev, stream)
    net.set_params(W.surrogate_init_params(seed=0))
    g = torch.Generator(device="cuda").manual_seed(0)
    phi = torch.rand((B, L, L), device="cuda", generator=g)
    u = (torch.rand((B, L, L), device="cuda", generator=g) - 0.5) * 0.1
    v = (torch.rand((B, L, L), device="cuda", generator=g) - 0.5) * 0.1
    out = torch.empty_like(phi)
    for _ in range(args.warmup):
        net.forward(phi, u, v, out, B, L, L)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(dev) as cs:
        e0.record(stream)
        for _ in range(steps):
            net.forward(phi, u, v, out, B, L, L)
        e1.record(stream)
        torch.cuda.synchronize()
    clk = cs.summary()
    fwd = e0.elapsed_time(e1) / 1e3 / steps
    flops = SURR_FLOP_PER_PIXEL * B * L * L
    peak, peak_kind = measured_bf16_peak()
    achieved = flops / fwd / 1e12
    line = {"metric": "MLUPS", "value": None, "unit": "MLUPS", "n_gpus": 1, "steps": steps, "warmup": args.warmup,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "bf16 (fp32 accumulate)",
            "data": "synthetic",
            "config": {"workload": f"learned surrogate of 16 LB steps: forward on {B} x {L}^2 images; hybrid rollout "
                                   f"of one period of the {L}^2 single vortex (eps 1, tau 0.8, U0 0.04, T 4096)",
                       "network": "5 x periodic 3x3 conv, 3-32-32-32-32-1, GELU, mass-conserving residual",
                       "parallelism": "single GPU",
                       "l2": "forward activations of the timed batch exceed L2 (5 x 64 MB BF16 at batch 16)"},
            "forward": {"ms": fwd * 1e3, "images": B, "lup_equivalent_mlups": B * L * L * 16 / fwd / 1e6},
            "roofline": {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                         "frac": achieved / peak, "traffic": None, "peak_kind": peak_kind,
                         "algorithmic_flop_per_launch": flops, "kernel": "whole forward (5 launches + residual)",
                         "note": "the GELU epilogue on the FP32 units bounds the narrow layers, not the tensor pipe"},
            "clocks": clk, "gpu_launches": 6 * steps}
    if args.surr_traj > 0:
        data = SG.generate(args.surr_traj, 32, L=L, seed=0, stream=stream)
        held = max(1, args.surr_traj // 25)
        n_train = (args.surr_traj - held) * 32
        tr = SG.Trainer(net, data, batch=16, seed=0)
        t0 = time.perf_counter()
        tr.train(args.surr_train_steps, train_pairs=np.arange(n_train))
        train_s = time.perf_counter() - t0
        ev = tr.evaluate(np.arange(n_train, data.n_pairs))
        del data
        ro = SG.vortex_rollout(net, L=L, stream=stream)
        lups = L * L * ro["T"]
        line["value"] = lups / ro["hybrid_seconds"] / 1e6   # wall clock of the period on a built lattice
        steps_w = ro["windows"]
        line["e2e"] = {"value": lups / ro["hybrid_e2e_seconds"] / 1e6, "unit": "MLUPS",
                       "h2d_bytes_per_step": 8 * L * L / steps_w, "d2h_bytes_per_step": 8 * L * L / steps_w,
                       "what": "lattice built from the host phi0 (FP64), one period by the hybrid, phi read back to "
                               "the host, wall clock; a step is one window of 16 LB steps, bytes are the run's "
                               "totals per window"}
        line["vs_plain_fp32_lbm"] = {"mlups_plain": lups / ro["lbm_seconds"] / 1e6, "speedup": ro["speedup"],
                                     "phi_l2_vs_plain_at_T": ro["E2_vs_lbm_T"],
                                     "phi_l2_vs_plain_at_T_half": ro["E2_vs_lbm_half"],
                                     "surrogate_windows": ro["surrogate_windows"],
                                     "fallback_windows": ro["fallback_windows"],
                                     "mass_drift": ro["mass_drift_hybrid"]}
        line["training"] = {"pairs": args.surr_traj * 32, "adam_steps": args.surr_train_steps, "seconds": train_s,
                            "held_out_phi_l2": ev["E2_net"], "persistence_phi_l2": ev["E2_persistence"]}
    net.close()
    if not args.no_cpu_baseline:
        from oracle import surrogate as S
        rng = np.random.default_rng(0)
        p0 = rng.uniform(0, 1, (1, L, L))
        t0 = time.perf_counter()
        S.forward(W.surrogate_init_params(seed=0), p0, p0 * 0.05, p0 * 0.05)
        dt = time.perf_counter() - t0
        line["cpu_baseline"] = {"value": L * L * 16 / dt / 1e6, "unit": "MLUPS", "cores": os.cpu_count(),
                                "kind": "oracle", "sample": f"one FP64 oracle forward of one {L}^2 image "
                                                            "(numpy, LB-step equivalents of 16 per pixel)"}
    print(json.dumps(line), flush=True)
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    if args.surrogate:
        return run_surrogate(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
