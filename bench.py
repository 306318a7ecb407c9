#!/usr/bin/env python
"""Walker-steps/s of the ph-AFQMC walker step (Split-2 + Krylov + E_loc),
mixed precision against FP64.

Headline workload (precision form): synthetic Hamiltonian with N=300
orbitals, 50+50 electrons, 1500 Cholesky vectors (lambda_g = rho^g,
rho = 1e-5^(1/1500)), RHF trial, 2048 walkers per GPU, tau = 0.05, Split-2
with the Krylov action of dimension 10, local energy and mixed estimator every
step, modified Gram-Schmidt every 5 steps, complex64 walkers (mixed path).
One step = one pass of the whole walker step over all walkers.  Beside it: the
FP64 path on the same workload, the large-step workload (N=128, 20+20, 640
vectors, 1024 walkers) and the other legs listed in run_ours.  Multi-GPU
(torchrun): every rank propagates its own walkers (weak scaling, no collective
on the data path).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--precision mixed|fp64]
  python bench.py --impl reference ...   # the CPU oracle, timed on host cores
"""
from __future__ import annotations

import argparse
import json
import math
import os
import platform
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "walker-steps/s (Split-2+Krylov+E_loc), mixed vs FP64 at ≤1e-4 Ha/walker"
HEADLINE = "precision"   # inputs.CONFIGS key of the headline workload
WORKLOAD = ("precision form: N=300, Na=Nb=50, N_gamma=1500 (decay rho=1e-5^(1/1500)), 2048 walkers/GPU, "
            "tau=0.05, Split-2 + Krylov dim 10, E_loc every step, MGS every 5 steps, complex64 walkers")
NW, TAU, KDIM, REORTHO = 2048, 0.05, 10, 5
LARGE_NW = 1024          # walkers of the large-step workload (N=128) legs
# peaks for the roofline denominators
NOMINAL_FP64_TFLOPS = 1.25          # GB300 FP64 (recipe table)
SM_COUNT, SM_MAX_MHZ = 152, 2070.0  # recipe table
FP32_LANES_PER_SM = 128


def measured_peaks() -> dict:
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--no-fp64-compare", action="store_true",
                    help="skip the FP64-path rate measured beside the mixed one")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-batched", action="store_true",
                    help="skip the batched workload (16 uneven systems in one graph)")
    ap.add_argument("--no-large", action="store_true",
                    help="skip the large-step workload (N=128, 1024 walkers) rates")
    ap.add_argument("--no-precision-errors", action="store_true",
                    help="skip the per-result error of the mixed path against the FP64 path")
    ap.add_argument("--no-adjoint", action="store_true",
                    help="skip the timed gradient of the differentiation workload")
    ap.add_argument("--no-block-krylov", action="store_true",
                    help="skip the large workload with the block-Krylov exponential")
    ap.add_argument("--no-propagators", action="store_true",
                    help="skip the large workload with Split-1, the Taylor and Crank-Nicolson propagators "
                         "and the Chebyshev action")
    ap.add_argument("--no-expm-accuracy", action="store_true",
                    help="skip the k_min study of the exponential actions (Fig. 1 analogue)")
    ap.add_argument("--no-tau-scan", action="store_true",
                    help="skip the energy runs and time-step extrapolation of the small workload")
    ap.add_argument("--cpu-sample-walkers", type=int, default=1)
    ap.add_argument("--walkers", type=int, default=NW,
                    help="walkers per GPU (the workload has 2048; fewer only for small profiling cases)")
    ap.add_argument("--only-headline", action="store_true",
                    help="time the headline workload and nothing else (profiling runs)")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


# ------------------------------------------------------------------ ranks
def slowest_rank(seconds: float, world: int, device) -> float:
    """The largest of one per-rank duration over all ranks (the job lasts as long
    as its slowest rank); the duration itself when the job has one rank."""
    if world == 1:
        return seconds
    import torch
    import torch.distributed as dist
    t = torch.tensor([seconds], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t[0])


def job_rate(units_per_rank: float, world: int, seconds: float) -> float:
    """Whole-job throughput: the units every rank processed over the slowest
    rank's time (walkers are sharded, so each rank holds the same number)."""
    return world * units_per_rank / seconds


def shard_seed(base: int, rank: int) -> int:
    """Seed of a rank's synthetic fields: each rank draws its own walkers' fields."""
    return base + rank


# ------------------------------------------------------------------ clocks
class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(gpu_index), f"--query-gpu={self.Q}",
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.p = None

    def stop(self):
        if self.p is None:
            return None
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.p.kill()
        self.f.flush()
        self.f.seek(0)
        rows = [r.strip().split(",") for r in self.f.read().splitlines() if r.strip()]
        os.unlink(self.f.name)
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            try:
                sm.append(float(r[1]))
                smax = float(r[2])
                for nm, v in zip(names, r[5:9]):
                    if v.strip().lower() == "active":
                        reasons.add(nm)
            except (ValueError, IndexError):
                continue
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": smax, "reasons": sorted(reasons),
                "samples": len(sm)}


# ------------------------------------------------------------------ CPU oracle
def cpu_model() -> str:
    """The host CPU's model name (lscpu on Linux, else the platform string)."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.strip().lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    return platform.processor() or platform.machine()


def oracle_rate(system, n_walkers: int, n_steps: int, tau: float = TAU):
    """Time the CPU oracle as it stands on a bounded sample of the workload:
    n_walkers walkers for n_steps steps (Split-2 + Krylov 10, E_L every step),
    walker by walker.  Returns the cpu_baseline object and the per-step times."""
    import torch

    from oracle import afqmc_ref as R
    from paper_2403_02542_gb300.inputs import make_fields

    ham = R.make_hamiltonian(system.h1, system.L, system.trial, system.na, system.nb)
    Lbar = R.mean_field_shift(ham)
    hpp, ec = R.propagation_h1(ham, Lbar)
    B = R.half_step_propagator(hpp, tau)
    psi, lo, W = R.init_walkers(ham, n_walkers)
    e0 = float(R.local_energy(ham, psi[:1]).real[0])
    t0 = time.perf_counter()
    per_step = []
    for k in range(n_steps):
        ts = time.perf_counter()
        x = make_fields(99, k, n_walkers, ham.G)
        psi, lo, W, _ = R.step(ham, psi, lo, W, x, tau, e0, method="krylov", k=KDIM,
                               reortho=(k + 1) % REORTHO == 0, B=B, L_bar=Lbar, ec=ec)
        El = R.local_energy(ham, psi)
        R.mixed_energy(W, R.energy_window(El, e0, tau, ham.na + ham.nb))
        per_step.append(time.perf_counter() - ts)
    dt = time.perf_counter() - t0
    return dict(value=n_walkers * n_steps / dt, unit="walker-steps/s", cores=torch.get_num_threads(),
                host_cores=os.cpu_count(), cpu_model=cpu_model(), kind="oracle",
                sample=f"{n_walkers} walker(s) x {n_steps} steps of the same workload (FP64 oracle, "
                       f"walker-by-walker Krylov, E_L every step), {dt:.1f} s"), per_step


def batched_cpu_rate(system, n_walkers: int, n_steps: int, tau: float = TAU):
    """Time the batched FP64 CPU variant of the step (oracle/batched_cpu.py:
    the same arithmetic as the oracle, batched over walkers and orbital
    columns, half-rotated Cholesky contractions) on a bounded sample of the
    workload: n_walkers walkers for n_steps steps with E_L every step."""
    import torch

    from oracle import afqmc_ref as R
    from oracle.batched_cpu import BatchedStep
    from paper_2403_02542_gb300.inputs import make_fields

    ham = R.make_hamiltonian(system.h1, system.L, system.trial, system.na, system.nb)
    bs = BatchedStep(ham, tau)
    psi, _, W = R.init_walkers(ham, n_walkers)
    lo = bs.log_overlap(psi)
    e0 = float(bs.local_energy(psi[:1]).real[0])
    t0 = time.perf_counter()
    for k in range(n_steps):
        x = make_fields(99, k, n_walkers, ham.G)
        psi, lo, W = bs.step(psi, lo, W, x, e0, k=KDIM, reortho=(k + 1) % REORTHO == 0)
        El = bs.local_energy(psi)
        R.mixed_energy(W, R.energy_window(El, e0, tau, ham.na + ham.nb))
    dt = time.perf_counter() - t0
    return dict(value=n_walkers * n_steps / dt, unit="walker-steps/s", cores=torch.get_num_threads(),
                host_cores=os.cpu_count(), cpu_model=cpu_model(), kind="batched (FP64, batched over walkers)",
                sample=f"{n_walkers} walkers x {n_steps} steps of the same workload (FP64, batched over walkers "
                       f"and orbital columns, half-rotated Cholesky contractions, E_L every step), {dt:.1f} s")


def config_dict(precision: str, world: int, nw: int):
    wl = WORKLOAD if nw == NW else WORKLOAD.replace(f"{NW} walkers/GPU", f"{nw} walkers/GPU (reduced)")
    return {"workload": wl, "walkers_per_gpu": nw, "N": 300, "na": 50, "nb": 50, "G": 1500,
            "tau": TAU, "expm": "krylov", "krylov_dim": KDIM, "reortho_every": REORTHO,
            "precision": precision, "parallelism": f"walkers sharded over {world} GPU(s)",
            "force_bias": "<L_g> of each step from the Coulomb traces of the previous step's E_L (same walkers)",
            "l2": "working set larger than L2 (walkers 0.49 GB, Krylov basis, A_w planes > 129 MB)"}


# ------------------------------------------------------------------ reference arm
def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    import torch

    from paper_2403_02542_gb300.inputs import config_system
    system = config_system(HEADLINE)
    nwalk = 1
    total_steps = args.warmup + args.steps
    cpu, per_step = oracle_rate(system, nwalk, total_steps)
    timed = per_step[args.warmup:]
    t = sum(timed)
    value = nwalk * len(timed) / t
    line = {
        "metric": METRIC, "value": value, "unit": "walker-steps/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000.0 * t / len(timed),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic (seeded Hamiltonian, Gaussian fields)", "impl": "reference",
        "config": config_dict("fp64 oracle", 1, NW),
        "cpu_baseline": {"value": value, "unit": "walker-steps/s", "cores": torch.get_num_threads(),
                         "host_cores": os.cpu_count(), "cpu_model": cpu["cpu_model"], "kind": "oracle",
                         "sample": f"{nwalk} walker per step of the same workload, {args.steps} "
                                   f"timed steps after {args.warmup} warm-up steps"},
        "e2e": {"value": value, "unit": "walker-steps/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))
    return 0


# ------------------------------------------------------------------ our arm
def adjoint_rate(dev):
    """Gradient of the mixed estimator through a 100-step fixed-field walk
    (differentiation workload: N=96, 15+15 electrons, 480 vectors, 512
    walkers, Taylor-6, QR every 10 steps, checkpoints every 10) in FP64 and in
    the mixed precision (complex64 walkers), timed with CUDA events; the plain
    forward walk of the same workload beside each, and the mixed J and
    gradients against the FP64 ones."""
    import torch
    from paper_2403_02542_gb300.api import Context
    from paper_2403_02542_gb300.inputs import CONFIGS, config_system
    cfg = CONFIGS["grad"]
    s = config_system("grad")
    nw, steps, tau, order, r = cfg["walkers"], cfg["steps"], cfg["tau"], cfg["order"], cfg["reortho"]
    gen = torch.Generator(device=dev)
    gen.manual_seed(99)
    fields = torch.randn(steps, nw, s.G, dtype=torch.float64, device=dev, generator=gen)
    stream = torch.cuda.current_stream(dev)
    e0 = None

    def one(precision):
        nonlocal e0
        ctx = Context(s.h1, s.L, s.trial, s.na, s.nb, s.e_const, precision=precision, device=dev)
        w = ctx.new_walkers(nw)
        ctx.init_walkers(w)
        el = torch.empty(nw, 2, dtype=torch.float64, device=dev)
        em = torch.empty(4, dtype=torch.float64, device=dev)
        if e0 is None:
            ctx.local_energy(w, 0.0, tau, el, em)
            e0 = float(el[0, 0])
        ctx.walk_backward(w, fields[:2], tau, e0, order=order, reortho_every=r, ckpt_every=10)   # warm-up
        torch.cuda.synchronize()
        l0 = ctx.launch_count
        a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a0.record(stream)
        J, gh, gL = ctx.walk_backward(w, fields, tau, e0, order=order, reortho_every=r, ckpt_every=10)
        a1.record(stream)
        torch.cuda.synchronize()
        t_adj = a0.elapsed_time(a1)
        launches = ctx.launch_count - l0
        f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        f0.record(stream)
        for k in range(steps):
            ctx.step(w, fields[k], tau, e0, expm="taylor", order=order, reortho=(k + 1) % r == 0,
                     measure=(k == steps - 1), e_loc=el, e_mix=em)
        f1.record(stream)
        torch.cuda.synchronize()
        t_fwd = f0.elapsed_time(f1)
        ctx.close()
        res = {"value": nw * steps / (t_adj / 1000.0), "unit": "walker-steps/s (gradient, forward + adjoint)",
               "ms": t_adj, "forward_ms": t_fwd, "adjoint_over_forward": t_adj / t_fwd,
               "J": float(J[2]), "live": float(J[3]), "gpu_launches": launches}
        return res, gh, gL

    r64, gh64, gL64 = one("fp64")
    r32, gh32, gL32 = one("mixed")
    return {
        "workload": "gradient of E_n after a 100-step fixed-field walk: N=96, Na=Nb=15, N_gamma=480, "
                    "512 walkers, tau=0.05, Split-2 + Taylor-6, QR every 10 steps, checkpoints every 10",
        "fp64": r64, "mixed": r32, "mixed_speedup": r64["ms"] / r32["ms"],
        "mixed_vs_fp64": {
            "dJ": abs(r32["J"] - r64["J"]),
            "grad_h1_rel": float((gh32 - gh64).abs().max() / gh64.abs().max()),
            "grad_L_rel": float((gL32 - gL64).abs().max() / gL64.abs().max()),
        },
    }


def bond_scan(dev, n_points=11, s_max=0.05):
    """The 11-point path scan of the differentiation workload (N=96, 15+15
    electrons, 480 vectors, 512 walkers, 100 fixed-field steps at tau=0.05,
    Split-2 + Taylor-6, QR every 10, checkpoints every 10, mixed precision):
    h1(s) = h1 + s dH1, L(s) = L + s dL with dH1, dL random symmetric scaled
    to 0.01 (of max|L| for dL), s in [-0.05, 0.05]; at every point J(s), the
    adjoint dJ/ds and a central difference of J (step 0.01), all with the same
    fields, trial and E_0."""
    import numpy as np
    import torch
    from paper_2403_02542_gb300.inputs import CONFIGS, config_system
    from paper_2403_02542_gb300.scan import path_scan
    cfg = CONFIGS["grad"]
    s = config_system("grad")
    rng = np.random.default_rng(2403)
    dH = rng.standard_normal(s.h1.shape)
    dH = 0.5 * (dH + dH.T)
    dH *= 0.01 / np.abs(dH).max()
    dL = rng.standard_normal(s.L.shape)
    dL = 0.5 * (dL + dL.transpose(0, 2, 1))
    dL *= 0.01 * np.abs(s.L).max() / np.abs(dL).max()
    gen = torch.Generator(device=dev)
    gen.manual_seed(2403)
    fields = torch.randn(cfg["steps"], cfg["walkers"], s.G, dtype=torch.float64, device=dev, generator=gen)
    from paper_2403_02542_gb300.api import Context
    c = Context(s.h1, s.L, s.trial, s.na, s.nb, s.e_const, precision="mixed", device=dev)
    w = c.new_walkers(1)
    c.init_walkers(w)
    el = torch.empty(1, 2, dtype=torch.float64, device=dev)
    em = torch.empty(4, dtype=torch.float64, device=dev)
    c.local_energy(w, 0.0, cfg["tau"], el, em)
    e0 = float(el[0, 0])
    c.close()
    t0 = time.perf_counter()
    pts = path_scan(s, fields, np.linspace(-s_max, s_max, n_points), dH, dL, cfg["tau"], e0, order=cfg["order"],
                    reortho_every=cfg["reortho"], ckpt_every=10, precision="mixed", fd_step=1e-2, device=dev)
    wall = time.perf_counter() - t0
    scale = max(abs(p["dJds"]) for p in pts)
    return {"workload": "differentiation workload (N=96, Na=Nb=15, N_gamma=480, 512 walkers, 100 fixed-field steps, "
                        "tau=0.05, Split-2 + Taylor-6, QR every 10, checkpoints every 10), mixed; "
                        "h1(s) = h1 + s dH1, L(s) = L + s dL, dH1 and dL random symmetric of max 0.01 (dL: 0.01 max|L|)",
            "points": pts, "max_abs_dJds_minus_fd": max(abs(p["dJds"] - p["dJds_fd"]) for p in pts),
            "max_abs_dJds": scale, "wall_s": wall}


def block_krylov_rate(dev, steps=5):
    """The large-step workload (N=128, 20+20 electrons, 640 vectors, 1024
    walkers, tau=0.05, E_L every step, MGS every 5 steps) with the block-Krylov
    exponential of k = 4 blocks (Eq. bkrylov, the order the paper recommends)
    instead of the column Krylov of dimension 10: mixed precision, CUDA-event
    timed after two warm-up steps, per-class kernel times."""
    import torch
    from paper_2403_02542_gb300.api import Context
    from paper_2403_02542_gb300.inputs import config_system
    s = config_system("large")
    k = 4
    ctx = Context(s.h1, s.L, s.trial, s.na, s.nb, s.e_const, precision="mixed", device=dev)
    w = ctx.new_walkers(LARGE_NW)
    ctx.init_walkers(w)
    el = torch.empty(LARGE_NW, 2, dtype=torch.float64, device=dev)
    em = torch.empty(4, dtype=torch.float64, device=dev)
    ctx.local_energy(w, 0.0, TAU, el, em)
    e0 = float(el[0, 0])
    gen = torch.Generator(device=dev)
    gen.manual_seed(11)
    x = torch.randn(steps + 2, LARGE_NW, s.G, dtype=torch.float64, device=dev, generator=gen)
    stream = torch.cuda.current_stream(dev)
    for i in range(2):
        ctx.step(w, x[i], TAU, e0, expm="bkrylov", order=k, measure=True, e_loc=el, e_mix=em, reuse_bias=True)
    torch.cuda.synchronize()
    ctx.profile(True)
    a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a0.record(stream)
    for i in range(steps):
        ctx.step(w, x[2 + i], TAU, e0, expm="bkrylov", order=k, reortho=(i + 1) % REORTHO == 0, measure=True,
                 e_loc=el, e_mix=em, reuse_bias=True)
    a1.record(stream)
    torch.cuda.synchronize()
    ctx.profile(False)
    prof = ctx.profile_read()
    ms = a0.elapsed_time(a1) / steps
    out = {"workload": "large-step workload (N=128, Na=Nb=20, N_gamma=640, 1024 walkers, tau=0.05, E_loc every "
                       "step, MGS every 5 steps) with block Krylov of 4 blocks, mixed",
           "value": LARGE_NW / (ms / 1000.0), "unit": "walker-steps/s", "ms_per_step": ms, "e_mix": float(em[2]),
           "kernel_ms_per_step": {c: v[0] / steps for c, v in prof.items()}}
    ctx.close()
    return out


def propagator_rates(dev, steps=3):
    """The large-step workload (N=128, 20+20 electrons, 640 vectors, 1024
    walkers, tau=0.05, E_L every step, MGS every 5 steps, mixed) with the other
    walker updates of Sec. III and the Chebyshev action of Sec. IV.B in place of
    Split-2 + Krylov 10: CUDA-event timed after two warm-up steps.  A variant
    that fails reports its error instead of a rate."""
    import torch
    from paper_2403_02542_gb300.api import Context
    from paper_2403_02542_gb300.inputs import config_system
    s = config_system("large")
    variants = [("split1", "krylov", 10), ("taylor", "taylor", 8), ("cn", "taylor", 0),
                ("split2", "chebyshev", 8), ("split2", "taylor", 8), ("split2", "lanczos", 10)]
    out = {"workload": "large-step workload (N=128, Na=Nb=20, N_gamma=640, 1024 walkers, tau=0.05, E_loc every "
                       "step, MGS every 5 steps), mixed", "unit": "walker-steps/s", "rates": {}}
    gen = torch.Generator(device=dev)
    gen.manual_seed(13)
    x = torch.randn(steps + 2, LARGE_NW, s.G, dtype=torch.float64, device=dev, generator=gen)
    stream = torch.cuda.current_stream(dev)
    for prop, expm, k in variants:
        name = f"{prop}+{expm}{k}" if prop != "cn" else "cn"
        ctx = None
        try:
            ctx = Context(s.h1, s.L, s.trial, s.na, s.nb, s.e_const, precision="mixed", device=dev)
            w = ctx.new_walkers(LARGE_NW)
            ctx.init_walkers(w)
            el = torch.empty(LARGE_NW, 2, dtype=torch.float64, device=dev)
            em = torch.empty(4, dtype=torch.float64, device=dev)
            ctx.local_energy(w, 0.0, TAU, el, em)
            e0 = float(el[0, 0])
            for i in range(2):
                ctx.step(w, x[i], TAU, e0, expm=expm, order=k, measure=True, e_loc=el, e_mix=em, reuse_bias=True,
                         propagator=prop)
            torch.cuda.synchronize()
            a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a0.record(stream)
            for i in range(steps):
                ctx.step(w, x[2 + i], TAU, e0, expm=expm, order=k, reortho=(i + 1) % REORTHO == 0, measure=True,
                         e_loc=el, e_mix=em, reuse_bias=True, propagator=prop)
            a1.record(stream)
            torch.cuda.synchronize()
            ms = a0.elapsed_time(a1) / steps
            out["rates"][name] = {"value": LARGE_NW / (ms / 1000.0), "ms_per_step": ms, "e_mix": float(em[2])}
        except Exception as exc:  # noqa: BLE001 - one failing variant must not end the bench line
            out["rates"][name] = {"error": f"{type(exc).__name__}: {exc}"}
        finally:
            if ctx is not None:
                ctx.close()
    return out


def lanczos_rate(dev, K=5, warmup=3):
    """The headline workload (N=300, 50+50 electrons, 1500 vectors, 2048
    walkers, tau=0.05, E_L every step, MGS every 5 steps, mixed) with the
    complex-symmetric Lanczos action of dimension 10 in place of Arnoldi:
    CUDA-event timed, per-class split from a separate pass, and E_L of the
    two actions on the same walkers after one step."""
    import torch
    system, ctx, w, el, em, e0, _ = make_context(dev, HEADLINE, "mixed", NW, tune=True)
    gen = torch.Generator(device=dev)
    gen.manual_seed(2718)
    fields = torch.randn(warmup + K, NW, system.G, dtype=torch.float64, device=dev, generator=gen)
    stream = torch.cuda.current_stream(dev)

    n_steps = 0

    def lstep(x):
        nonlocal n_steps
        n_steps += 1
        ctx.step(w, x, TAU, e0, expm="lanczos", order=KDIM, reortho=(n_steps % REORTHO == 0), measure=True,
                 e_loc=el, e_mix=em, reuse_bias=True)

    for i in range(warmup):
        lstep(fields[i])
    ms = timed_steps(lstep, fields, warmup, K, stream) / K
    split = class_split(ctx, lstep, fields, 0, 3, stream)
    # one step from the same walkers with each action
    psi0, W0, lo0, st0 = w.psi.clone(), w.weight.clone(), w.logovl.clone(), w.status.clone()
    out_e = {}
    for expm in ("krylov", "lanczos"):
        w.psi.copy_(psi0); w.weight.copy_(W0); w.logovl.copy_(lo0); w.status.copy_(st0)
        ctx.step(w, fields[0], TAU, e0, expm=expm, order=KDIM, measure=True, e_loc=el, e_mix=em)
        out_e[expm] = el[:, 0].clone()
    live = W0 > 0
    dE = float((out_e["krylov"] - out_e["lanczos"]).abs()[live].max())
    ctx.close()
    del fields, w
    torch.cuda.empty_cache()
    return {"workload": "precision workload (N=300, Na=Nb=50, N_gamma=1500, 2048 walkers, tau=0.05, E_loc every "
                        "step, MGS every 5 steps), mixed, complex-symmetric Lanczos of dimension 10",
            "value": NW / (ms / 1000.0), "unit": "walker-steps/s", "ms_per_step": ms, "steps": K,
            "kernel_ms_per_step": split,
            "E_L_vs_arnoldi_max_abs_Ha": dE}


def expm_accuracy(dev, nw=2400, n_steps=10, taus=(0.02, 0.1, 0.3), budget_s=60.0):
    """The accuracy study of Sec. IV.E (Fig. 1) through the library: on one
    synthetic system (N=64, Na=Nb=10, N_gamma=320, FP64), 2400 walkers, 10 steps
    per run, the smallest order of the Taylor, Chebyshev, Krylov,
    block-Krylov and Lanczos actions (orders up to 24; None beyond) whose run energy is
    within 1e-5 Ha of the order-64 Taylor run, at each time step.  Stops after
    budget_s seconds (the time steps not reached are left out)."""
    import time
    import torch
    from paper_2403_02542_gb300 import expm_study as S
    from paper_2403_02542_gb300.api import Context
    from paper_2403_02542_gb300.inputs import make_system
    out = {"workload": "N=64, Na=Nb=10, N_gamma=320 (rho = 1e-5^(1/320)), 2400 walkers, 10 steps per run, FP64, "
                       "eps = 1e-5 Ha against the order-64 Taylor run", "k_min": {}}
    ctx = None
    try:
        s = make_system(64, 10, 10, 320, rho=1e-5 ** (1 / 320), seed=64)
        ctx = Context(s.h1, s.L, s.trial, s.na, s.nb, s.e_const, precision="fp64", device=dev)
        w = ctx.new_walkers(1)
        ctx.init_walkers(w)
        el = torch.empty(1, 2, dtype=torch.float64, device=dev)
        em = torch.empty(4, dtype=torch.float64, device=dev)
        ctx.local_energy(w, 0.0, 0.1, el, em)
        e0 = float(el[0, 0])
        t0 = time.time()
        for tau in taus:
            if time.time() - t0 > budget_s:
                break
            gen = torch.Generator(device=dev)
            gen.manual_seed(17)
            x = torch.randn(n_steps, nw, s.G, dtype=torch.float64, device=dev, generator=gen)
            res = S.sweep(ctx, nw, n_steps, lambda _t: (lambda k: x[k]), (tau,), e0, k_max=24)[tau]
            out["k_min"][str(tau)] = res
        out["seconds"] = time.time() - t0
    except Exception as exc:  # noqa: BLE001 - the study must not end the bench line
        out["error"] = f"{type(exc).__name__}: {exc}"
    finally:
        if ctx is not None:
            ctx.close()
    return out


def tau_scan(dev, imag_time=10.0, taus=(0.01, 0.02, 0.05, 0.1), nw=1024):
    """Energy runs and the time-step extrapolation (Sec. V.G) on the small
    workload (N=8, 2+2 electrons, 32 vectors lambda_g = 0.5^g, Taylor-6, QR
    every 5 steps, FP64): for each tau, imag_time / tau steps of 1024 walkers
    with E_L every step, comb population control every 10 steps and E_0
    updates, the first 30 % as equilibration; the blocking analysis of each
    run and the fits E(tau) = E_0 + beta tau^2 and E_0 + alpha tau + beta tau^2
    (Eq. square_fit) for Split-2.  A Split-1 series, whose time-step error is
    linear, runs at tau < 0.05 (the range the paper fits linearly) and is fitted
    by E_0 + alpha tau: the fits estimate the same E_0.  The same time steps
    then run on the large workload (N=128, 20+20, 640 vectors) in mixed
    precision with Split-2 + Krylov 10."""
    import torch
    from paper_2403_02542_gb300 import energy as S
    from paper_2403_02542_gb300.api import Context
    from paper_2403_02542_gb300.inputs import config_system
    s = config_system("small")

    def series(propagator, seed_base, taus, sys_=s, precision="fp64", expm="taylor", order=6):
        s = sys_
        runs = []
        total_steps = 0
        for i, tau in enumerate(taus):
            n_steps = int(round(imag_time / tau))
            n_eq = int(0.3 * n_steps)
            ctx = Context(s.h1, s.L, s.trial, s.na, s.nb, s.e_const, precision=precision, device=dev)
            w = ctx.new_walkers(nw)
            ctx.init_walkers(w)
            gen = torch.Generator(device=dev)
            gen.manual_seed(seed_base + i)
            x = torch.empty(nw, s.G, dtype=torch.float64, device=dev)

            def fields(k):
                return x.normal_(generator=gen)

            # E_0 starts at the uncapped mean E_L of the starting walkers (initial_e0)
            out = S.energy_run(ctx, w, tau, None, n_steps, fields=fields, n_eq=n_eq, expm=expm,
                               order=order, reortho_every=5, pop_every=10, seed=seed_base + 100 + i,
                               update_e0=True, propagator=propagator)
            st = out["stats"]
            runs.append({"tau": tau, "steps": n_steps, "E": st["E_bar"], "sigma": st["sigma"],
                         "kappa": st["kappa"]})
            total_steps += n_steps
            ctx.close()
        return runs, total_steps

    def fit(runs, power):
        e0, c, s0, sc, chi2 = S.extrapolate([r["tau"] for r in runs], [r["E"] for r in runs],
                                            [r["sigma"] for r in runs], power)
        return {"E0": e0, ("beta" if power == 2 else "alpha"): c, "sigma_E0": s0,
                ("sigma_beta" if power == 2 else "sigma_alpha"): sc, "chi2_dof": chi2,
                "sigma_x": S.extrapolation_error([r["sigma"] for r in runs])}

    t0 = time.perf_counter()
    runs, total_steps = series("split2", 100, taus)
    wall = time.perf_counter() - t0
    general = S.fit_time_step([r["tau"] for r in runs], [r["E"] for r in runs], [r["sigma"] for r in runs], (1, 2))
    out = {"workload": "small workload (N=8, Na=Nb=2, N_gamma=32, lambda_g=0.5^g), FP64, 1024 walkers, "
                       "Split-2 + Taylor-6, QR every 5, comb every 10 steps, E_0 updated, imaginary time 10 per tau",
           "runs": runs, "fit": fit(runs, 2),
           "fit_general": {"E0": general["E0"], "alpha": general["c"][0], "beta": general["c"][1],
                           "sigma_E0": general["sigma_E0"], "chi2_dof": general["chi2_dof"]},
           "wall_s": wall, "walker_steps_per_s": nw * total_steps / wall}
    try:
        runs1, _ = series("split1", 300, (0.005, 0.01, 0.02, 0.04))
        f1 = fit(runs1, 1)
        out["split1"] = {"runs": runs1, "fit": f1,
                         "E0_difference_sigmas": (f1["E0"] - out["fit"]["E0"])
                         / max(1e-300, (f1["sigma_E0"] ** 2 + out["fit"]["sigma_E0"] ** 2) ** 0.5)}
    except Exception as exc:  # noqa: BLE001 - the Split-2 series stands on its own
        out["split1"] = {"error": f"{type(exc).__name__}: {exc}"}
    # the large workload over the same time steps, mixed precision, Split-2 + Krylov 10
    try:
        t1 = time.perf_counter()
        runs_l, steps_l = series("split2", 500, taus, config_system("large"), "mixed", "krylov", 10)
        wall_l = time.perf_counter() - t1
        gen_l = S.fit_time_step([r["tau"] for r in runs_l], [r["E"] for r in runs_l],
                                [r["sigma"] for r in runs_l], (1, 2))
        out["large"] = {"workload": "large workload (N=128, Na=Nb=20, N_gamma=640), mixed, 1024 walkers, "
                                    "Split-2 + Krylov 10, QR every 5, comb every 10 steps, E_0 updated, "
                                    "imaginary time 10 per tau",
                        "runs": runs_l, "fit": fit(runs_l, 2),
                        "fit_general": {"E0": gen_l["E0"], "alpha": gen_l["c"][0], "beta": gen_l["c"][1],
                                        "sigma_E0": gen_l["sigma_E0"], "chi2_dof": gen_l["chi2_dof"]},
                        "wall_s": wall_l, "walker_steps_per_s": nw * steps_l / wall_l}
    except Exception as exc:  # noqa: BLE001 - the small-workload series stand on their own
        out["large"] = {"error": f"{type(exc).__name__}: {exc}"}
    return out


def batched_rate(dev, steps=3, warmup=2):
    """Batched workload: 16 systems with N uniform in 64..400, N/6 electrons
    per spin, 5N vectors, 256-2048 walkers each; all systems advanced by one
    captured CUDA graph per step (afqmc_batch_step), tile shapes autotuned,
    mixed precision, Krylov 10, tau=0.05, E_L every step, force bias reused.
    value = sum of walker-steps over all systems per second."""
    import torch
    from paper_2403_02542_gb300.api import Batch, Context
    from paper_2403_02542_gb300.inputs import batched_systems
    t0 = time.perf_counter()
    systems = batched_systems()
    t_gen = time.perf_counter() - t0
    t0 = time.perf_counter()
    ctxs, ws, els, ems, e0s, xs = [], [], [], [], [], []
    for s, nw in systems:
        c = Context(s.h1, s.L, s.trial, s.na, s.nb, s.e_const, precision="mixed", device=dev)
        w = c.new_walkers(nw)
        c.init_walkers(w)
        el = torch.empty(nw, 2, dtype=torch.float64, device=dev)
        em = torch.empty(4, dtype=torch.float64, device=dev)
        c.local_energy(w, 0.0, TAU, el, em)
        e0s.append(float(el[0, 0]))
        c.autotune(nw)
        gen = torch.Generator(device=dev)
        gen.manual_seed(11 + len(ctxs))
        xs.append(torch.randn(warmup + steps, nw, s.G, dtype=torch.float64, device=dev, generator=gen))
        ctxs.append(c)
        ws.append(w)
        els.append(el)
        ems.append(em)
    torch.cuda.synchronize()
    t_setup = time.perf_counter() - t0
    batch = Batch(ctxs)
    stream = torch.cuda.current_stream(dev)

    def one(k):
        batch.step(ws, [x[k] for x in xs], TAU, e0s, expm="krylov", order=KDIM, reortho=False, measure=True,
                   e_loc=els, e_mix=ems, reuse_bias=True)

    for k in range(warmup):
        one(k)
    torch.cuda.synchronize()
    l0 = sum(c.launch_count for c in ctxs)
    a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a0.record(stream)
    for k in range(steps):
        one(warmup + k)
    a1.record(stream)
    torch.cuda.synchronize()
    ms = a0.elapsed_time(a1) / steps
    launches = sum(c.launch_count for c in ctxs) - l0
    total_w = sum(nw for _, nw in systems)

    # the same systems and steps without the graph: every system's step by
    # plain afqmc_step calls, one system after another on one stream, each
    # timed with its own event pair
    def seq_one(k):
        evs = []
        for i, c in enumerate(ctxs):
            e_a, e_b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e_a.record(stream)
            c.step(ws[i], xs[i][k], TAU, e0s[i], expm="krylov", order=KDIM, measure=True, e_loc=els[i],
                   e_mix=ems[i], reuse_bias=True)
            e_b.record(stream)
            evs.append((e_a, e_b))
        return evs

    seq_one(0)
    torch.cuda.synchronize()
    per_sys = [0.0] * len(ctxs)
    b0, b1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    b0.record(stream)
    all_evs = [seq_one(warmup + k) for k in range(steps)]
    b1.record(stream)
    torch.cuda.synchronize()
    for evs in all_evs:
        for i, (e_a, e_b) in enumerate(evs):
            per_sys[i] += e_a.elapsed_time(e_b) / steps
    seq_ms = b0.elapsed_time(b1) / steps
    out = {
        "workload": "batched form: 16 synthetic systems, N uniform in 64..400, Na=Nb=N/6, N_gamma=5N, "
                    "256-2048 walkers each, one CUDA graph per step over all systems, autotuned tiles, "
                    "tau=0.05, Split-2 + Krylov dim 10, mixed, E_loc every step",
        "systems": [[s.N, nw] for s, nw in systems], "walkers": total_w, "steps": steps,
        "ms_per_step": ms, "value": total_w / (ms / 1000.0), "unit": "walker-steps/s (sum over systems)",
        "gpu_launches_per_step": launches / steps, "generate_s": t_gen, "setup_s": t_setup,
        "e_mix": [float(em[2]) for em in ems],
        "sequential": {"ms_per_step": seq_ms, "value": total_w / (seq_ms / 1000.0),
                       "per_system_ms": per_sys,
                       "note": "the same steps by plain afqmc_step calls, one system after another on one stream"},
        "graph_over_sequential": seq_ms / ms,
    }
    batch.close()
    for c in ctxs:
        c.close()
    del ws, xs
    torch.cuda.empty_cache()
    return out


# DRAM bytes (read + write) of one exchange_tc_kernel launch on the headline
# workload at 2048 walkers, from one single-pass ncu capture (command and
# figures in profiles/exchange_tc_kernel_precision_2048walkers_dram.txt), valid
# while the kernel's sources are the ones captured (sha256 below).
EXCHANGE_TRAFFIC = {
    "bytes": 2.38e9 + 198.56e6,
    "walkers": 2048,
    "source": "profiles/exchange_tc_kernel_precision_2048walkers_dram.txt",
    "sha256": {"paper_2403_02542_gb300/csrc/k_exchange_tc.cu":
               "a86febb3905dde7f6f0de6e3a9183fac1236d5cc746f6dcf0130592e22973d24",
               "paper_2403_02542_gb300/csrc/tc_common.cuh":
               "17add56279122795b8af511ad3d8faaf192d72127be1b26c8b888975eed98633"},
}


def exchange_traffic(precision: str, nw: int):
    """(bytes per launch, note) of the captured exchange launch, or (None,
    reason) when the workload or the kernel's sources differ from the capture."""
    import hashlib
    if precision != "mixed" or nw != EXCHANGE_TRAFFIC["walkers"]:
        return None, "no capture for this precision / walker count"
    root = os.path.dirname(os.path.abspath(__file__))
    for rel, digest in EXCHANGE_TRAFFIC["sha256"].items():
        try:
            with open(os.path.join(root, rel), "rb") as f:
                if hashlib.sha256(f.read()).hexdigest() != digest:
                    return None, f"{rel} changed since the capture"
        except OSError:
            return None, f"{rel} not found"
    return EXCHANGE_TRAFFIC["bytes"], ("ncu dram__bytes_read.sum + dram__bytes_write.sum, one launch at full size, "
                                       + EXCHANGE_TRAFFIC["source"])


def exchange_flop_per_walker(system) -> int:
    """Algorithmic flops of the Coulomb + exchange contraction per walker:
    T_gs = Lh_gs Theta_s for every g and spin, G * 4 (na^2 + nb^2) * N real
    flops (a real-times-complex multiply-add is 4 flops)."""
    return system.G * 4 * (system.na * system.na + system.nb * system.nb) * system.N


def step_flop_per_walker(system, k: int = KDIM) -> int:
    """Algorithmic flops of one Split-2 + Krylov-k step with E_L, per walker:
    exchange + Coulomb 4 G (na^2 + nb^2) N, the k products A v over the
    nc = na + nb orbitals 8 k N^2 nc, the field assembly 2 G N^2 (the
    independent half of the symmetric A), the force bias 2 G nc N, the two
    half steps 8 N^2 nc, the Arnoldi projections 8 nc N k (k + 1) and the
    overlap, ratio and one-body terms 20 N (na^2 + nb^2)."""
    N, G, na, nb = system.N, system.G, system.na, system.nb
    nc, n2 = na + nb, na * na + nb * nb
    return (4 * G * n2 * N + 8 * k * N * N * nc + 2 * G * N * N + 2 * G * nc * N + 8 * N * N * nc
            + 8 * nc * N * k * (k + 1) + 20 * N * n2)


def exchange_peak(precision: str):
    """Roofline denominator of the exchange kernel: (peak, bound, note)."""
    if precision == "fp64":
        return NOMINAL_FP64_TFLOPS, "alu", "FP64 nominal 1.25 TFLOP/s (recipe table); own FMA probe measured 1.19"
    # BF16x3 split on tcgen05: three bf16 MMAs per algorithmic product; the kernel
    # runs inside a long step, so the sustained bf16 figure is the denominator
    peaks = measured_peaks()
    bf16 = peaks.get("bf16_tflops_sustained") or 1700.0
    src = "MEASURED_PEAKS.json" if peaks else "fallback 1.7 PFLOP/s"
    return bf16 / 3.0, "tensor", (f"of measured: sustained bf16 {bf16:.1f} TFLOP/s ({src}) / 3 MMA passes "
                                  "(BF16x3 split); achieved counts algorithmic flops once")


def make_context(dev, cfg_name, precision, nw, tune=True):
    """Context, initialised walkers, E_L buffers and an uncapped E_0 for one workload."""
    import torch
    from paper_2403_02542_gb300.api import Context
    from paper_2403_02542_gb300.inputs import config_system
    system = config_system(cfg_name)
    ctx = Context(system.h1, system.L, system.trial, system.na, system.nb, system.e_const,
                  precision=precision, device=dev)
    w = ctx.new_walkers(nw)
    ctx.init_walkers(w)
    el = torch.empty(nw, 2, dtype=torch.float64, device=dev)
    em = torch.empty(4, dtype=torch.float64, device=dev)
    ctx.local_energy(w, 0.0, TAU, el, em)
    e0 = float(el[0, 0])            # uncapped E_L of the trial (all walkers start there)
    tiles = ctx.autotune(nw) if tune else None
    return system, ctx, w, el, em, e0, tiles


class Stepper:
    """Split-2 + Krylov 10 steps with E_L every step, MGS every REORTHO steps
    and the force bias from the previous E_L, counting steps for the MGS
    schedule."""

    def __init__(self, ctx, w, el, em, e0):
        self.ctx, self.w, self.el, self.em, self.e0 = ctx, w, el, em, e0
        self.k = 0

    def __call__(self, x):
        self.k += 1
        self.ctx.step(self.w, x, TAU, self.e0, expm="krylov", order=KDIM, reortho=(self.k % REORTHO == 0),
                      measure=True, e_loc=self.el, e_mix=self.em, reuse_bias=True)


def timed_steps(step, fields, first, K, stream):
    """K steps on device-resident fields, CUDA events on the launching stream."""
    import torch
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    ev0.record(stream)
    for i in range(K):
        step(fields[(first + i) % fields.shape[0]])
    ev1.record(stream)
    torch.cuda.synchronize()
    return ev0.elapsed_time(ev1)


def class_split(ctx, step, fields, first, n, stream):
    """Per-kernel-class device time per step from a separate, untimed pass of
    n steps with an event pair around every launch."""
    ctx.profile(True)
    timed_steps(step, fields, first, n, stream)
    ctx.profile(False)
    return {c: v[0] / n for c, v in ctx.profile_read().items()}


def large_rates(dev, K=10, warmup=3):
    """The large-step workload (N=128, 20+20 electrons, 640 vectors, 1024
    walkers, tau=0.05, Split-2 + Krylov 10, E_L every step, MGS every 5 steps):
    the mixed path (exchange roofline and per-class split) and the FP64 path,
    CUDA-event timed."""
    import torch
    out = {"workload": "large-step workload: N=128, Na=Nb=20, N_gamma=640 (rho = 1e-5^(1/640)), 1024 walkers, "
                       "tau=0.05, Split-2 + Krylov 10, E_loc every step, MGS every 5 steps"}
    stream = torch.cuda.current_stream(dev)
    for prec, k in (("mixed", K), ("fp64", 3)):
        system, ctx, w, el, em, e0, _ = make_context(dev, "large", prec, LARGE_NW)
        gen = torch.Generator(device=dev)
        gen.manual_seed(1234)
        fields = torch.randn(warmup + k, LARGE_NW, system.G, dtype=torch.float64, device=dev, generator=gen)
        step = Stepper(ctx, w, el, em, e0)
        for i in range(warmup):
            step(fields[i])
        ctx.profile(True, classes=("exchange",))
        ms = timed_steps(step, fields, warmup, k, stream) / k
        ctx.profile(False)
        ex_ms, ex_n = ctx.profile_read()["exchange"]
        peak, bound, _ = exchange_peak(prec)
        ach = exchange_flop_per_walker(system) * LARGE_NW / (ex_ms / ex_n / 1000.0) / 1e12
        res = {"value": LARGE_NW / (ms / 1000.0), "unit": "walker-steps/s", "ms_per_step": ms, "steps": k,
               "e_mix": float(em[2]),
               "exchange": {"avg_launch_ms": ex_ms / ex_n, "achieved_tflops": ach, "peak": peak, "bound": bound,
                            "frac": ach / peak}}
        if prec == "mixed":
            res["kernel_ms_per_step"] = class_split(ctx, step, fields, 0, 3, stream)
        out[prec] = res
        ctx.close()
        del fields, w
        torch.cuda.empty_cache()
    out["mixed_over_fp64"] = out["mixed"]["value"] / out["fp64"]["value"]
    return out


def precision_errors(dev, cfg_name, nw=16, pre_steps=3):
    """Error of the mixed path against the FP64 path (which matches the FP64
    oracle to 1e-10) per result, from a common state: nw walkers of the
    workload after pre_steps FP64 steps are copied into a mixed context, and
    both contexts run one step with the same fields (Split-2 + Krylov 10,
    force bias recomputed) and one with re-orthonormalisation.  Reported: the
    largest |E_L| difference (the local energy of the same FP64 state through
    the mixed kernels, and after one step), the relative errors of the weights,
    walkers and log-overlaps after the step, and the orthonormality
    max |Q^H Q - I| of the mixed re-orthonormalisation."""
    import torch
    from paper_2403_02542_gb300.api import Context
    from paper_2403_02542_gb300.inputs import config_system, make_fields
    s = config_system(cfg_name)
    ctxs = {p: Context(s.h1, s.L, s.trial, s.na, s.nb, s.e_const, precision=p, device=dev)
            for p in ("fp64", "mixed")}
    w64 = ctxs["fp64"].new_walkers(nw)
    ctxs["fp64"].init_walkers(w64)
    el = torch.empty(nw, 2, dtype=torch.float64, device=dev)
    em = torch.empty(4, dtype=torch.float64, device=dev)
    ctxs["fp64"].local_energy(w64, 0.0, TAU, el, em)
    e0 = float(el[0, 0])
    for k in range(pre_steps):
        x = torch.as_tensor(make_fields(71, k, nw, s.G), device=dev)
        ctxs["fp64"].step(w64, x, TAU, e0, expm="krylov", order=KDIM)
    state = {"psi": w64.psi.clone(), "W": w64.weight.clone(), "lo": w64.logovl.clone()}

    def load(ctx):
        w = ctx.new_walkers(nw)
        w.psi.copy_(state["psi"].to(ctx.ctype))
        w.weight.copy_(state["W"])
        w.logovl.copy_(state["lo"])
        w.status.zero_()
        return w

    out = {"workload": f"{cfg_name} workload, {nw} walkers after {pre_steps} FP64 steps, tau={TAU}, "
                       "Split-2 + Krylov 10"}
    eloc = {}
    res = {}
    for p, ctx in ctxs.items():
        w = load(ctx)
        e_l = torch.empty(nw, 2, dtype=torch.float64, device=dev)
        e_m = torch.empty(4, dtype=torch.float64, device=dev)
        ctx.local_energy(w, e0, TAU, e_l, e_m)
        eloc[p] = e_l.clone()
        x = torch.as_tensor(make_fields(71, pre_steps, nw, s.G), device=dev)
        ctx.step(w, x, TAU, e0, expm="krylov", order=KDIM, measure=True, e_loc=e_l, e_mix=e_m)
        r = {"El": e_l.clone(), "W": w.weight.clone(), "lo": w.logovl.clone(),
             "psi": w.psi.to(torch.complex128).clone(), "emix": float(e_m[2])}
        w2 = load(ctx)
        ctx.step(w2, x, TAU, e0, expm="krylov", order=KDIM, reortho=True)
        r["Q"] = w2.psi.to(torch.complex128).clone()
        res[p] = r
    torch.cuda.synchronize()
    a, b = res["mixed"], res["fp64"]
    live = b["W"] > 0
    dpsi = ((a["psi"] - b["psi"]).flatten(1).norm(dim=1) / b["psi"].flatten(1).norm(dim=1))[live]
    dlo = (a["lo"] - b["lo"])
    dlo_im = torch.remainder(dlo[:, 1] + math.pi, 2 * math.pi) - math.pi
    Q = a["Q"][live]
    orth = 0.0
    for spin, (o, n) in enumerate(((0, s.na), (s.na, s.nb))):
        if n:
            q = Q[:, o:o + n, :]
            gram = q.conj() @ q.transpose(1, 2)
            orth = max(orth, float((gram - torch.eye(n, dtype=gram.dtype, device=dev)).abs().max()))
    out.update({
        "live": int(live.sum()),
        "E_L_same_state_max_abs_Ha": float((eloc["mixed"] - eloc["fp64"]).norm(dim=1).max()),
        "E_L_after_step_max_abs_Ha": float((a["El"] - b["El"]).norm(dim=1)[live].max()),
        "E_k_after_step_abs_Ha": abs(a["emix"] - b["emix"]),
        "W_after_step_max_rel": float(((a["W"] - b["W"]).abs() / b["W"])[live].max()),
        "psi_after_step_max_rel": float(dpsi.max()),
        "logovl_after_step_max_abs": float(torch.maximum(dlo[:, 0].abs(), dlo_im.abs())[live].max()),
        "mgs_orthonormality_max": orth,
    })
    for c in ctxs.values():
        c.close()
    torch.cuda.empty_cache()
    return out


def run_ours(args):
    import numpy as np
    import torch
    import torch.distributed as dist

    global NW
    NW = args.walkers
    rank, world, local = dist_env()
    if world > 1:
        dist.init_process_group("nccl", init_method="env://")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    from paper_2403_02542_gb300 import build as B
    if not B.up_to_date():
        if rank == 0:
            B.build()
        if world > 1:
            dist.barrier()

    system, ctx, w, e_loc, e_mix, e0, tune = make_context(dev, HEADLINE, args.precision, NW)
    G = system.G
    K, Wm = args.steps, args.warmup
    gen = torch.Generator(device=dev)
    gen.manual_seed(shard_seed(1234, rank))
    fields = torch.randn(Wm + K, NW, G, dtype=torch.float64, device=dev, generator=gen)
    step = Stepper(ctx, w, e_loc, e_mix, e0)
    for i in range(Wm):
        step(fields[i])
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream(dev)

    # -------- device-timed region: inputs resident in HBM; events recorded
    # only around the exchange kernel (its launch time for the roofline)
    clocks = ClockSampler(local)
    if world > 1:
        dist.barrier()
    ctx.profile(True, classes=("exchange",))
    l0 = ctx.launch_count
    ms = slowest_rank(timed_steps(step, fields, Wm, K, stream), world, dev)
    launches = ctx.launch_count - l0
    ctx.profile(False)
    ex_ms, ex_n = ctx.profile_read()["exchange"]
    clk = clocks.stop()
    if world > 1:
        dist.barrier()
    value = job_rate(NW * K, world, ms / 1000.0)
    emix_final = float(e_mix[2])

    # -------- per-class split: a separate, untimed pass with events around every launch
    split = class_split(ctx, step, fields, 0, min(K, 5), stream)

    # -------- end to end through the API with host buffers
    rng = np.random.default_rng(shard_seed(4321, rank))
    host_fields = torch.from_numpy(rng.standard_normal((K, NW, G))).pin_memory()
    x_dev = torch.empty(NW, G, dtype=torch.float64, device=dev)
    emix_host = torch.empty(4, dtype=torch.float64).pin_memory()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for i in range(K):
        x_dev.copy_(host_fields[i], non_blocking=True)
        step(x_dev)
        emix_host.copy_(e_mix, non_blocking=True)
        stream.synchronize()
        _ = float(emix_host[2])
    torch.cuda.synchronize()
    te = slowest_rank(time.perf_counter() - t0, world, dev)
    if world > 1:
        dist.barrier()
    e2e = job_rate(NW * K, world, te)
    del host_fields

    # -------- the same step replayed as a CUDA graph (one-system batch)
    graph_value = None
    if not args.only_headline:
        from paper_2403_02542_gb300.api import Batch
        batch = Batch([ctx])
        x_graph = torch.empty(NW, G, dtype=torch.float64, device=dev)
        graph_steps = 0

        def graph_step(x):
            nonlocal graph_steps
            graph_steps += 1
            x_graph.copy_(x)
            batch.step([w], [x_graph], TAU, e0, expm="krylov", order=KDIM,
                       reortho=(graph_steps % REORTHO == 0), measure=True, e_loc=[e_loc], e_mix=[e_mix],
                       reuse_bias=True)

        for i in range(2 * REORTHO):  # capture both graphs (with and without MGS)
            graph_step(fields[i % (Wm + K)])
        if world > 1:
            dist.barrier()
        tg = slowest_rank(timed_steps(graph_step, fields, 0, K, stream), world, dev)
        graph_value = job_rate(NW * K, world, tg / 1000.0)
        batch.close()
    ctx.close()
    del fields, w
    torch.cuda.empty_cache()

    # -------- the FP64 path on the same workload (walkers are independent:
    # per-walker throughput on 512 of them), for the mixed-vs-FP64 comparison
    fp64 = None
    if args.precision == "mixed" and not args.no_fp64_compare and not args.only_headline:
        nw64, k64 = min(512, NW), 2
        s64, c64, w64, el64, em64, e064, _ = make_context(dev, HEADLINE, "fp64", nw64, tune=False)
        gen64 = torch.Generator(device=dev)
        gen64.manual_seed(shard_seed(99, rank))
        f64 = torch.randn(1 + k64, nw64, G, dtype=torch.float64, device=dev, generator=gen64)
        st64 = Stepper(c64, w64, el64, em64, e064)
        st64(f64[0])
        th = slowest_rank(timed_steps(st64, f64, 1, k64, stream), world, dev)
        fp64 = {"value": job_rate(nw64 * k64, world, th / 1000.0), "walkers": nw64, "steps": k64,
                "ms_per_step": th / k64, "unit": "walker-steps/s", "e_mix": float(em64[2])}
        c64.close()
        del f64, w64
        torch.cuda.empty_cache()

    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return 0

    # -------- roofline of the dominant kernel (exchange contraction of E_L)
    peak, bound, peak_note = exchange_peak(args.precision)
    ex_flop = exchange_flop_per_walker(system) * NW
    achieved = (ex_flop / (ex_ms / ex_n / 1000.0)) / 1e12 if ex_n else None
    kname = "exchange_kernel<double> (SIMT FP64)" if args.precision == "fp64" else "exchange_tc_kernel (tcgen05 BF16x3)"
    # DRAM bytes of one exchange launch (read + write) from ncu, when taken on
    # the current kernel (None otherwise)
    traffic, traffic_note = exchange_traffic(args.precision, NW)
    total_split = sum(split.values())
    extras = {}
    if world == 1 and not args.only_headline:
        legs = [("large_workload", args.no_large, lambda: large_rates(dev)),
                ("precision_errors", args.no_precision_errors,
                 lambda: {"precision": precision_errors(dev, HEADLINE), "large": precision_errors(dev, "large")}),
                ("adjoint", args.no_adjoint, lambda: adjoint_rate(dev)),
                ("bond_scan", args.no_adjoint, lambda: bond_scan(dev)),
                ("batched_workload", args.no_batched, lambda: batched_rate(dev)),
                ("block_krylov_workload", args.no_block_krylov, lambda: block_krylov_rate(dev)),
                ("propagator_workload", args.no_propagators, lambda: propagator_rates(dev)),
                ("lanczos_workload", args.no_propagators, lambda: lanczos_rate(dev)),
                ("expm_accuracy", args.no_expm_accuracy, lambda: expm_accuracy(dev)),
                ("tau_extrapolation", args.no_tau_scan, lambda: tau_scan(dev))]
        for name, skip, fn in legs:
            if skip:
                continue
            try:
                extras[name] = fn()
            except Exception as exc:  # noqa: BLE001 - one failing leg must not end the bench line
                extras[name] = {"error": f"{type(exc).__name__}: {exc}"}
            torch.cuda.empty_cache()
    cpu = None
    if world == 1 and not args.no_cpu_baseline and not args.only_headline:
        cpu, _ = oracle_rate(system, args.cpu_sample_walkers, 2)
        try:
            cpu["batched"] = batched_cpu_rate(system, 64, 3)
        except Exception as exc:  # noqa: BLE001 - the second CPU number must not end the bench line
            cpu["batched"] = {"error": f"{type(exc).__name__}: {exc}"}
    line = {
        "metric": METRIC, "value": value, "unit": "walker-steps/s", "n_gpus": world,
        "steps": K, "warmup": Wm, "ms_per_step": ms / K, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": "f64" if args.precision == "fp64" else "f32+f64 (mixed)",
        "data": "synthetic (seeded Hamiltonian, Gaussian fields)",
        "config": config_dict(args.precision, world, NW),
        "roofline": {"kernel": kname + ": Coulomb+exchange contraction of E_L",
                     "bound": bound, "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                     "frac": (achieved / peak) if achieved else None, "traffic": traffic,
                     "traffic_source": traffic_note,
                     "flop_per_launch": ex_flop, "avg_launch_ms": ex_ms / ex_n if ex_n else None,
                     "launches_timed": ex_n, "peak_source": peak_note,
                     "share_of_step": (split.get("exchange", 0.0) / total_split) if total_split else None},
        "kernel_ms_per_step": split,
        # the whole step against the same roofline: algorithmic flops of all its parts
        "step_roofline": {"flop_per_walker_step": step_flop_per_walker(system),
                          "achieved": step_flop_per_walker(system) * NW * world / (ms / K / 1000.0) / 1e12,
                          "peak": peak, "unit": "TFLOP/s",
                          "frac": step_flop_per_walker(system) * NW * world / (ms / K / 1000.0) / 1e12 / peak},
        "cpu_baseline": cpu,
        "e2e": {"value": e2e, "unit": "walker-steps/s",
                "h2d_bytes_per_step": NW * G * 8, "d2h_bytes_per_step": 4 * 8},
        "gpu_launches": launches,
        "gemm_tiles": tune,
        "graph_value": graph_value,
        "fp64": fp64,
        "fp64_value": fp64["value"] if fp64 else None,
        "mixed_over_fp64": (value / fp64["value"]) if fp64 else None,
        "clocks": clk,
        "e_mix_last": emix_final,
    }
    line.update(extras)
    print(json.dumps(line))
    if world > 1:
        dist.destroy_process_group()
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
