#!/usr/bin/env python3
"""Throughput benchmark of the fused thermal pseudopotential D2Q9 LB step.

Workload (one GPU): spinodal decomposition on a periodic 4096 x 4096 lattice,
Carnahan-Starling EOS (a = 1, b = 4, R = 1), T = 0.75 T_c, rho = 0.12 plus
seeded noise +-0.01 (seed 3), G = -1, tau_f = 1, tau_g = 0.8, mixed
pseudopotential force Eq. (4) with beta = 1.3, corrected temperature
treatment Eq. (24), FP32 populations.

A bench "step" is a segment of SEG fused LB time steps over the whole lattice
(every time step is one kernel launch that reads and writes every population
once).  The lattice state (2 x 1.23 GB ping-pong) is far larger than the
129 MB L2, so no L2 flush is needed between steps.

Metric: MLUPS (million lattice-site updates per second); value = device time
of K segments measured with CUDA events on the library's stream, max over
ranks.  ``e2e`` repeats the job through the public C ABI from pinned host
buffers: lb_init (upload of rho0, T0 and the equilibrium start) + SEG*K steps
+ lb_moments (download of rho, u, T), wall-clocked.

``sweep`` (after the timed region, not part of ``value``): the batched
solver on 256 seeded domains of the sweep recipe (L ~ U{64..512}, T/T_c,
G, tau_f drawn per domain), one persistent kernel per step with autotuned
work-list granularity, run to residual < 1e-8 with a step cap: batched MLUPS
and the wall-clock time to steady state, with converged / failed / capped
counts.

``warm_start`` (after the timed region, rank 0): the second half of the
metric, time to a steady-state residual of 1e-8, warm-started vs plain, on a
reduced case that fits the benchmark's few minutes: the network is trained
on the converged ones of 1024 solves of 128 x 128 sweep cases (60 epochs) and
128 unseen cases are solved plain (f^eq at u = 0), warm (the prediction at rest
under the force) and warm with the plain solve as fallback after 2000 steps;
wall seconds (inference included), converged / failed / capped counts and
steps on the cases both arms converge.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
Under torchrun (N > 1) every rank runs its own lattice: weak scaling, no
data-path collective (independent problems).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

NX = NY = 4096
SEG = 100                       # LB time steps per bench step
# the 16-bit modes store 16 moving populations in 16 bits and the two rest
# populations in 32 bits (FP32 deviations that close mass and energy): 40 B
# read + 40 B written per site
BYTES_PER_SITE = {"fp64": 288, "fp32": 144, "fp16": 80, "bf16": 80}
# finite-difference temperature treatment (Eqs. 26-27): f read + write and the
# T field read + write per site (rho^n, u^n and the RK2 stage fields are overhead)
BYTES_PER_SITE_FD = {"fp64": 160, "fp32": 80}
CPU_SAMPLE = 1024               # oracle sample lattice (CPU baseline / reference arm)
# Mixed force Eq. (4) with beta = 1.3: with Eq. (2) (beta = 1) this deep quench
# (T = 0.75 T_c) drives the vapour density below zero within ~200 steps, and
# beta = 1.16 still loses the psi domain at a few of the 16.8 M sites.
BETA = 1.3


def workload_params(lb, precision="fp32", thermal=None, nx=None, ny=None):
    from paper_1405_2232_gb300 import inputs as I
    nx = NX if nx is None else nx
    ny = NY if ny is None else ny
    thermal = lb.LB_THERMAL_EQ24 if thermal is None else thermal
    return lb.lb_params_default(nx=nx, ny=ny, tau_f=1.0, tau_g=0.8, G=-1.0, beta=BETA,
                                a=1.0, b=4.0, R=1.0, cv=1.0, thermal=thermal,
                                precision=precision, rho0=0.12, T0=0.75 * I.CS_TC)


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def kernel_source_hash():
    h = hashlib.sha256()
    for fn in ("lb_device.cuh", "lb_step_strip.cuh", "lb_prec_impl.cuh", "lb_prec_fp32.cu"):
        with open(os.path.join(ROOT, "paper_1405_2232_gb300", "csrc", fn), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def ncu_traffic():
    """DRAM bytes per launch of the step kernel from the committed ncu summary
    (profiles/step_traffic.txt), or None when the kernel sources changed since
    it was captured."""
    path = os.path.join(ROOT, "profiles", "step_traffic.txt")
    try:
        kv = {}
        with open(path) as fh:
            for line in fh:
                if line.startswith("#") or ":" not in line:
                    continue
                k, v = line.split(":", 1)
                kv[k.strip()] = v.strip()
        if kv.get("kernel_hash") != kernel_source_hash():
            return None
        return float(kv["dram_bytes_per_launch"])
    except Exception:
        return None


class ClockSampler:
    """nvidia-smi clock/throttle samples during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "100", "-i", str(self.gpu)],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
        return False

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx = float(parts[2])
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": mx, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def max_over_ranks(dist, value, device):
    """The largest value over all ranks (the job takes as long as its slowest rank)."""
    if not dist:
        return float(value)
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def combine_sweep(dist, wall, converged, failed, capped, sites, device):
    """Whole-job sweep result: the slowest rank's wall time, summed counts and sites."""
    if not dist:
        return float(wall), int(converged), int(failed), int(capped), int(sites)
    import torch
    res = torch.tensor([wall, converged, failed, capped, sites], dtype=torch.float64, device=device)
    mx = res.clone()
    dist.all_reduce(mx, op=dist.ReduceOp.MAX)
    dist.all_reduce(res, op=dist.ReduceOp.SUM)
    return float(mx[0]), int(res[1]), int(res[2]), int(res[3]), int(res[4])


def shard(items, rank, world, cost=None):
    """Share of independent work items of one rank (no exchange).  With a cost
    function, items are dealt longest first to the least loaded rank (ties to
    the lower rank), so ranks get about equal work when the costs are uneven;
    without one, round robin.  Every rank computes the same deal."""
    if cost is None:
        return items[rank::world]
    order = sorted(range(len(items)), key=lambda k: (-cost(items[k]), k))
    load = [0.0] * world
    mine = []
    for k in order:
        r = min(range(world), key=lambda q: (load[q], q))
        load[r] += cost(items[k])
        if r == rank:
            mine.append(k)
    return [items[k] for k in sorted(mine)]


def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def time_device(lb, ctx, stream, K, W, torch):
    """W warm-up and K timed segments of SEG steps on the library's stream."""
    for _ in range(W):
        lb.lb_step(ctx, SEG)
    stream.synchronize()
    start = torch.cuda.Event(enable_timing=True)
    stop = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    start.record(stream)
    for _ in range(K):
        lb.lb_step(ctx, SEG)
    stop.record(stream)
    stop.synchronize()
    return start.elapsed_time(stop) / 1e3


def cpu_oracle_rate(steps, threads=None):
    """The FP64 oracle as it stands, on the host cores: MLUPS on a CPU_SAMPLE^2
    sample of the spinodal workload (same recipe, smaller lattice)."""
    import oracle as O
    from paper_1405_2232_gb300 import inputs as I
    threads = threads or os.cpu_count() or 1
    rho, T = I.spinodal_fields(CPU_SAMPLE, CPU_SAMPLE)
    P = O.params(CPU_SAMPLE, CPU_SAMPLE, tau_f=1.0, tau_g=0.8, G=-1.0, beta=BETA,
                 eos=O.EOS_CS, a=1.0, b=4.0, R=1.0, thermal=O.THERMAL_EQ24)
    f, g = O.init_equilibrium(P, rho, T)
    t0 = time.perf_counter()
    O.step(P, f, g, n=steps, threads=threads, check=False)
    dt = time.perf_counter() - t0
    return CPU_SAMPLE * CPU_SAMPLE * steps / dt / 1e6, threads, dt


def run_reference(args, world, rank):
    """Reference arm: the FP64 CPU oracle, as it stands, on the host cores (rank 0
    only).  Each bench step is one oracle time step of a CPU_SAMPLE^2 lattice of
    the same spinodal recipe."""
    if rank != 0:
        return 0
    import oracle as O
    from paper_1405_2232_gb300 import inputs as I
    threads = os.cpu_count() or 1
    rho, T = I.spinodal_fields(CPU_SAMPLE, CPU_SAMPLE)
    P = O.params(CPU_SAMPLE, CPU_SAMPLE, tau_f=1.0, tau_g=0.8, G=-1.0, beta=BETA,
                 eos=O.EOS_CS, a=1.0, b=4.0, R=1.0, thermal=O.THERMAL_EQ24)
    f, g = O.init_equilibrium(P, rho, T)
    f, g, _ = O.step(P, f, g, n=args.warmup, threads=threads, check=False)
    t0 = time.perf_counter()
    O.step(P, f, g, n=args.steps, threads=threads, check=False)
    t_total = time.perf_counter() - t0
    value = CPU_SAMPLE * CPU_SAMPLE * args.steps / t_total / 1e6
    sample = f"one oracle time step of a {CPU_SAMPLE}x{CPU_SAMPLE} spinodal lattice per bench step"
    print(json.dumps({
        "impl": "reference", "metric": "MLUPS", "value": round(value, 4), "unit": "MLUPS",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": round(1e3 * t_total / args.steps, 3), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": f"spinodal CS T=0.75Tc rho=0.12+-0.01 Eq24 (oracle sample "
                               f"{CPU_SAMPLE}x{CPU_SAMPLE})", "nx": CPU_SAMPLE, "ny": CPU_SAMPLE},
        "cpu_baseline": {"value": round(value, 4), "unit": "MLUPS", "cores": threads,
                         "kind": "oracle", "sample": sample},
        "e2e": {"value": round(value, 4), "unit": "MLUPS", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }))
    return 0


def set_size(n, seg):
    global NX, NY, SEG
    NX = NY = n
    SEG = seg


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-variants", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--nx", type=int, default=NX, help="lattice side (profiling: small case)")
    ap.add_argument("--seg", type=int, default=SEG, help="LB time steps per bench step")
    ap.add_argument("--no-sweep", action="store_true", help="skip the batched-sweep run to steady state")
    ap.add_argument("--sweep-cap", type=int, default=60000, help="step cap of the batched sweep")
    ap.add_argument("--thermal", default="eq24", choices=["eq24", "fd26"],
                    help="temperature treatment of the timed lattice: Eq. (24) (the headline) "
                         "or the finite-difference Eqs. (26)-(27) (profiling)")
    ap.add_argument("--no-warm", action="store_true",
                    help="skip the warm vs plain time-to-steady-state comparison")
    ap.add_argument("--precision", default="fp32", choices=["fp32", "fp16", "bf16", "fp64"],
                    help="storage of the timed lattice: FP32 (the headline) or another mode (profiling)")
    ap.add_argument("--sweep-domains", type=int, default=256,
                    help="domains of the batched sweep (profiling: a smaller case)")
    args = ap.parse_args()
    world, rank, local = dist_setup()
    if args.impl == "reference":
        return run_reference(args, world, rank)
    set_size(args.nx, args.seg)
    if args.warmup < 3:
        args.warmup = 3

    import torch
    from paper_1405_2232_gb300 import inputs as I
    from paper_1405_2232_gb300 import lb

    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    args.dist = dist
    stream = torch.cuda.Stream()
    rho, T = I.spinodal_fields(NX, NY)
    fd = args.thermal == "fd26"
    p = workload_params(lb, precision=args.precision, thermal=lb.LB_THERMAL_FD26 if fd else None)

    # ---- device-resident timing
    d_rho = torch.from_numpy(rho).cuda()
    d_T = torch.from_numpy(T).cuda()
    torch.cuda.synchronize()
    ctx = lb.lb_init_device(p, d_rho, d_T, stream)
    lb.lb_synchronize(ctx)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    vis = os.environ.get("CUDA_VISIBLE_DEVICES")
    gpu_id = vis.split(",")[local] if vis else str(local)
    with ClockSampler(gpu_id) as clk:
        t = time_device(lb, ctx, stream, args.steps, args.warmup, torch)
    lb.lb_synchronize(ctx)  # raises if the run left the EOS domain or went non-finite
    t = max_over_ranks(dist, t, "cuda")
    sites = NX * NY
    updates = sites * SEG * args.steps
    value = world * updates / t / 1e6
    launch_s = t / (SEG * args.steps)
    alg_bytes = (BYTES_PER_SITE_FD if fd else BYTES_PER_SITE)[args.precision] * sites
    tot = lb.lb_totals(ctx)
    lb.lb_free(ctx)
    del d_rho, d_T

    # ---- end to end through the C ABI from pinned host buffers
    t_e2e = None
    if not args.no_e2e:
        t_e2e = run_e2e(lb, torch, dist, p, rho, T, stream, args)
    e2e = world * updates / t_e2e / 1e6 if t_e2e else None

    # ---- other storage modes and the Eq. (7) treatment (same lattice, shorter)
    variants = {}
    if not args.no_variants:
        variants = run_variants(lb, torch, rho, T, stream, sites)

    # ---- the batched sweep (256 domains) run to steady state
    sweep = None
    if not args.no_sweep:
        sweep = run_sweep(lb, torch, dist, world, rank, args)

    # ---- time to steady state, learned warm start vs plain (rank 0, reduced case)
    warm = None
    if not args.no_warm and rank == 0:
        from paper_1405_2232_gb300 import warmstart as WS
        warm = WS.compare()

    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return 0
    return report(args, world, value, t, launch_s, alg_bytes, tot, e2e, variants, clk, sites, sweep, warm)


def run_sweep(lb, torch, dist, world, rank, args):
    """256 seeded domains (L ~ U{64..512}), FP32, Eq. (24), beta 1.3, psi from T0;
    domains are dealt to the ranks by site count, longest first (no exchange).  Times one batched
    step (autotuned row chunks) and the run to residual < 1e-8 (K = 100)."""
    from paper_1405_2232_gb300 import inputs as I
    # domains differ up to 64x in sites: deal them to the ranks by site count
    doms = shard(I.batched_sweep(n_domains=args.sweep_domains), rank, world, cost=lambda d: d.L * d.L)
    params = [lb.lb_params_default(nx=d.L, ny=d.L, tau_f=d.tau_f, tau_g=d.tau_g, G=d.G, beta=BETA,
                                   precision="fp32", psi_uses_local_T=0, T_psi=d.T_over_Tc * I.CS_TC)
              for d in doms]
    sites = sum(q.nx * q.ny for q in params)
    with lb.Batch(params, [d.rho for d in doms], [d.T for d in doms]) as B:
        rows, _ = B.autotune(20)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        B.step(200)
        B.check()  # synchronises
        t_step = (time.perf_counter() - t0) / 200
    with lb.Batch(params, [d.rho for d in doms], [d.T for d in doms]) as B:
        B.chunk_rows = rows
        if dist:
            dist.barrier()
        t0 = time.perf_counter()
        steps, resid, st = B.run(1e-8, K=100, max_steps=args.sweep_cap)
        wall = time.perf_counter() - t0
    wall, conv, fail, capped, tot_sites = combine_sweep(
        dist, wall, int(np.sum(st == 0)), int(np.sum((st != 0) & (st != 8))), int(np.sum(st == 8)), sites,
        "cuda")
    ok = st == 0
    return {"workload": f"{args.sweep_domains} periodic domains, L~U{{64..512}}, T/Tc~U[0.6,0.95], "
                        "G~U[-1.2,-0.8], tau_f~U[0.6,1.2], droplet/slab, seed 4; FP32, Eq.24, beta 1.3, "
                        "psi(rho, T0)",
            "sites": int(tot_sites), "chunk_rows": rows,
            "batched_step_ms": round(t_step * 1e3, 3),
            "batched_MLUPS": round(world * sites / t_step / 1e6, 1),
            "tol": 1e-8, "K": 100, "max_steps": args.sweep_cap,
            "time_to_steady_s": round(wall, 2),
            "converged": int(conv), "failed": int(fail), "capped": int(capped),
            "median_steps_converged_rank0": float(np.median(steps[ok])) if ok.any() else None}


def run_e2e(lb, torch, dist, p, rho, T, stream, args):
    h_rho = torch.from_numpy(rho).pin_memory()
    h_T = torch.from_numpy(T).pin_memory()
    outs = [torch.empty((NY, NX), dtype=torch.float64).pin_memory() for _ in range(4)]
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    t0 = time.perf_counter()
    ctx = lb.lb_init(p, h_rho.numpy(), h_T.numpy(), stream)
    lb.lb_step(ctx, SEG * args.steps)
    lb.load().lb_moments(ctx, *[lb._dptr(o.numpy()) for o in outs])
    t_e2e = time.perf_counter() - t0
    lb.lb_free(ctx)
    t_e2e = max_over_ranks(dist, t_e2e, "cuda")
    return t_e2e


def run_variants(lb, torch, rho, T, stream, sites):
    variants = {}
    if True:
        for name, prec, thermal in (("fp32_eq7", "fp32", lb.LB_THERMAL_EQ7),
                                    ("fp16dev_eq24", "fp16", None), ("bf16dev_eq24", "bf16", None),
                                    ("fp64_eq24", "fp64", None),
                                    ("fp32_fd26", "fp32", lb.LB_THERMAL_FD26),
                                    ("fp64_fd26", "fp64", lb.LB_THERMAL_FD26)):
            pv = workload_params(lb, prec, thermal)
            d_rho = torch.from_numpy(rho).cuda()
            d_T = torch.from_numpy(T).cuda()
            torch.cuda.synchronize()  # the copies ran on torch's stream, the start on the library's
            c = lb.lb_init_device(pv, d_rho, d_T, stream)
            nseg = 2 if prec == "fp64" else 5
            tv = time_device(lb, c, stream, nseg, 1, torch)
            try:
                lb.lb_synchronize(c)
                ok = True
            except lb.LbError:
                ok = False
            lb.lb_free(c)
            mlups = sites * SEG * nseg / tv / 1e6
            bps = BYTES_PER_SITE_FD[prec] if thermal is not None and thermal >= lb.LB_THERMAL_FD26 else BYTES_PER_SITE[prec]
            if ok:
                variants[name] = {"MLUPS": round(mlups, 1),
                                  "GBps_algorithmic": round(bps * mlups / 1e3, 1),
                                  "state_ok": True}
            else:
                # the run left the EOS domain or went non-finite: its rate was
                # taken on a broken state and is no throughput figure
                variants[name] = {"timing_only_MLUPS": round(mlups, 1), "state_ok": False}
            del d_rho, d_T
    return variants


def report(args, world, value, t, launch_s, alg_bytes, tot, e2e, variants, clk, sites, sweep=None, warm=None):
    peak, peak_kind = peaks()
    achieved = alg_bytes / launch_s / 1e9
    cpu = None
    if not args.no_cpu_baseline and world == 1:
        v, thr, dt = cpu_oracle_rate(2)
        if dt < 5.0:
            v, thr, dt2 = cpu_oracle_rate(max(2, int(2 * 15.0 / max(dt, 1e-3))))
            dt = dt2
        cpu = {"value": round(v, 4), "unit": "MLUPS", "cores": thr, "kind": "oracle",
               "sample": f"FP64 oracle steps of a {CPU_SAMPLE}x{CPU_SAMPLE} lattice of the same "
                         f"spinodal recipe ({dt:.1f} s)"}

    fd = getattr(args, "thermal", "eq24") == "fd26"
    prec = getattr(args, "precision", "fp32")
    traffic = None if fd or prec != "fp32" else ncu_traffic()
    clocks = clk.summary()
    out = {
        "metric": "MLUPS", "value": round(value, 1), "unit": "MLUPS", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": round(1e3 * t / args.steps, 3), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64" if prec == "fp64" else "f32", "data": "synthetic",
        "config": {"workload": f"spinodal_{NX}x{NY}_CS_T0.75Tc_rho0.12pm0.01_{'fd26' if fd else 'eq24'}_{prec}",
                   "nx": NX, "ny": NY, "lb_steps_per_bench_step": SEG,
                   "thermal": "Eqs.26-27" if fd else "Eq.24", "storage": prec, "tau_f": 1.0, "tau_g": 0.8,
                   "G": -1.0,
                   "force": "Eq.4", "beta": BETA,
                   "l2": "state 2x1.23 GB > 129 MB L2, no flush needed",
                   "parallelism": f"independent lattice per GPU x{world}"},
        "roofline": {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak,
                     "unit": "GB/s", "frac": round(achieved / peak, 4),
                     "traffic": traffic, "peak_kind": peak_kind,
                     "algorithmic_bytes_per_launch": alg_bytes,
                     "avg_launch_us": round(launch_s * 1e6, 2)},
        "cpu_baseline": cpu,
        "e2e": None if e2e is None else {
            "value": round(e2e, 1), "unit": "MLUPS",
            "h2d_bytes_per_step": int(2 * 8 * sites / args.steps),
            "d2h_bytes_per_step": int(4 * 8 * sites / args.steps)},
        "gpu_launches": SEG * args.steps,
        "clocks": clocks,
        "totals_after": {"mass": tot[0], "energy": tot[1]},
        "variants": variants,
        "sweep": sweep,
        "warm_start": warm,
    }
    print(json.dumps(out))
    if args.dist:
        args.dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
