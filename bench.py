#!/usr/bin/env python
"""Benchmark: one EMPSO generation of the plain elitist-PSO workload.

Workload (the headline configuration): 461 x 151 grid at 20 m with a 40-cell
damping layer (541 x 231 padded), 8th order in space, 3 s record (1414 steps),
6 Hz Ricker, seeded synthetic layered/faulted model (1500-4700 m/s), particle =
4 x 8 control nodes (natural cubic spline), swarm of 32, 16 shots, 461
receivers, FP32 wavefields.  One step = one EMPSO generation through the
public API (empso_generation): a replay of one CUDA graph that interpolates
the 32 particles, models all 32 x 16 (particle, shot) instances in one
persistent launch (kernel and cluster size picked by the autotuner on this
batch first), reduces the misfits and runs the EMPSO step.

Prints one JSON line.  value = grid-point updates per second over the padded
grid (whole job); fitness_evals_per_s alongside.  The L2 is flushed between
timed steps by writing a 256 MiB buffer outside the timed region.

--impl reference times the FP64 CPU oracle (the method restated plainly, no
GPU) on a bounded sample of the same workload and prints the same line with
"impl": "reference".
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

from paper_1905_12795_gb300 import synth  # noqa: E402

METRIC = ("grid-pt updates/s + PSO fitness evals/s at 1 GB300; wall-clock to target misfit, "
          "surrogate vs plain")
WORKLOAD = "empso-461x151-P32-S16"
BYTES_PER_UPDATE = 16          # read u^n, u^{n-1}, a; write u^{n+1} (FP32)
# FP32 lane operations per grid-point update of the on-chip kernel (an FMA
# counts one), from its ncu instruction counters: 2 (FADD2 + FFMA2 + FMUL2) +
# FADD + FFMA + FMUL per update = 2 (2.573 + 8.163 + 1.006) + 3.273 + 0.023
# (profiles/wave_resident_kernel_empso-461x151.md); the FP32 pipes retire 128
# lane operations per SM per clock
FP32_OPS_PER_UPDATE = {"wave_resident_kernel": 26.78}
FP32_LANES_PER_SM = 128
FALLBACK_HBM_GBS = 6800.0


def _args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default=WORKLOAD)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-sample-particles", type=int, default=2)
    ap.add_argument("--case", default=None,
                    help="P,S: small profiling case on the workload's grid (no JSON line)")
    ap.add_argument("--kernel", type=int, default=0, help="0 auto, 1 streaming, 2 on-chip, 3 L2 cluster")
    ap.add_argument("--cluster", type=int, default=0, help="--case: CTAs per instance (0 automatic)")
    ap.add_argument("--rows", type=int, default=0, help="--case: on-chip rows per thread (0 automatic)")
    ap.add_argument("--chains", type=int, default=0,
                    help="--gradient-case: backward chains (0: the library default)")
    ap.add_argument("--reps", type=int, default=2)
    ap.add_argument("--no-surrogate", action="store_true",
                    help="skip the surrogate-vs-plain wall-clock comparison")
    ap.add_argument("--surrogate-seeds", type=int, default=18)
    ap.add_argument("--trials", type=int, default=5, help="PSO vs EMPSO comparison trials")
    ap.add_argument("--bands", type=int, default=0, help="fwi workload: number of bands (0: all six)")
    ap.add_argument("--no-sub-workloads", action="store_true",
                    help="default run: skip the bounded uneven and hires sub-results")
    ap.add_argument("--gradient-case", type=int, default=0,
                    help="time one adjoint gradient of this many shots")
    ap.add_argument("--surrogate-case", type=int, default=0,
                    help="time the surrogate kernels alone for this many particles")
    ap.add_argument("--generations", type=int, default=0,
                    help="PSO vs EMPSO comparison generations (0: the workload's)")
    ap.add_argument("--particles", type=int, default=0,
                    help="hires workload: particles in the bounded sample (default 8)")
    return ap.parse_args()


def _setup(name):
    wl = synth.workloads()[name]
    gs = wl.grids[0]
    S = wl.shots_per_grid[0]
    Lx = (gs.nx - 1) * gs.hx
    shots = synth.shot_line(S, Lx, wl.src_z)
    rec = synth.receiver_line(gs.nx, gs.hx, wl.rec_z)
    true = synth.layered_faulted_model(gs.nx, gs.nz, gs.hx, gs.hz, seed=wl.seed_model,
                                       vmin=gs.vmin, vmax=gs.vmax)
    return wl, gs, S, shots, rec, true


def _updates_per_instance(gs, nt):
    return (gs.nx + 2 * gs.pad) * (gs.nz + 2 * gs.pad) * nt


def _peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            pk = json.load(f)
        return float(pk["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


_KERNEL_SOURCES = {"wave_kernel": "wave.cu", "wave_resident_kernel": "wave_resident.cu",
                   "wave_stream_kernel": "wave_stream.cu", "wave_l2_kernel": "wave_l2.cu"}


def _wave_source_hash(kernel):
    """First 16 hex digits of the SHA-256 of the kernel's source file."""
    with open(os.path.join(ROOT, "paper_1905_12795_gb300", "csrc", _KERNEL_SOURCES[kernel]),
              "rb") as fh:
        return hashlib.sha256(fh.read()).hexdigest()[:16]


def _traffic_from_profile(kernel, grid="empso-461x151"):
    """DRAM bytes per launch of the modelling kernel from its committed ncu
    summary, or None when absent or taken on another version of the kernel."""
    if kernel not in _KERNEL_SOURCES:
        return None
    path = os.path.join(ROOT, "profiles", f"{kernel}_{grid}.md")
    try:
        txt = open(path).read()
    except OSError:
        return None
    m = re.search(r"traffic_bytes_per_full_launch:\s*([0-9.eE+]+)", txt)
    hsh = re.search(r"kernel_source_sha256_16:\s*([0-9a-f]+)", txt)
    if not m or not hsh or hsh.group(1) != _wave_source_hash(kernel):
        return None
    return float(m.group(1))


class _Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    def __init__(self, index):
        self.proc = None
        self.path = None
        self.index = index

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={q}",
                 "--format=csv,noheader,nounits", "-lms", "200", "-f", self.path],
                stdout=subprocess.DEVNULL, stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.3)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i] == "Active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "samples": len(rows)}


def aggregate(total_ms: float, updates_per_rank: float, dist=None, device=None):
    """Whole-job throughput over N replicas: every rank runs its own swarm (the
    method has no exchange step, so replicas only); the job time is the
    slowest rank's, value = N x updates per rank / that time.  Returns
    (max_ms, value, world)."""
    world = 1
    if dist is not None and dist.is_initialized():
        import torch
        world = dist.get_world_size()
        t = torch.tensor([total_ms], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_ms = float(t.item())
    return total_ms, world * updates_per_rank / (total_ms / 1e3), world


def _cpu_baseline(wl, gs, S, shots, rec, n_particles, nt_expected):
    """Time the FP64 oracle on `n_particles` particles x all S shots (host cores)."""
    import oracle
    og = oracle.Grid(gs.nx, gs.nz, gs.hx, gs.hz, gs.pad, gs.order, gs.T, gs.f0, gs.vmax)
    assert og.nt == nt_expected
    parts = synth.random_particles(n_particles, gs.kx * gs.kz, wl.xmin, wl.xmax,
                                   seed=wl.seed_pso)
    nrec = len(rec)
    zeros = [np.zeros((og.nt, nrec)) for _ in range(S)]
    cores = os.cpu_count() or 1
    t0 = time.perf_counter()
    for p in range(n_particles):
        vel = oracle.interp_model(parts[p].reshape(gs.kz, gs.kx), gs.nz, gs.nx, 0, gs.vmin,
                                  gs.vmax)
        oracle.shot_batch(og, vel, shots, rec, [0] * S, [nrec] * S, dobs=zeros, nthreads=cores)
    el = time.perf_counter() - t0
    upd = n_particles * S * _updates_per_instance(gs, og.nt)
    return {"value": upd / el, "unit": "grid-pt updates/s", "cores": cores, "kind": "oracle",
            "sample": f"{n_particles} particles x {S} shots of the same grid "
                      f"({n_particles * S} instances, {upd:.3e} updates) in {el:.1f} s",
            "fitness_evals_per_s": n_particles / el, "seconds": el}


def run_reference(a):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    wl, gs, S, shots, rec, _ = _setup(a.workload)
    import oracle
    og = oracle.Grid(gs.nx, gs.nz, gs.hx, gs.hz, gs.pad, gs.order, gs.T, gs.f0, gs.vmax)
    steps = []
    for _ in range(a.warmup + a.steps):
        steps.append(_cpu_baseline(wl, gs, S, shots, rec, 1, og.nt))
    timed = steps[a.warmup:]
    val = float(np.mean([s["value"] for s in timed]))
    per = _updates_per_instance(gs, og.nt) * S
    cb = dict(timed[-1])
    cb["value"] = val
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": "grid-pt updates/s",
            "n_gpus": a.gpus, "steps": a.steps, "warmup": a.warmup,
            "ms_per_step": 1e3 * per / val, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": a.workload, "grid": f"{gs.nx}x{gs.nz}", "step_sample":
                       f"1 particle x {S} shots of the {wl.P}x{S} generation"},
            "cpu_baseline": cb,
            "e2e": {"value": val, "unit": "grid-pt updates/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_ours(a):
    import torch
    from paper_1905_12795_gb300 import binding as B

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    dev = torch.device("cuda", torch.cuda.current_device())

    wl, gs, S, shots, rec, true = _setup(a.workload)
    nrec = len(rec)
    grid = B.make_grid(gs.nx, gs.nz, gs.hx, gs.hz, gs.pad, gs.order, gs.T, gs.f0, gs.vmin,
                       gs.vmax, kx=gs.kx, kz=gs.kz, mode=gs.mode)
    K = gs.kx * gs.kz
    pso = B.EmpsoPso(wl.P, K, 1.2, 2.9, 0.5, 0.3, 0.25, max(1, wl.gens // 10), 1,
                     wl.seed_pso + rank)
    ctx = B.Context([grid], rec, pso, wl.xmin, wl.xmax)
    dt, nt = ctx.grid_info(0)
    sh = B.make_shots(shots, [0] * S, [nrec] * S)
    # observed data of the true model (FP32, on this GPU)
    dobs = torch.zeros(S * nt * nrec, device=dev)
    ctx.forward_traces(torch.tensor(true, dtype=torch.float32, device=dev)[None], sh, dobs)
    x = torch.zeros(wl.P, K, device=dev)
    mis = torch.zeros(wl.P, dtype=torch.float64, device=dev)
    ctx.pso_init(x)
    # pick the kernel / cluster size on this batch, then run generations as
    # replays of one captured CUDA graph (fitness of all instances + EMPSO step)
    tuned = ctx.autotune(x, sh, dobs, mis)
    ctx.pso_init(x)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream()
    ctx.set_timing(True)

    def step():
        ctx.generation(sh, dobs, mis)

    for _ in range(a.warmup):
        step()
    torch.cuda.synchronize()
    launch = ctx.last_launch()
    clocks = _Clocks(torch.cuda.current_device()) if rank == 0 else None
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    if clocks:
        clocks.start()
    step_ms, wave_ms = [], []
    for _ in range(a.steps):
        flush.fill_(1)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        step()
        e1.record(stream)
        e1.synchronize()
        step_ms.append(e0.elapsed_time(e1))
        wave_ms.append(ctx.read_timing()[1])
    torch.cuda.synchronize()
    clk = clocks.stop() if clocks else None
    total_ms = sum(step_ms)
    upd_step = wl.P * S * _updates_per_instance(gs, nt)
    total_ms, value, _ = aggregate(total_ms, upd_step * a.steps, dist, dev)
    if dist:
        dist.barrier()

    # end-to-end through the public API: the step's input (the observed
    # traces) copied from pinned host memory every step, the fitness read back
    dobs_host = dobs.cpu().pin_memory()
    mis_host = torch.zeros(wl.P, dtype=torch.float64).pin_memory()
    torch.cuda.synchronize()
    e2e_ms = []
    for _ in range(a.steps):
        flush.fill_(1)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        dobs.copy_(dobs_host, non_blocking=True)
        ctx.generation(sh, dobs, mis)
        mis_host.copy_(mis, non_blocking=True)
        e1.record(stream)
        e1.synchronize()
        e2e_ms.append(e0.elapsed_time(e1))
    ctx.set_timing(False)
    e2e_total, e2e_value, _ = aggregate(sum(e2e_ms), upd_step * a.steps, dist, dev)

    evals = world * wl.P * a.steps / (total_ms / 1e3)
    wave_mean = float(np.mean(wave_ms))
    peak, peak_kind = _peaks()
    achieved = BYTES_PER_UPDATE * upd_step / (wave_mean / 1e3) / 1e9
    kname = ctx.last_kernel_name()
    traffic = _traffic_from_profile(kname)
    rows = ctx.last_tile_rows()
    props = torch.cuda.get_device_properties(dev)
    sm_count = props.multi_processor_count
    roof_sm = None
    if kname in FP32_OPS_PER_UPDATE:
        ops = FP32_OPS_PER_UPDATE[kname]
        mhz = (clk or {}).get("sm_mhz") or 2070.0
        busy = launch[1] * ctx.last_clusters() if launch[0] == 2 else sm_count
        peak_ops = sm_count * FP32_LANES_PER_SM * mhz * 1e6
        ach_ops = ops * upd_step / (wave_mean / 1e3)
        roof_sm = {"kernel": kname, "bound": "fp32", "achieved": ach_ops / 1e12,
                   "peak": peak_ops / 1e12, "unit": "T FP32 ops/s (FMA = 1)",
                   "frac": ach_ops / peak_ops, "ops_per_update": ops,
                   "peak_from": f"{sm_count} SMs x {FP32_LANES_PER_SM} lanes x {mhz:.0f} MHz (median under load)",
                   "sms_busy": busy, "frac_of_busy_sms": ach_ops / (busy * FP32_LANES_PER_SM * mhz * 1e6)}

    cpu = None
    if rank == 0 and world == 1 and not a.no_cpu_baseline:
        cpu = _cpu_baseline(wl, gs, S, shots, rec, a.cpu_sample_particles, nt)
    sur = None
    if rank == 0 and not a.no_surrogate:
        sur = surrogate_vs_plain(a.surrogate_seeds)
        # the same comparison modelling the predicted-best 12.5 % (context for
        # the configured 25 %: fewer true evaluations per generation)
        sur12 = surrogate_vs_plain(a.surrogate_seeds, keep=0.125, train_steps=10, batch=512)
        sur["keep_12_5_percent"] = {k: sur12[k] for k in (
            "problem", "training", "reached", "faster_seeds", "median_plain_s", "median_surrogate_s",
            "median_speedup", "mean_plain_s", "mean_surrogate_s", "speedup_of_means",
            "median_surrogate_spearman")}
    subs = {}
    if rank == 0 and world == 1 and not a.no_sub_workloads:
        # bounded sub-results: one uneven generation of the mixed-resolution
        # batch (planner's shape) and a 2 x 64 sample of the hires generation
        # (autotuned over the L2 cluster kernel's sizes)
        subs["uneven"] = _uneven_result("uneven-P256-S16x2", steps=2, warmup=1, tune=False)
        subs["hires"] = _hires_result("hires-921x301-P512-S64", P=2, steps=2, warmup=1, tune_kind=3,
                                      prescreen=False)
        subs["gradient"] = _gradient_result(16, reps=5)

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "grid-pt updates/s", "n_gpus": world,
            "steps": a.steps, "warmup": a.warmup, "ms_per_step": total_ms / a.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": a.workload, "grid": f"{gs.nx}x{gs.nz} (+{gs.pad} damping)",
                       "space_order": gs.order, "nt": nt, "particles": wl.P, "shots": S,
                       "receivers": nrec, "instances_per_step": wl.P * S,
                       "updates_per_step": upd_step, "l2": "flushed (256 MiB write) between "
                       "timed steps", "parallelism": f"replicas x{world}"},
            "fitness_evals_per_s": evals,
            "e2e": {"value": e2e_value, "unit": "grid-pt updates/s",
                    "h2d_bytes_per_step": int(dobs.numel() * 4),
                    "d2h_bytes_per_step": int(mis.numel() * 8),
                    "fitness_evals_per_s": world * wl.P * a.steps / (e2e_total / 1e3)},
            "kernel": {"kind": {1: "streaming", 2: "on-chip cluster", 3: "L2 cluster"}.get(launch[0], "?"),
                       "cluster_ctas": launch[1], "rows_per_thread": rows, "autotuned": list(tuned),
                       "sm_count": sm_count,
                       "sms_busy": launch[1] * ctx.last_clusters() if launch[0] == 2 else None,
                       "step": "CUDA graph: interpolation, persistent modelling launch, "
                               "misfit reduction, EMPSO step"},
            "roofline": {"kernel": kname,
                         "bound": "hbm", "achieved": achieved,
                         "peak": peak, "peak_kind": peak_kind, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": traffic,
                         "algorithmic_bytes_per_launch": BYTES_PER_UPDATE * upd_step,
                         "kernel_ms": wave_mean},
            "roofline_sm": roof_sm,
            "gpu_launches": 5 * a.steps,
            "clocks": clk,
            "cpu_baseline": cpu,
            "surrogate_vs_plain": sur,
        }
        line.update(subs)
        print(json.dumps(line), flush=True)
    ctx.close()
    if dist:
        dist.destroy_process_group()


def surrogate_vs_plain(seeds, gens=100, P=1024, keep=0.25, train_steps=6, batch=1024, overlap=True,
                       recent=4096, min_rank_corr=0.0, patience=0, lr=1e-3):
    """Wall-clock to a target misfit, surrogate-assisted vs plain EMPSO.

    Problem: the 101 x 101 / 10 m / order-4 / 0.5 s / 10 Hz grid with a
    20-cell damping layer, one shot at (500, 20) m, 101 receivers at 20 m,
    observed data of the two-layer model (1500 / 2500 m/s, interface 500 m)
    with +5 % velocity; particles of 4 x 8 nodes in [1200, 3200] m/s, swarm
    1024.  The plain run does `gens` generations (graph replays); its final
    best misfit is the target.  The surrogate run models the predicted-best
    quarter each generation (after a one-generation warm-up), training the
    network beside the modelling (`overlap`), and stops when it reaches the
    target.  Both times include a host read of the best misfit every
    generation.  One untimed run of each comes first (module loading, first
    launches).  Policy: half of every minibatch from the newest `recent`
    pairs; the whole swarm is modelled after a pre-screened generation whose
    rank correlation fell below `min_rank_corr` (0: never) and after
    `patience` pre-screened generations in a row without a new best (0:
    never)."""
    import torch
    from paper_1905_12795_gb300 import binding as B
    wl = synth.workloads()["surrogate-101x101-P1024"]
    gs = wl.grids[0]
    rec = synth.receiver_line(gs.nx, gs.hx, wl.rec_z)
    shots = synth.shot_line(1, (gs.nx - 1) * gs.hx, wl.src_z)
    grid = B.make_grid(gs.nx, gs.nz, gs.hx, gs.hz, gs.pad, gs.order, gs.T, gs.f0, gs.vmin,
                       gs.vmax, kx=gs.kx, kz=gs.kz)
    sh = B.make_shots(shots, [0], [len(rec)])
    true = synth.two_layer_model(gs.nx, gs.nz, gs.hz) * 1.05
    K = gs.kx * gs.kz

    def one(seed, n_gens):
        pso = B.EmpsoPso(P, K, 1.2, 2.9, 0.5, 0.3, 0.25, max(1, gens // 10), 1, 12795 + seed)
        ctx = B.Context([grid], rec, pso, wl.xmin, wl.xmax)
        _, nt = ctx.grid_info(0)
        dobs = torch.zeros(nt * len(rec), device="cuda")
        ctx.forward_traces(torch.tensor(true, dtype=torch.float32, device="cuda")[None], sh, dobs)
        mis = torch.zeros(P, dtype=torch.float64, device="cuda")
        ctx.pso_init()
        ctx.generation(sh, dobs, mis)          # capture outside the clock
        ctx.pso_init()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        best, hist = float("inf"), []
        for _ in range(n_gens):
            ctx.generation(sh, dobs, mis)
            best = min(best, mis.min().item())
            hist.append((time.perf_counter() - t0, best))
        ctx.close()
        target = best
        t_plain = next(t for t, b in hist if b <= target)
        ctx = B.Context([grid], rec, pso, wl.xmin, wl.xmax)
        ctx.surrogate_init(hidden=256, capacity=50000, lr=lr, seed=seed + 1)
        ctx.surrogate_set_overlap(overlap)
        ctx.surrogate_set_policy(recent, min_rank_corr, patience)
        ctx.pso_init()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        best_s, modelled, g, t_sur, full = float("inf"), 0, 0, None, 0
        while g < 4 * n_gens:
            n_mod = ctx.surrogate_generation(sh, dobs, keep, warm=P, train_steps=train_steps,
                                             batch=batch, misfit_out=mis)
            modelled += n_mod
            full += n_mod == P
            g += 1
            best_s = min(best_s, mis.min().item())
            if best_s <= target:
                t_sur = time.perf_counter() - t0
                break
        # surrogate error against the true misfit on the final swarm
        x = torch.zeros(P, K, dtype=torch.float64, device="cuda")
        ctx.pso_get_state(x=x)
        xf = x.float().contiguous()
        pred = torch.zeros(P, device="cuda")
        ctx.surrogate_predict(xf, pred)
        true_m = torch.zeros(P, dtype=torch.float64, device="cuda")
        ctx.eval_fitness(xf, sh, dobs, true_m)
        lt = torch.log(true_m).cpu().numpy()
        lp = pred.double().cpu().numpy()
        rank = lambda v: np.argsort(np.argsort(v))  # noqa: E731
        err = {"median_abs_log_error": float(np.median(np.abs(lp - lt))),
               "spearman": float(np.corrcoef(rank(lp), rank(lt))[0, 1])}
        ctx.close()
        return {"seed": seed, "target_misfit": target, "plain_s": t_plain, "plain_models": P * n_gens,
                "surrogate_s": t_sur, "surrogate_generations": g, "surrogate_models": modelled,
                "full_generations": full,
                "surrogate_best": best_s, "surrogate_error": err}

    one(-1, 5)                                   # untimed
    runs = [one(seed, gens) for seed in range(seeds)]
    reached = [r for r in runs if r["surrogate_s"] is not None]
    med = lambda v: float(np.median(v)) if v else None  # noqa: E731
    mean = lambda v: float(np.mean(v)) if v else None  # noqa: E731
    return {"problem": f"101x101 order 4, 1 shot, swarm {P}, {gens} plain generations, keep {100 * keep:g} %",
            "training": {"steps_per_generation": train_steps, "batch": batch, "lr": lr,
                         "beside_modelling": overlap, "recent_pairs": recent,
                         "min_rank_corr": min_rank_corr, "patience": patience},
            "seeds": seeds, "reached": len(reached),
            "faster_seeds": sum(1 for r in reached if r["surrogate_s"] < r["plain_s"]),
            "median_plain_s": med([r["plain_s"] for r in runs]),
            "median_surrogate_s": med([r["surrogate_s"] for r in reached]),
            "median_speedup": med([r["plain_s"] / r["surrogate_s"] for r in reached]),
            "mean_plain_s": mean([r["plain_s"] for r in runs]),
            "mean_surrogate_s": mean([r["surrogate_s"] for r in reached]),
            "speedup_of_means": (mean([r["plain_s"] for r in runs]) / mean([r["surrogate_s"] for r in reached])
                                 if reached else None),
            "median_surrogate_abs_log_error": med([r["surrogate_error"]["median_abs_log_error"] for r in runs]),
            "median_surrogate_spearman": med([r["surrogate_error"]["spearman"] for r in runs]),
            "runs": runs}


def run_uneven(a):
    print(json.dumps(_uneven_result(a.workload, a.steps, a.warmup, tune=True)), flush=True)


def _uneven_result(workload, steps, warmup, tune):
    """Uneven batching: 256 particles x 32 shots, 16 shots on a 40 m / 3 Hz /
    4 s grid and 16 on a 20 m / 6 Hz / 3 s grid, in one persistent launch per
    generation (graph replay); shot weights 1 / E of each band.  `tune`: the
    autotuner picks the kernel shape first (else the planner's choice)."""
    import torch
    from paper_1905_12795_gb300 import binding as B
    wl = synth.workloads()[workload]
    coarse, fine = wl.grids
    grids = [B.make_grid(g.nx, g.nz, g.hx, g.hz, g.pad, g.order, g.T, g.f0, g.vmin, g.vmax,
                         kx=g.kx, kz=g.kz) for g in (coarse, fine)]
    recs = [synth.receiver_line(g.nx, g.hx, wl.rec_z) for g in (coarse, fine)]
    shots = [synth.shot_line(S, (g.nx - 1) * g.hx, wl.src_z)
             for g, S in zip((coarse, fine), wl.shots_per_grid)]
    K = coarse.kx * coarse.kz
    pso = B.EmpsoPso(wl.P, K, 1.2, 2.9, 0.5, 0.3, 0.25, 10, 1, wl.seed_pso)
    ctx = B.Context(grids, np.concatenate(recs), pso, wl.xmin, wl.xmax)
    nts = [ctx.grid_info(i)[1] for i in range(2)]
    n0 = len(recs[0])
    S0, S1 = wl.shots_per_grid
    xz = np.concatenate(shots)
    rb = [0] * S0 + [n0] * S1
    rc = [n0] * S0 + [len(recs[1])] * S1
    gid = [0] * S0 + [1] * S1
    # observed data per band from the true model of each grid, then 1/E weights
    obs = []
    for i, g in enumerate((coarse, fine)):
        true = synth.layered_faulted_model(g.nx, g.nz, g.hx, g.hz, seed=wl.seed_model)
        sh_i = B.make_shots(shots[i], [rb[0] if i == 0 else n0] * len(shots[i]),
                            [len(recs[i])] * len(shots[i]), grid_ids=[i] * len(shots[i]))
        tr = torch.zeros(len(shots[i]) * nts[i] * len(recs[i]), device="cuda")
        ctx.forward_traces(torch.tensor(true, dtype=torch.float32, device="cuda")[None], sh_i, tr)
        obs.append(tr)
    energy = [0.5 * float((o.double() ** 2).sum()) for o in obs]
    w = [1.0 / energy[0]] * S0 + [1.0 / energy[1]] * S1
    sh = B.make_shots(xz, rb, rc, grid_ids=gid, weights=w)
    dobs = torch.cat(obs)
    mis = torch.zeros(wl.P, dtype=torch.float64, device="cuda")
    x = torch.zeros(wl.P, K, device="cuda")
    ctx.pso_init(x)
    tuned = ctx.autotune(x, sh, dobs, mis) if tune else None
    ctx.pso_init()
    ctx.set_timing(True)
    for _ in range(warmup):
        ctx.generation(sh, dobs, mis)
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    clocks = _Clocks(torch.cuda.current_device())
    clocks.start()
    ms, wave = [], []
    for _ in range(steps):
        flush.fill_(1)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        ctx.generation(sh, dobs, mis)
        e1.record(stream)
        e1.synchronize()
        ms.append(e0.elapsed_time(e1))
        wave.append(ctx.read_timing()[1])
    clk = clocks.stop()
    launch = ctx.last_launch()
    upd = wl.P * sum(S * _updates_per_instance(g, nt)
                     for g, S, nt in zip((coarse, fine), wl.shots_per_grid, nts))
    total = sum(ms)
    peak, peak_kind = _peaks()
    achieved = BYTES_PER_UPDATE * upd / (np.mean(wave) / 1e3) / 1e9
    line = {"metric": METRIC, "value": upd * steps / (total / 1e3), "unit": "grid-pt updates/s",
            "n_gpus": 1, "steps": steps, "warmup": warmup, "ms_per_step": total / steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": workload, "grids": [f"{g.nx}x{g.nz}@{g.hx:g}m/{g.f0:g}Hz/"
                                                         f"{g.T:g}s nt={nt}" for g, nt in
                                                         zip((coarse, fine), nts)],
                       "particles": wl.P, "shots": list(wl.shots_per_grid),
                       "instances_per_step": wl.P * sum(wl.shots_per_grid),
                       "updates_per_step": upd, "l2": "flushed between timed steps"},
            "fitness_evals_per_s": wl.P * steps / (total / 1e3),
            "kernel": {"kind": {1: "streaming", 2: "on-chip cluster", 3: "L2 cluster"}.get(launch[0], "?"),
                       "cluster_ctas": launch[1], "rows_per_thread": ctx.last_tile_rows(),
                       "autotuned": list(tuned) if tuned else "planner's choice"},
            "roofline": {"kernel": ctx.last_kernel_name(),
                         "bound": "hbm", "achieved": achieved, "peak": peak, "peak_kind": peak_kind,
                         "unit": "GB/s", "frac": achieved / peak, "traffic": None,
                         "kernel_ms": float(np.mean(wave))},
            "gpu_launches": 5 * steps, "clocks": clk}
    ctx.close()
    return line


def _hires_prescreen(ctx_model, B, gs, rec, sh, dobs, P=32, shots=4, gens=3):
    """Surrogate pre-screening on the high-resolution grid, bounded: a swarm of
    P particles of 24 x 8 nodes on `shots` of the shots; one warm-up
    generation models everyone, then `gens` pre-screening generations model
    the predicted-best quarter.  Returns the device-synchronised wall time of
    each kind of generation."""
    import torch
    del ctx_model
    K = gs.kx * gs.kz
    grid = B.make_grid(gs.nx, gs.nz, gs.hx, gs.hz, gs.pad, gs.order, gs.T, gs.f0, gs.vmin,
                       gs.vmax, kx=gs.kx, kz=gs.kz)
    pso = B.EmpsoPso(P, K, 1.2, 2.9, 0.5, 0.3, 0.25, 2, 1, 12795)
    ctx = B.Context([grid], rec, pso, 1500.0, 4700.0)
    ctx.surrogate_init(hidden=256, capacity=4096, lr=1e-3, seed=1)
    ctx.surrogate_set_overlap(True)
    _, nt = ctx.grid_info(0)
    sub = (B.EmpsoShot * shots)(*sh[:shots])
    d = dobs[: shots * nt * len(rec)]
    mis = torch.zeros(P, dtype=torch.float64, device="cuda")
    ctx.pso_init()
    times = []
    for g in range(1 + gens):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        n = ctx.surrogate_generation(sub, d, 0.25, warm=P, train_steps=10, batch=64, misfit_out=mis)
        torch.cuda.synchronize()
        times.append((n, time.perf_counter() - t0))
    ctx.close()
    return {"swarm": P, "shots": shots, "nodes": K,
            "warm_generation": {"modelled": times[0][0], "s": times[0][1]},
            "prescreen_generations": [{"modelled": n, "s": t} for n, t in times[1:]],
            "speedup_per_generation": times[0][1] / float(np.median([t for _, t in times[1:]]))}


def run_hires(a):
    print(json.dumps(_hires_result(a.workload, a.particles or 8, a.steps, a.warmup, tune_kind=0,
                                   prescreen=True)), flush=True)


def _hires_result(workload, P, steps, warmup, tune_kind, prescreen):
    """High-resolution grid (921 x 301 at 10 m + 60 damping cells, order 8,
    12 Hz, 4 s): a bounded sample of the generation, P particles x 64 shots
    in one launch.  The instance does not fit on chip: the autotuner times the
    kernels of kind `tune_kind` (0: every kind) on this batch first and keeps
    the fastest."""
    import torch
    from paper_1905_12795_gb300 import binding as B
    wl = synth.workloads()[workload]
    gs = wl.grids[0]
    S = wl.shots_per_grid[0]
    rec = synth.receiver_line(gs.nx, gs.hx, wl.rec_z)
    shots = synth.shot_line(S, (gs.nx - 1) * gs.hx, wl.src_z)
    grid = B.make_grid(gs.nx, gs.nz, gs.hx, gs.hz, gs.pad, gs.order, gs.T, gs.f0, gs.vmin,
                       gs.vmax, kx=gs.kx, kz=gs.kz)
    ctx = B.Context([grid], rec)
    _, nt = ctx.grid_info(0)
    sh = B.make_shots(shots, [0] * S, [len(rec)] * S)
    true = synth.layered_faulted_model(gs.nx, gs.nz, gs.hx, gs.hz, seed=wl.seed_model)
    dobs = torch.zeros(S * nt * len(rec), device="cuda")
    ctx.forward_traces(torch.tensor(true, dtype=torch.float32, device="cuda")[None], sh, dobs)
    x = torch.tensor(synth.random_particles(P, gs.kx * gs.kz, wl.xmin, wl.xmax, wl.seed_pso),
                     dtype=torch.float32, device="cuda")
    mis = torch.zeros(P, dtype=torch.float64, device="cuda")
    ctx.set_kernel(tune_kind)
    tuned = ctx.autotune(x, sh, dobs, mis)
    ctx.set_timing(True)
    for _ in range(warmup):
        ctx.eval_fitness(x, sh, dobs, mis)
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream()
    ms, wave = [], []
    clocks = _Clocks(torch.cuda.current_device())
    clocks.start()
    for _ in range(steps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        ctx.eval_fitness(x, sh, dobs, mis)
        e1.record(stream)
        e1.synchronize()
        ms.append(e0.elapsed_time(e1))
        wave.append(ctx.read_timing()[1])
    clk = clocks.stop()
    launch = ctx.last_launch()
    upd = P * S * _updates_per_instance(gs, nt)
    total = sum(ms)
    peak, peak_kind = _peaks()
    achieved = BYTES_PER_UPDATE * upd / (np.mean(wave) / 1e3) / 1e9
    line = {"metric": METRIC, "value": upd * steps / (total / 1e3), "unit": "grid-pt updates/s",
            "n_gpus": 1, "steps": steps, "warmup": warmup, "ms_per_step": total / steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": workload, "grid": f"{gs.nx}x{gs.nz} (+{gs.pad} damping)",
                       "nt": nt, "sample": f"{P} particles x {S} shots of the {wl.P} x {S} "
                                           "generation (bounded sample)",
                       "updates_per_step": upd, "l2": "inputs larger than L2"},
            "fitness_evals_per_s": P * steps / (total / 1e3),
            "kernel": {"kind": {1: "streaming", 2: "on-chip cluster", 3: "L2 cluster"}.get(launch[0], "?"),
                       "cluster_ctas": launch[1], "autotuned": list(tuned)},
            "roofline": {"kernel": ctx.last_kernel_name(),
                         "bound": "hbm", "achieved": achieved, "peak": peak, "peak_kind": peak_kind,
                         "unit": "GB/s", "frac": achieved / peak,
                         "traffic": _traffic_from_profile(ctx.last_kernel_name(), "hires-921x301"),
                         "kernel_ms": float(np.mean(wave))},
            "gpu_launches": 3 * steps, "clocks": clk}
    if prescreen:
        line["surrogate_prescreen"] = _hires_prescreen(ctx, B, gs, rec, sh, dobs)
    ctx.close()
    return line


def run_compare(a):
    """Standard PSO against EMPSO (the paper's Results comparison of
    convergence), seeded trials on the paper-faithful parameterisation: the
    plain workload's grid, true model and 16 shots, a 200 m water layer, a
    level-wise irregular control grid (levels 0.75 local wavelengths apart,
    bilinear), depth-dependent search ranges around a 1-D prior linear from
    1500 to 4500 m/s.  Both variants start from the same swarm (same seed);
    PSO has the EM step switched off.  Per trial: best misfit after every
    generation, the longest stretch without improvement, and the relative
    L2 error of the final global-best model against the true model."""
    import torch
    from paper_1905_12795_gb300 import binding as B
    wl = synth.workloads()["compare-461x151-P32-S16"]
    gs, S, ex = wl.grids[0], wl.shots_per_grid[0], wl.extra
    Lx, Lz = (gs.nx - 1) * gs.hx, (gs.nz - 1) * gs.hz
    lz, lc, node_x, v1d = synth.level_layout(Lx, Lz, ex["water"], *ex["v_prior"], f0=gs.f0,
                                             frac=ex["frac"])
    K = int(lc.sum())
    lo, hi = B.level_bounds(lz, lc, float(v1d(lz[0])), float(v1d(lz[-1])), *ex["ranges"])
    true = synth.layered_faulted_model(gs.nx, gs.nz, gs.hx, gs.hz, seed=wl.seed_model,
                                       vmin=gs.vmin, vmax=gs.vmax, water_depth=ex["water"])
    rec = synth.receiver_line(gs.nx, gs.hx, wl.rec_z)
    shots = synth.shot_line(S, Lx, wl.src_z)
    grid = B.make_grid(gs.nx, gs.nz, gs.hx, gs.hz, gs.pad, gs.order, gs.T, gs.f0, gs.vmin,
                       gs.vmax, mode=gs.mode)
    sh = B.make_shots(shots, [0] * S, [len(rec)] * S)
    gens, trials, P = a.generations or wl.gens, a.trials, wl.P
    em_start = max(1, gens // 10)
    true_t = torch.tensor(true, dtype=torch.float32, device="cuda")
    dobs = None
    out = {}
    t_start = time.perf_counter()
    for name, em in (("pso", 0), ("empso", 1)):
        curves, finals, stalls, errors = [], [], [], []
        for t in range(trials):
            pso = B.EmpsoPso(P, K, 1.2, 2.9, 0.5, 0.3, 0.25, em_start, em, wl.seed_pso + t)
            ctx = B.Context([grid], rec, pso, lo, hi)
            ctx.set_levels(0, lz, lc, node_x)
            ctx.set_water(0, ex["water"], 1500.0)
            _, nt = ctx.grid_info(0)
            if dobs is None:
                dobs = torch.zeros(S * nt * len(rec), device="cuda")
                ctx.forward_traces(true_t[None], sh, dobs)
            mis = torch.zeros(P, dtype=torch.float64, device="cuda")
            ctx.pso_init()
            best, curve = float("inf"), []
            for _ in range(gens):
                ctx.generation(sh, dobs, mis)
                best = min(best, mis.min().item())
                curve.append(best)
            # global best after the last update: p[g]
            p = torch.zeros(P, K, dtype=torch.float64, device="cuda")
            gk = torch.zeros(2, dtype=torch.int32, device="cuda")
            ctx.pso_get_state(p=p, gk=gk)
            g = int(gk[0].item())
            vel = torch.zeros(1, gs.nz, gs.nx, device="cuda")
            ctx.interp(0, p[g:g + 1].float().contiguous(), vel)
            errors.append(float(torch.linalg.norm(vel[0] - true_t) / torch.linalg.norm(true_t)))
            ctx.close()
            run, longest = 0, 0
            for i in range(1, gens):
                run = run + 1 if curve[i] >= curve[i - 1] else 0
                longest = max(longest, run)
            curves.append(curve)
            finals.append(curve[-1])
            stalls.append(longest)
        c = np.array(curves)
        out[name] = {"final_best": finals, "median_final": float(np.median(finals)),
                     "median_curve": [float(v) for v in np.median(c, axis=0)],
                     "longest_stall_gens": stalls, "model_rel_l2": errors,
                     "median_model_rel_l2": float(np.median(errors))}
    wins = int(sum(e < p for e, p in zip(out["empso"]["final_best"], out["pso"]["final_best"])))
    line = {"metric": "best misfit after G generations, standard PSO vs EMPSO (seeded trials)",
            "data": "synthetic", "dtype": "f32",
            "config": {"workload": wl.name, "grid": f"{gs.nx}x{gs.nz}@{gs.hx:g}m", "shots": S,
                       "swarm": P, "generations": gens, "trials": trials, "nodes": K,
                       "levels": len(lz), "water_m": ex["water"], "em_start": em_start,
                       "c1": 1.2, "c2": 2.9, "nm_frac": 0.25, "p_em": 0.3},
            "empso_wins": wins, "pso": out["pso"], "empso": out["empso"],
            "wall_s": time.perf_counter() - t_start}
    print(json.dumps(line), flush=True)


def run_noncrime(a):
    """Non-inverse-crime search (the paper's data preparation: observed data
    recorded with a 17 Hz Ricker, low-passed below 6 Hz, modelled with a 6 Hz
    Ricker).  Observed data are modelled on a finer 921 x 301 / 10 m grid
    (order 8, 60-cell damping layer, 3 s) with a 17 Hz Ricker at the plain
    workload's 16 shots and 461 receivers, then band-limited below 6 Hz and
    resampled onto the inversion grid's time axis by empso_lowpass
    (half-width 0.5 s).  EMPSO then searches on the plain workload's 461 x 151
    / 20 m grid with a 6 Hz Ricker.  The same search on inverse-crime data
    (observed data modelled on the inversion grid itself) is the reference.
    Reports the filter's device time and, for both searches, the best misfit
    (relative to 1/2 |d_obs|^2) and the model error after the generations."""
    import torch
    from paper_1905_12795_gb300 import binding as B
    wl, gs, S, shots, rec, true = _setup("empso-461x151-P32-S16")
    fine = synth.GridSpec(921, 301, 10.0, 10.0, 60, 8, 3.0, 17.0, 4700.0)
    gf = B.make_grid(fine.nx, fine.nz, fine.hx, fine.hz, fine.pad, fine.order, fine.T, fine.f0,
                     fine.vmin, fine.vmax)
    gc = B.make_grid(gs.nx, gs.nz, gs.hx, gs.hz, gs.pad, gs.order, gs.T, gs.f0, gs.vmin, gs.vmax,
                     kx=gs.kx, kz=gs.kz, mode=gs.mode)
    nrec = len(rec)
    sh = B.make_shots(shots, [0] * S, [nrec] * S)
    cf = B.Context([gf], rec)
    dt_f, nt_f = cf.grid_info(0)
    true_f = synth.layered_faulted_model(fine.nx, fine.nz, fine.hx, fine.hz, seed=wl.seed_model,
                                         vmin=fine.vmin, vmax=fine.vmax)
    tr_f = torch.zeros(S, nt_f, nrec, device="cuda")
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    cf.forward_traces(torch.tensor(true_f, dtype=torch.float32, device="cuda")[None], sh, tr_f)
    torch.cuda.synchronize()
    fine_s = time.perf_counter() - t0
    cf.close()
    gens = a.generations or 30
    P = wl.P
    out = {}
    for name in ("non_crime", "inverse_crime"):
        pso = B.EmpsoPso(P, gs.kx * gs.kz, 1.2, 2.9, 0.5, 0.3, 0.25, max(1, gens // 10), 1,
                         wl.seed_pso)
        ctx = B.Context([gc], rec, pso, wl.xmin, wl.xmax)
        dt, nt = ctx.grid_info(0)
        dobs = torch.zeros(S, nt, nrec, device="cuda")
        extra = {}
        if name == "non_crime":
            ms = []
            for _ in range(3):
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record()
                ctx.lowpass(tr_f, dt_f, dobs, dt, 6.0, 0.5)
                e1.record()
                e1.synchronize()
                ms.append(e0.elapsed_time(e1))
            macs = S * nt * nrec * (2 * 0.5 / dt_f)
            extra = {"filter_ms": float(np.median(ms)), "filter_gmac_s": macs / (np.median(ms) / 1e3) / 1e9,
                     "fine_grid": f"{fine.nx}x{fine.nz}@{fine.hx:g}m/{fine.f0:g}Hz", "fine_nt": nt_f,
                     "fine_dt_ms": dt_f * 1e3, "fine_forward_s": fine_s}
        else:
            ctx.forward_traces(torch.tensor(true, dtype=torch.float32, device="cuda")[None], sh, dobs)
        energy = 0.5 * float((dobs.double() ** 2).sum())
        mis = torch.zeros(P, dtype=torch.float64, device="cuda")
        ctx.pso_init()
        best, curve = float("inf"), []
        for _ in range(gens):
            ctx.generation(sh, dobs, mis)
            best = min(best, mis.min().item())
            curve.append(best / energy)
        p = torch.zeros(P, gs.kx * gs.kz, dtype=torch.float64, device="cuda")
        gk = torch.zeros(2, dtype=torch.int32, device="cuda")
        ctx.pso_get_state(p=p, gk=gk)
        g = int(gk[0].item())
        vel = torch.zeros(1, gs.nz, gs.nx, device="cuda")
        ctx.interp(0, p[g:g + 1].float().contiguous(), vel)
        tt = torch.tensor(true, dtype=torch.float32, device="cuda")
        out[name] = dict(extra, best_rel_misfit=best / energy,
                         model_rel_l2=float(torch.linalg.norm(vel[0] - tt) / torch.linalg.norm(tt)),
                         curve_rel_misfit=[float(v) for v in curve])
        ctx.close()
    line = {"metric": "EMPSO on low-passed fine-grid data (non-inverse crime) vs inverse-crime data",
            "data": "synthetic", "dtype": "f32",
            "config": {"workload": "noncrime-461x151-P32-S16", "observed": "17 Hz Ricker on "
                       "921x301@10m, low-passed below 6 Hz, resampled to the 6 Hz grid's steps",
                       "inversion_grid": f"{gs.nx}x{gs.nz}@{gs.hx:g}m/{gs.f0:g}Hz",
                       "swarm": P, "shots": S, "generations": gens},
            **out}
    print(json.dumps(line), flush=True)


# algorithmic bytes per point-step of a gradient: forward 16 B (read u^n,
# u^{n-1}, a; write u^{n+1}) + adjoint step 28 B (read mu^{k+1}, mu^{k+2},
# f a, u^{k-1}, G; write mu^k, G)
ADJ_BYTES_PER_UPDATE = 44


FWI_BANDS = (4.6, 11.5, 18.4, 25.3, 32.2, 39.0)   # maximum frequencies of the paper's bands (Hz)


def run_fwi(a):
    """The paper's full workflow ("Testing approach", local FWI paragraph):
    EMPSO (32 particles of 4 x 8 control nodes, 30 generations, on the plain
    workload's 461 x 151 / 20 m grid) gives the starting model, then a
    multiscale local FWI (steepest descent, Barzilai-Borwein initial step,
    backtracking) runs 30 iterations in each of the six bands with maximum
    frequencies 4.6, 11.5, 18.4, 25.3, 32.2 and 39 Hz, with the 16th-order
    operator in space, on a grid that resolves 39 Hz (the same 9.2 km x 3 km
    area at 10 m, 60 damping cells, the same 3 s record, 16 shots and one
    receiver per horizontal node).  Each band is modelled with a Ricker of
    peak f_max / 2.5 and has its own observed data from the true model.
    Reports the model error after each stage, the misfit histories, and the
    device time of one adjoint gradient of all 16 shots with its algorithmic
    traffic against the HBM peak."""
    import torch
    from paper_1905_12795_gb300 import binding as B
    wl, gs, S, shots, rec, true = _setup("empso-461x151-P32-S16")
    nrec = len(rec)
    sh = B.make_shots(shots, [0] * S, [nrec] * S)
    tt = torch.tensor(true, dtype=torch.float32, device="cuda")
    # 1. EMPSO starting model on the plain grid
    grid = B.make_grid(gs.nx, gs.nz, gs.hx, gs.hz, gs.pad, gs.order, gs.T, gs.f0, gs.vmin, gs.vmax,
                       kx=gs.kx, kz=gs.kz, mode=gs.mode)
    K = gs.kx * gs.kz
    pso = B.EmpsoPso(wl.P, K, 1.2, 2.9, 0.5, 0.3, 0.25, 3, 1, wl.seed_pso)
    ctx = B.Context([grid], rec, pso, wl.xmin, wl.xmax)
    _, nt = ctx.grid_info(0)
    dobs = torch.zeros(S * nt * nrec, device="cuda")
    ctx.forward_traces(tt[None], sh, dobs)
    mis = torch.zeros(wl.P, dtype=torch.float64, device="cuda")
    ctx.pso_init()
    gens = a.generations or 30
    t0 = time.perf_counter()
    for _ in range(gens):
        ctx.generation(sh, dobs, mis)
    torch.cuda.synchronize()
    empso_s = time.perf_counter() - t0
    p = torch.zeros(wl.P, K, dtype=torch.float64, device="cuda")
    gk = torch.zeros(2, dtype=torch.int32, device="cuda")
    ctx.pso_get_state(p=p, gk=gk)
    best = p[int(gk[0].item())][None].float().contiguous()
    ctx.close()
    # 2. the FWI grid: the same area at 10 m, the control nodes' model on it
    h = 10.0
    fx, fz = int(round((gs.nx - 1) * gs.hx / h)) + 1, int(round((gs.nz - 1) * gs.hz / h)) + 1
    pad = 60
    true_f = torch.tensor(synth.layered_faulted_model(fx, fz, h, h, seed=wl.seed_model, vmin=gs.vmin,
                                                      vmax=gs.vmax), dtype=torch.float32, device="cuda")
    rec_f = synth.receiver_line(fx, h, wl.rec_z)
    nrec_f = len(rec_f)
    sh_f = B.make_shots(shots, [0] * S, [nrec_f] * S)
    gstart = B.make_grid(fx, fz, h, h, pad, 16, gs.T, gs.f0, gs.vmin, gs.vmax, kx=gs.kx, kz=gs.kz)
    cs = B.Context([gstart], rec_f)
    vel = torch.zeros(1, fz, fx, device="cuda")
    cs.interp(0, best, vel)
    cs.close()
    vel = vel[0].contiguous()
    err = lambda v: float(torch.linalg.norm(v - true_f) / torch.linalg.norm(true_f))  # noqa: E731
    stages = [{"stage": f"EMPSO {gens} generations ({gs.nx}x{gs.nz} @ {gs.hx:g} m)",
               "model_rel_l2": err(vel), "wall_s": empso_s}]
    grad_line = None
    iters = a.trials if a.trials != 5 else 30
    bands = FWI_BANDS[:a.bands] if a.bands else FWI_BANDS
    nt_f = 0
    for fmax in bands:
        f0 = fmax / 2.5
        gb = B.make_grid(fx, fz, h, h, pad, 16, gs.T, f0, gs.vmin, gs.vmax)
        cb = B.Context([gb], rec_f)
        _, nt_f = cb.grid_info(0)
        d_b = torch.zeros(S * nt_f * nrec_f, device="cuda")
        cb.forward_traces(true_f[None], sh_f, d_b)
        if grad_line is None:
            g = torch.zeros(1, fz, fx, device="cuda")
            cb.gradient(vel[None], sh_f, d_b, g)           # warm-up (workspace allocation)
            ms = []
            for _ in range(3):
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record()
                cb.gradient(vel[None], sh_f, d_b, g)
                e1.record()
                e1.synchronize()
                ms.append(e0.elapsed_time(e1))
            upd = S * (fx + 2 * pad) * (fz + 2 * pad) * nt_f
            t = float(np.median(ms)) / 1e3
            peak, peak_kind = _peaks()
            achieved = ADJ_BYTES_PER_UPDATE * upd / t / 1e9
            grad_line = {"gradient_ms": t * 1e3, "point_steps": upd, "space_order": 16,
                         "forward_plus_adjoint_updates_per_s": 2 * upd / t,
                         "roofline": {"kernel": "adjoint path (adj_fwd_kernel / adj_step_kernel, radius 8)",
                                      "bound": "hbm", "achieved": achieved, "peak": peak,
                                      "peak_kind": peak_kind, "unit": "GB/s",
                                      "frac": achieved / peak,
                                      "bytes_per_point_step": ADJ_BYTES_PER_UPDATE}}
        t0 = time.perf_counter()
        hist = cb.fwi(vel, sh_f, d_b, iters, gs.vmin, gs.vmax)
        torch.cuda.synchronize()
        stages.append({"stage": f"FWI band f_max {fmax} Hz (Ricker {f0:.2f} Hz)",
                       "iterations": len(hist) - 1, "misfit_first": hist[0], "misfit_last": hist[-1],
                       "misfit_history": hist, "model_rel_l2": err(vel),
                       "wall_s": time.perf_counter() - t0})
        cb.close()
    line = {"metric": "EMPSO + multiscale local FWI (16th order): model error per stage; adjoint gradient time",
            "data": "synthetic", "dtype": "f32",
            "config": {"workload": f"fwi-{fx}x{fz}-S16", "grid": f"{fx}x{fz}@{h:g}m (+{pad} damping)",
                       "space_order": 16, "shots": S, "nt": nt_f, "bands_hz": list(bands),
                       "iterations_per_band": iters},
            "stages": stages, "gradient": grad_line}
    print(json.dumps(line), flush=True)


def run_case(a):
    """P particles x S shots of the workload's grid through eval_fitness, with
    the kernel time of each repetition (used for profiler captures)."""
    import torch
    from paper_1905_12795_gb300 import binding as B
    P, S = (int(v) for v in a.case.split(","))
    wl, gs, _, _, rec, _ = _setup(a.workload)
    shots = synth.shot_line(S, (gs.nx - 1) * gs.hx, wl.src_z)
    grid = B.make_grid(gs.nx, gs.nz, gs.hx, gs.hz, gs.pad, gs.order, gs.T, gs.f0, gs.vmin,
                       gs.vmax, kx=gs.kx, kz=gs.kz, mode=gs.mode)
    ctx = B.Context([grid], rec)
    ctx.set_kernel(a.kernel)
    ctx.set_cluster(a.cluster)
    ctx.set_tile_rows(a.rows)
    _, nt = ctx.grid_info(0)
    sh = B.make_shots(shots, [0] * S, [len(rec)] * S)
    dobs = torch.zeros(S * nt * len(rec), device="cuda")
    x = torch.tensor(synth.random_particles(P, gs.kx * gs.kz, wl.xmin, wl.xmax, 1),
                     dtype=torch.float32, device="cuda")
    mis = torch.zeros(P, dtype=torch.float64, device="cuda")
    ctx.set_timing(True)
    upd = P * S * _updates_per_instance(gs, nt)
    for r in range(a.reps):
        ctx.eval_fitness(x, sh, dobs, mis)
        torch.cuda.synchronize()
        ms = ctx.read_timing()[1]
        print(f"rep {r}: modelling kernel {ms:.3f} ms, {upd / ms / 1e6:.1f} G updates/s, "
              f"launch {ctx.last_launch()} rows {ctx.last_tile_rows()} clusters {ctx.last_clusters()} "
              f"{ctx.last_kernel_name()}",
              flush=True)
    ctx.close()


def _gradient_result(S, reps):
    """The local FWI's adjoint gradient of S shots on the plain workload's
    grid (the layered/faulted model against observed data of the model +5 %),
    after one untimed call (workspace and graph): median device time, and the
    rate at ADJ_BYTES_PER_UPDATE per point-step against the HBM peak."""
    import torch
    from paper_1905_12795_gb300 import binding as B
    wl, gs, _, _, rec, true = _setup("empso-461x151-P32-S16")
    shots = synth.shot_line(S, (gs.nx - 1) * gs.hx, wl.src_z)
    grid = B.make_grid(gs.nx, gs.nz, gs.hx, gs.hz, gs.pad, gs.order, gs.T, gs.f0, gs.vmin, gs.vmax)
    ctx = B.Context([grid], rec)
    _, nt = ctx.grid_info(0)
    sh = B.make_shots(shots, [0] * S, [len(rec)] * S)
    v = torch.tensor(true, dtype=torch.float32, device="cuda")[None].contiguous()
    dobs = torch.zeros(S * nt * len(rec), device="cuda")
    ctx.forward_traces(v * 1.05, sh, dobs)
    g = torch.zeros_like(v)
    ctx.gradient(v, sh, dobs, g)
    ms = []
    for _ in range(reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        ctx.gradient(v, sh, dobs, g)
        e1.record()
        e1.synchronize()
        ms.append(e0.elapsed_time(e1))
    ctx.close()
    t = float(np.median(ms))
    upd = S * _updates_per_instance(gs, nt)
    peak, peak_kind = _peaks()
    achieved = ADJ_BYTES_PER_UPDATE * upd / (t / 1e3) / 1e9
    return {"workload": f"gradient-{gs.nx}x{gs.nz}-S{S}", "shots": S, "nt": nt, "ms": t,
            "point_steps": upd,
            "roofline": {"kernel": "adjoint path (on-chip forward with history, adj_step2_kernel)",
                         "bound": "hbm", "achieved": achieved, "peak": peak, "peak_kind": peak_kind,
                         "unit": "GB/s", "frac": achieved / peak, "bytes_per_point_step": ADJ_BYTES_PER_UPDATE}}


def run_gradient_case(a):
    """One adjoint gradient of S shots of the plain workload's grid for the
    layered/faulted model against observed data of the model +5 %, after one
    untimed call (workspace and graph); prints the device time per call and
    the traffic rate at ADJ_BYTES_PER_UPDATE per point-step (used for profiler captures)."""
    import torch
    from paper_1905_12795_gb300 import binding as B
    S = a.gradient_case
    wl, gs, _, _, rec, true = _setup("empso-461x151-P32-S16")
    shots = synth.shot_line(S, (gs.nx - 1) * gs.hx, wl.src_z)
    grid = B.make_grid(gs.nx, gs.nz, gs.hx, gs.hz, gs.pad, gs.order, gs.T, gs.f0, gs.vmin, gs.vmax)
    ctx = B.Context([grid], rec)
    if a.chains:
        ctx.set_gradient_chains(a.chains)
    ctx.set_cluster(a.cluster)
    _, nt = ctx.grid_info(0)
    sh = B.make_shots(shots, [0] * S, [len(rec)] * S)
    v = torch.tensor(true, dtype=torch.float32, device="cuda")[None].contiguous()
    dobs = torch.zeros(S * nt * len(rec), device="cuda")
    ctx.forward_traces(v * 1.05, sh, dobs)
    g = torch.zeros_like(v)
    ctx.gradient(v, sh, dobs, g)
    for r in range(a.reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        ctx.gradient(v, sh, dobs, g)
        e1.record()
        e1.synchronize()
        ms = e0.elapsed_time(e1)
        upd = S * _updates_per_instance(gs, nt)
        print(f"rep {r}: gradient of {S} shots {ms:.3f} ms, "
              f"{ADJ_BYTES_PER_UPDATE * upd / (ms / 1e3) / 1e9:.0f} GB/s at {ADJ_BYTES_PER_UPDATE} B/point-step",
              flush=True)
    ctx.close()


def run_surrogate_case(a):
    """Surrogate network kernels alone: predictions for P particles and
    20-step training rounds (batch 256, hidden 256, K = 32) with each
    dense-layer backend; prints milliseconds per call (used for profiler
    captures of the dense-layer kernels)."""
    import torch
    from paper_1905_12795_gb300 import binding as B
    P, K = a.surrogate_case, 32
    grid = B.make_grid(101, 101, 10.0, 10.0, 20, 4, 0.5, 10.0, 1200.0, 3200.0)
    pso = B.EmpsoPso(P, K, 1.2, 2.9, 0.5, 0.3, 0.25, 10, 1, 5)
    ctx = B.Context([grid], synth.receiver_line(101, 10.0, 20.0), pso, 1200.0, 3200.0)
    ctx.surrogate_init(hidden=256, capacity=50000, lr=1e-3, seed=1)
    x = torch.tensor(synth.random_particles(P, K, 1200.0, 3200.0, 3), dtype=torch.float32,
                     device="cuda")
    f = torch.rand(P, dtype=torch.float64, device="cuda") + 0.1
    for _ in range(max(1, 2048 // P)):
        ctx.surrogate_add(x, f)
    y = torch.zeros(P, device="cuda")
    for kind, name in ((0, "mma.sync"), (1, "tcgen05")):
        ctx.surrogate_set_backend(kind)
        for _ in range(a.reps):
            ctx.surrogate_train(20, 256)
            ctx.surrogate_predict(x, y)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(10):
            ctx.surrogate_train(20, 256)
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        for _ in range(50):
            ctx.surrogate_predict(x, y)
        torch.cuda.synchronize()
        t2 = time.perf_counter()
        print(f"{name}: train 20 steps {(t1 - t0) / 10 * 1e3:.3f} ms, predict {P} "
              f"{(t2 - t1) / 50 * 1e3:.4f} ms", flush=True)
    assert ctx.device_error() == 0
    ctx.close()


def main():
    a = _args()
    if a.case:
        run_case(a)
    elif a.surrogate_case:
        run_surrogate_case(a)
    elif a.gradient_case:
        run_gradient_case(a)
    elif a.impl != "reference" and a.workload.startswith("uneven"):
        run_uneven(a)
    elif a.impl != "reference" and a.workload.startswith("hires"):
        run_hires(a)
    elif a.impl != "reference" and a.workload.startswith("compare"):
        run_compare(a)
    elif a.impl != "reference" and a.workload.startswith("noncrime"):
        run_noncrime(a)
    elif a.impl != "reference" and a.workload.startswith("fwi"):
        run_fwi(a)
    elif a.impl == "reference":
        run_reference(a)
    else:
        run_ours(a)


if __name__ == "__main__":
    main()
