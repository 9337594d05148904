#!/usr/bin/env python3
"""Throughput of the 3-D Yee leapfrog sweep on GB300 (Gcell-updates/s).

Workload: the 256^3 PEC sphere cavity (64 seeded lossy dielectric spheres,
a centre Ez Gaussian-modulated-sine source, 16 seeded Ez probes), 1000 time
steps. One bench step = one whole run of that workload through the library:
reset fields, 1000 leapfrog steps (H, E with loss, PEC, source, probes), one
energy evaluation. Inputs (fields, material words) are resident in HBM and
larger than L2 (~0.9 GB of fields per step), so no extra L2 flush is needed.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Multi-GPU: the sweep is run as independent replicas (one cavity per rank, no
collective); `value` sums the cell-updates of all ranks over the slowest rank's
time (weak scaling).

The reference arm (--impl reference) times the plain CPU oracle, unmodified, on
the host cores on a bounded sample of the same workload (same grid and
materials, fewer time steps per bench step).
"""

from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))

N_CELLS_SIDE = 256
T_STEPS = 1000
FIELD_BYTES = 48   # read + write six float32 components per cell-update
NOMINAL_HBM_GBS = 7900.0  # GB300 HBM3e, nominal (the measured copy bandwidth is the primary peak)
# Algorithmic bytes per cell and launch: the six fields read and written once
# plus a one-byte material identifier per cell (the method's minimum). The
# kernels read a 4-byte material word per index point instead (three edge
# classes and the source/probe flags), so they move 52 B; rooflines are
# reported against the algorithmic 49 B, with the 52 B figure beside them.
MAT_BYTES = 1
LAYOUT_MAT_BYTES = 4
ALG_BYTES = FIELD_BYTES + MAT_BYTES
# Field bytes per cell-update (six values read and written) of each storage form.
STORAGE_FIELD_BYTES = {"fp32": 48, "fp16": 24, "bf16": 24, "fp16hl": 48, "fp24": 36}
LAYOUT_BYTES = FIELD_BYTES + LAYOUT_MAT_BYTES
# DRAM bytes (read + write) per launch from ncu captures of each kernel on
# this workload (the kept ncu summaries), each with the launch configuration
# it was captured in (Grid.launch_config keys). A blocked launch's traffic
# depends on its work split (how many halo planes are re-read, and whether
# neighbouring tiles stream the same planes from L2 at the same time), so a
# figure is reported only for a run in the captured configuration.
NCU_TRAFFIC = {
    ("yee_blocked", 2): [({"blocked_ctas": 150, "blocked_rows": 4}, 522.219520e6 + 358.833664e6),
                         ({"blocked_ctas": 150, "blocked_rows": 2}, 876.9e6)],
    ("yee_plain", 1): [({"plain_ctas": 256}, 504.180736e6 + 361.739008e6)],
    # graded 256^3 cavity
    ("yee_plain_nu", 1): [({"plain_ctas": 256}, 509.154304e6 + 363.904512e6)],
    ("yee_blocked_nu", 2): [({"blocked_ctas": 150, "blocked_rows": 4}, 512.795648e6 + 356.909824e6),
                            ({"blocked_ctas": 152, "blocked_rows": 4}, 723.845376e6 + 370.375680e6)],
}


def ncu_traffic(kernel: str, k: int, cfg: dict):
    """(DRAM bytes per launch, the captured configurations): the bytes of the
    capture whose configuration the run shares, else None."""
    entries = NCU_TRAFFIC.get((kernel, k), [])
    for want, v in entries:
        if all(cfg.get(key) == val for key, val in want.items()):
            return v, [c for c, _ in entries]
    return None, [c for c, _ in entries]


# Batching workload: DRAM bytes per cell per launch of the batch-mode plain
# kernel (3.697188 GB for the 54436430 cells of a 300-cavity instance).
BATCH_TRAFFIC_PER_CELL = (2.349405e9 + 1.347783e9) / 54436430


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=5)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--n", type=int, default=N_CELLS_SIDE)
    p.add_argument("--tsteps", type=int, default=T_STEPS)
    p.add_argument("--k", type=int, default=0, help="steps fused per launch (0 = library default)")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-adjoint", action="store_true")
    p.add_argument("--no-batch", action="store_true")
    p.add_argument("--no-768", action="store_true")
    p.add_argument("--no-graded", action="store_true")
    p.add_argument("--graded-tsteps", type=int, default=1000, help="time steps per run of the graded-mesh workload")
    p.add_argument("--batch-cavities", type=int, default=4096)
    p.add_argument("--precision", default="fp32", choices=list(STORAGE_FIELD_BYTES),
                   help="field storage of the timed runs (arithmetic is float in every form)")
    return p.parse_args()


def peaks():
    here = os.path.dirname(os.path.abspath(__file__))
    try:
        with open(os.path.join(here, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clock/throttle samples every 200 ms while the timed region runs."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.rows = []
        self.proc = None
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([c.strip() for c in line.split(",")])

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in self.rows:
            if len(r) < 9:
                continue
            try:
                sm.append(float(r[1]))
                mx.append(float(r[2]))
            except ValueError:
                continue
            for nm, v in zip(names, r[5:9]):
                if v.strip().lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def max_over_ranks(value: float) -> float:
    """The largest `value` over all ranks (the slowest rank's time); the
    value itself when no process group is running. Works with NCCL (a CUDA
    tensor) and gloo (a host tensor)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(value)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_rate(cell_updates_per_rank: float, world: int, ms_max: float) -> float:
    """Whole-job throughput (G cell-updates/s) of `world` independent replicas:
    all ranks' updates over the slowest rank's device time (weak scaling)."""
    return cell_updates_per_rank * world / (ms_max / 1e3) / 1e9


def workload(n: int):
    from paper_1301_4539_gb300 import workloads as wl
    return wl.sphere_cavity(n)


def cpu_model() -> str:
    """The host CPU as the OS reports it (model name, else implementer/part, else the architecture)."""
    import platform
    try:
        info = open("/proc/cpuinfo").read().splitlines()
        for key in ("model name", "CPU part"):
            for line in info:
                if line.startswith(key):
                    return f"{platform.machine()} {key}: {line.split(':', 1)[1].strip()}"
    except OSError:
        pass
    return platform.machine()


def cpu_baseline(w, budget_s: float = 15.0):
    """Time the float32 oracle on the host cores on a bounded sample of the workload."""
    import oracle
    oracle.build()
    nthreads = os.cpu_count() or 1
    os.environ.setdefault("OMP_NUM_THREADS", str(nthreads))
    n = w["nx"]
    g = oracle.OracleGrid(n, n, n, w["dx"], w["dt"], "f32")
    g.set_materials(w["eps"], w["sigma"])
    for s in w["sources"]:
        g.add_source(*s)
    for p in w["probes"]:
        g.add_probe(*p)
    g.step(2)  # warm the pages and caches
    t0 = time.perf_counter()
    g.step(3)
    per = max((time.perf_counter() - t0) / 3, 1e-4)
    m = max(1, min(1000, int(budget_s / per)))
    t0 = time.perf_counter()
    g.step(m)
    dt = time.perf_counter() - t0
    g.energy()
    cells = n ** 3
    out = {"value": cells * m / dt / 1e9, "unit": "Gcell-updates/s", "cores": nthreads,
           "kind": "oracle", "cpu": cpu_model(), "cpu_count": os.cpu_count(),
           "sample": f"{n}^3 sphere cavity, float32 oracle, {m} time steps (of the {T_STEPS}-step run), "
                     f"OMP over z-planes, {dt:.1f} s"}
    # the same oracle on one core (a separate process, so that its OpenMP
    # runtime starts with one thread): 2 steps of the same workload
    code = ("import sys, time; sys.path.insert(0, %r)\n"
            "import oracle, bench\n"
            "w = bench.workload(%d)\n"
            "g = oracle.OracleGrid(%d, %d, %d, w['dx'], w['dt'], 'f32')\n"
            "g.set_materials(w['eps'], w['sigma'])\n"
            "[g.add_source(*s) for s in w['sources']]\n"
            "g.step(1)\n"
            "t = time.perf_counter(); g.step(2); print(time.perf_counter() - t)\n") % (ROOT, n, n, n, n)
    try:
        env = dict(os.environ, OMP_NUM_THREADS="1")
        r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env, timeout=300)
        t1 = float(r.stdout.strip().splitlines()[-1])
        out["one_core"] = {"value": cells * 2 / t1 / 1e9, "unit": "Gcell-updates/s", "cores": 1,
                           "sample": f"2 time steps of the same workload, {t1:.1f} s"}
    except Exception as e:  # reported, not fatal: the main baseline above stands
        out["one_core"] = {"error": str(e)[:200]}
    return out


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    w = workload(args.n)
    import oracle
    oracle.build()
    nthreads = os.cpu_count() or 1
    n = w["nx"]
    g = oracle.OracleGrid(n, n, n, w["dx"], w["dt"], "f32")
    g.set_materials(w["eps"], w["sigma"])
    for s in w["sources"]:
        g.add_source(*s)
    for p in w["probes"]:
        g.add_probe(*p)
    g.step(2)  # warm the pages and caches
    t0 = time.perf_counter()
    g.step(3)
    per = max((time.perf_counter() - t0) / 3, 1e-4)
    # each bench step: a bounded sample of the run, ~10 s of CPU work
    m = max(1, min(1000, int(10.0 / per)))
    for _ in range(args.warmup):
        g.step(1)
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        g.step(m)
        g.energy()
        times.append(time.perf_counter() - t0)
    tot = sum(times)
    val = n ** 3 * m * args.steps / tot / 1e9
    line = {"metric": "Gcell-updates/s 3D Yee FDTD", "value": val, "unit": "Gcell-updates/s",
            "impl": "reference", "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": tot / args.steps * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": f"{n}^3 PEC sphere cavity (64 lossy dielectric spheres, centre Ez "
                                   f"source, 16 probes); {m} time steps per bench step",
                       "grid": [n, n, n], "time_steps_per_bench_step": m},
            "cpu_baseline": {"value": val, "unit": "Gcell-updates/s", "cores": nthreads, "kind": "oracle",
                             "cpu": cpu_model(), "cpu_count": os.cpu_count(),
                             "sample": f"{m} time steps of the {n}^3 sphere cavity per bench step"},
            "e2e": {"value": val, "unit": "Gcell-updates/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_ours(args):
    import torch
    import torch.distributed as dist

    rank, world, local = dist_env()
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    torch.cuda.set_device(local)
    from paper_1301_4539_gb300 import sophie as so

    w = workload(args.n)
    n = w["nx"]
    cells = n ** 3
    g = so.Grid(n, n, n, w["dx"], w["dt"])
    stream = torch.cuda.current_stream()
    g.set_stream(stream.cuda_stream)
    g.set_materials(w["eps"], w["sigma"])
    for s in w["sources"]:
        g.add_source(*s)
    pids = [g.add_probe(*p) for p in w["probes"]]
    storage = {"fp32": so.FP32, "fp16": so.FP16, "bf16": so.BF16, "fp16hl": so.FP16HL, "fp24": so.FP24}
    g_prec = [storage[args.precision]]
    if args.precision in ("fp16", "fp16hl"):
        g.configure(temporal_k=1, precision=g_prec[0])
        g.set_storage_scale([2.0 ** 10] * 6)

    step_ms = []  # per bench step of the last timed() call

    def timed(k, steps, warmup, profile):
        """Device time of `steps` whole runs (reset, tsteps steps, energy) at k steps per launch."""
        g.configure(temporal_k=k, precision=g_prec[0])
        for _ in range(warmup):
            g.reset()
            g.step(args.tsteps)
            g.energy()
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        l0 = g.launch_count()
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        ev0.record(stream)
        energy = None
        marks = []  # an event after each bench step: per-step times for best / median
        torch.cuda.nvtx.range_push("timed")  # lets ncu capture only timed launches (--nvtx-include timed/)
        for si in range(steps):
            if profile and si == steps - 1:
                g.profile(True)  # per-launch events during the last bench step only (small overhead)
            g.reset()
            g.step(args.tsteps)
            energy = g.energy()
            marks.append(torch.cuda.Event(enable_timing=True))
            marks[-1].record(stream)
        torch.cuda.nvtx.range_pop()
        ev1.record(stream)
        torch.cuda.synchronize()
        ms = ev0.elapsed_time(ev1)
        step_ms.clear()
        prev = ev0
        for m in marks:
            step_ms.append(prev.elapsed_time(m))
            prev = m
        launches = g.launch_count() - l0
        prof = None
        if profile:
            prof = {kk: g.profile_read(kk) for kk in (so.KERNEL_PLAIN, so.KERNEL_BLOCKED, so.KERNEL_ENERGY)}
            g.profile(False)
        ms = max_over_ranks(ms)
        return ms, launches, prof, energy

    if args.k:
        K, tuned_ms = args.k, None
    else:
        # the library's autotuner picks k and the tilings (state untouched)
        K, tuned_ms = g.autotune()
    sampler = ClockSampler(local)
    sampler.start()
    ms, launches, prof, energy = timed(0 if not args.k else K, args.steps, args.warmup, True)
    clocks = sampler.stop()
    head_steps = sorted(step_ms)
    bench_step_ms = {"best": head_steps[0], "median": head_steps[len(head_steps) // 2], "all": list(step_ms),
                     "note": "device time of each bench step; the last one carries the per-launch events"}
    value = replica_rate(cells * args.tsteps * args.steps, world, ms)

    # dominant kernel of the timed region and its roofline
    kid = max(prof, key=lambda k: prof[k][1])
    kl, kms = prof[kid]
    alg_bytes = STORAGE_FIELD_BYTES[args.precision] + MAT_BYTES
    bytes_per_launch = cells * alg_bytes
    peak, peak_kind = peaks()
    avg_ms = kms / max(kl, 1)
    achieved = bytes_per_launch / (avg_ms / 1e3) / 1e9
    layout_bytes = STORAGE_FIELD_BYTES[args.precision] + LAYOUT_MAT_BYTES
    achieved_layout = cells * layout_bytes / (avg_ms / 1e3) / 1e9
    kname = {0: "yee_plain", 1: "yee_blocked", 2: "energy"}[kid]
    launch_cfg = g.launch_config()
    traffic, traffic_cfgs = ncu_traffic(kname, K if kid == so.KERNEL_BLOCKED else 1, launch_cfg)
    roof = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
            "traffic": traffic if args.precision == "fp32" else None, "launch_config": launch_cfg,
            "traffic_captured_configs": traffic_cfgs, "kernel": kname,
            "steps_per_launch": K if kid == so.KERNEL_BLOCKED else 1, "avg_launch_ms": avg_ms,
            "peak_source": peak_kind, "algorithmic_bytes_per_launch": bytes_per_launch,
            "algorithmic_bytes_per_cell": alg_bytes,
            "layout_bytes_per_launch": cells * layout_bytes, "achieved_layout": achieved_layout,
            "frac_layout": achieved_layout / peak,
            "kernel_share_of_timed_region": kms / (ms / args.steps),  # of the profiled bench step
            "frac_of_nominal": achieved / NOMINAL_HBM_GBS}

    # the other step kernels on the same workload (fewer runs), for comparison
    variants = {"autotuned" if not args.k else f"k{K}": value}
    nv = max(2, min(args.steps, 3))
    cfg_k1 = launch_cfg if args.k == 1 else {}
    for kk in (1, 2, 3, 4, 6, 8):
        if kk == K and args.k:
            continue
        vms, _, _, _ = timed(kk, nv, 1, False)
        variants[f"k{kk}"] = cells * args.tsteps * nv * world / (vms / 1e3) / 1e9
        if kk == 1:
            cfg_k1 = g.launch_config()
    # storage-precision forms (float arithmetic; 2-, 3- or 4-byte values in HBM)
    for pname, prec in (("fp16", so.FP16), ("bf16", so.BF16), ("fp16hl", so.FP16HL), ("fp24", so.FP24)):
        g.configure(temporal_k=1, precision=prec)
        g_prec[0] = prec
        if prec in (so.FP16, so.FP16HL):
            g.set_storage_scale([2.0 ** 10] * 6)
        for kk in (1, 2):
            vms, _, _, _ = timed(kk, nv, 1, False)
            variants[f"{pname}_k{kk}"] = cells * args.tsteps * nv * world / (vms / 1e3) / 1e9
        g_prec[0] = so.FP32
        g.configure(temporal_k=1, precision=so.FP32)
    # zero-field skipping (opt-in; not part of the headline): the same runs from
    # zero fields with the work units outside the known-nonzero box skipped
    g.set_zero_skip(True)
    vms, _, _, _ = timed(2, nv, 1, False)
    variants["k2_zero_skip"] = cells * args.tsteps * nv * world / (vms / 1e3) / 1e9
    g.set_zero_skip(False)
    variants["speedup_vs_plain"] = {k: v / variants["k1"] for k, v in variants.items() if k != "speedup_vs_plain"}
    # each form as a fraction of the HBM roof: its algorithmic bytes per
    # cell-update (fields read and written once per launch of K steps plus the
    # one-byte material identifier: float and hi+lo 48 + 1, 24-bit 36 + 1,
    # half and bfloat16 24 + 1, over K) times the rate, over the measured (and
    # the nominal) copy bandwidth
    variants_roof = {}
    for name, rate in variants.items():
        if name == "speedup_vs_plain":
            continue
        kk = K if name == "autotuned" else int(name.split("_")[0][1:]) if name[0] == "k" else int(name[-1])
        per = (FIELD_BYTES // 2 + MAT_BYTES if name.startswith(("fp16_", "bf16_"))
               else FIELD_BYTES * 3 // 4 + MAT_BYTES if name.startswith("fp24_") else ALG_BYTES) / kk
        variants_roof[name] = {"bytes_per_cell_update": per, "frac": rate * per / peaks()[0],
                               "frac_of_nominal": rate * per / NOMINAL_HBM_GBS}
    # the plain (one step per launch) kernel's own roofline on this workload
    plain_roof = {"kernel": "yee_plain", "gcell_per_s": variants["k1"],
                  "achieved_GBs_49B": variants["k1"] * ALG_BYTES,
                  "frac_49B": variants["k1"] * ALG_BYTES / peaks()[0],
                  "frac_52B_layout": variants["k1"] * LAYOUT_BYTES / peaks()[0],
                  "frac_48B_fields_only": variants["k1"] * FIELD_BYTES / peaks()[0],
                  "traffic": ncu_traffic("yee_plain", 1, cfg_k1)[0], "launch_config": cfg_k1,
                  "peak": peaks()[0], "unit": "GB/s"}
    g_prec[0] = so.FP32
    g.configure(temporal_k=0 if not args.k else K, precision=so.FP32)
    if not args.k:
        g.autotune()

    e2e = None
    if not args.no_e2e and rank == 0:
        e2e = run_e2e(args, g, w, pids, stream)

    cpu = None
    if not args.no_cpu_baseline and rank == 0 and world == 1:
        cpu = cpu_baseline(w)

    adjoint = None
    if not args.no_adjoint and rank == 0:
        adjoint = run_adjoint(stream)

    batch = None
    if not args.no_batch and rank == 0:
        batch = run_batch(args.batch_cavities, packed=True)
        batch["work_list"] = run_batch(args.batch_cavities, packed=False)
        batch["packed_over_work_list"] = batch["value"] / batch["work_list"]["value"]

    precision_768 = None
    if not args.no_768 and rank == 0:
        precision_768 = run_precision_768(stream)

    graded = None
    if not args.no_graded and rank == 0:
        graded = run_graded(stream, variants["k1"], tsteps=args.graded_tsteps, k=args.k)

    if rank == 0:
        line = {"metric": "Gcell-updates/s 3D Yee FDTD", "value": value, "unit": "Gcell-updates/s",
                "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
                "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                "config": {"workload": f"{n}^3 PEC sphere cavity (64 lossy dielectric spheres, centre Ez "
                                       f"source, 16 probes), {args.tsteps} time steps per bench step",
                           "grid": [n, n, n], "time_steps_per_bench_step": args.tsteps,
                           "temporal_k": K, "autotuned": not args.k, "parallelism": f"replicas x{world}",
                           "storage": args.precision,
                           "l2": "inputs larger than L2 (no flush)"},
                "roofline": roof, "plain_gcell_per_s": variants["k1"],
                "blocked_over_plain": value / variants["k1"],
                "plain_roofline": plain_roof, "variants_gcells": variants,
                "variants_roofline": variants_roof, "bench_step_ms": bench_step_ms, "cpu_baseline": cpu, "e2e": e2e,
                "gpu_launches": launches, "clocks": clocks, "energy_J": energy, "adjoint": adjoint,
                "batch": batch, "precision_768": precision_768, "graded_mesh": graded}
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def run_e2e(args, g, w, pids, stream):
    """Same metric through the public API with host buffers: every bench step
    uploads its materials (the host builds the material words from eps/sigma
    and copies them from pinned staging), runs, and reads the probes and the
    energy back. The steps are pipelined the way a caller streaming many runs
    would: the next step's set_materials (host build, then an upload queued on
    the grid's stream behind the running steps) is issued before this step's
    results are read, so the host build overlaps the device run."""
    import torch
    n = w["nx"]
    eps = torch.from_numpy(np.ascontiguousarray(w["eps"])).pin_memory().numpy()
    sig = torch.from_numpy(np.ascontiguousarray(w["sigma"])).pin_memory().numpy()
    reps = max(1, min(args.steps, 10))  # the same K bench steps as the device-timed value
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    g.set_materials(eps, sig)
    for r in range(reps):
        g.reset()
        g.step(args.tsteps)
        if r + 1 < reps:
            g.set_materials(eps, sig)  # the next step's inputs, uploaded after this run in stream order
        for p in pids:
            g.read_probe(p, args.tsteps)
        g.energy()
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    npts = (n + 1) * (n + 1) * (((n + 1) + 7) // 8 * 8)
    return {"value": n ** 3 * args.tsteps * reps / dt / 1e9, "unit": "Gcell-updates/s",
            "h2d_bytes_per_step": npts * 4, "d2h_bytes_per_step": len(pids) * args.tsteps * 4 + 8,
            "note": "material words built on the host from eps/sigma and uploaded each step; the next "
                    "step's host build overlaps the current run"}


def run_adjoint(stream, reps: int = 3):
    """The differentiation form on its workload (128^3 design cavity, 800 steps;
    traced record of the design box, else checkpoints every 50): wall time of one objective evaluation and of its
    gradient over the whole 32^3 design region, and the adjoint step kernel's
    HBM roofline (49 algorithmic bytes per cell: 6 float adjoint fields read and
    written, one material identifier)."""
    import torch
    from paper_1301_4539_gb300 import sophie as so
    from paper_1301_4539_gb300 import workloads as wl
    w = wl.design_cavity()
    n = w["nx"]
    N = 800
    g = so.Grid(n, n, n, w["dx"], w["dt"])
    g.set_stream(stream.cuda_stream)
    g.set_materials(w["eps"], w["sigma"])
    g.add_source(*w["sources"][0])
    k_tuned, _ = g.autotune()
    # the gradient's design box is known before the forward pass: the record
    # gathers its traces as it goes and the reverse sweep recomputes nothing
    g.objective_set_design(*w["design"])
    fwd, rev = [], []
    for r in range(reps + 1):
        g.reset()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        g.objective_forward(N, *w["probe"], 50)
        t1 = time.perf_counter()
        g.objective_grad_eps(*w["design"])
        t2 = time.perf_counter()
        if r > 0:
            fwd.append(t1 - t0)
            rev.append(t2 - t1)
    # one more evaluation with per-launch events (which keep consecutive
    # launches from overlapping), for the step kernels' own durations
    g.reset()
    g.profile(True)
    g.objective_forward(N, *w["probe"], 50)
    g.objective_grad_eps(*w["design"])
    la, ams = g.profile_read(so.KERNEL_ADJOINT)
    lp, pms = g.profile_read(so.KERNEL_PLAIN)
    g.profile(False)
    g.close()
    peak, peak_kind = peaks()
    cells = n ** 3
    avg = ams / max(la, 1)
    achieved = cells * ALG_BYTES / (avg / 1e3) / 1e9
    t_f, t_r = float(np.median(fwd)), float(np.median(rev))
    return {"workload": f"{n}^3 vacuum PEC cavity, 32^3 design region eps_r U(1,4), Gaussian-pulse Ez "
                        f"source, {N} steps, gradient over the 32^3 design cells (design box registered: the "
                        f"forward gathers its traces, no recompute)",
            "forward_ms": t_f * 1e3, "gradient_ms": t_r * 1e3, "total_ms": (t_f + t_r) * 1e3,
            "cell_steps_per_s_total": 2 * cells * N / (t_f + t_r) / 1e9,
            "unit_cell_steps": "G (forward + adjoint step) cell-updates/s",
            "adjoint_kernel": {"bound": "hbm", "avg_launch_ms": avg, "achieved": achieved, "peak": peak,
                               "unit": "GB/s", "frac": achieved / peak, "peak_source": peak_kind,
                               "launches": la},  # of the profiled evaluation
            "forward_kernel_avg_launch_ms": pms / max(lp, 1), "reps": reps,
            "forward_temporal_k": k_tuned}


def run_precision_768(stream, tsteps: int = 2000):
    """Throughput of the storage forms on the precision workload's grid: the
    768^3 sphere cavity (same generator, centre source, 16 probes), reset +
    `tsteps` steps per run, device time with CUDA events. Accuracy of the same
    forms against the FP64 oracle is measured at 256^3 by the tests."""
    import torch
    from paper_1301_4539_gb300 import sophie as so
    n = 768
    w = workload(n)
    g = so.Grid(n, n, n, w["dx"], w["dt"])
    g.set_stream(stream.cuda_stream)
    g.set_materials(w["eps"], w["sigma"])
    for src in w["sources"]:
        g.add_source(*src)
    for p in w["probes"]:
        g.add_probe(*p)
    out = {"workload": f"{n}^3 PEC sphere cavity (64 lossy spheres, centre Ez source, 16 probes), "
                       f"{tsteps} steps per run", "unit": "Gcell-updates/s"}
    for name, prec, k in (("fp32_autotuned", so.FP32, 0), ("fp32_k1", so.FP32, 1), ("fp16_k2", so.FP16, 2),
                          ("bf16_k2", so.BF16, 2), ("fp16hl_k2", so.FP16HL, 2), ("fp24_k2", so.FP24, 2)):
        g.configure(temporal_k=k, precision=prec)
        g.set_storage_scale([2.0 ** 10 if prec in (so.FP16, so.FP16HL) else 1.0] * 6)
        if k == 0:
            out["fp32_autotuned_k"], _ = g.autotune()
        g.reset()
        g.step(20)
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        ev0.record(stream)
        g.reset()
        g.step(tsteps)
        ev1.record(stream)
        torch.cuda.synchronize()
        out[name] = n ** 3 * tsteps / (ev0.elapsed_time(ev1) / 1e3) / 1e9
    g.close()
    return out


def run_graded(stream, uniform_k1: float, n: int = 256, tsteps: int = 1000, reps: int = 3, k: int = 0):
    """The non-uniform mesh on its workload: the 256^3 sphere cavity on a mesh
    refined around the source (every axis dx down to dx/2, Gaussian profile;
    dt at the refined Courant limit), reset + `tsteps` steps per run, device
    time with CUDA events, autotuned (k = 0) or at a fixed k, and the plain
    kernel (k = 1) beside it. Roofline of the dominant kernel of each: the
    same 49 algorithmic bytes per cell and launch as on the uniform mesh (the
    ratio arrays are a few KB, read from L1) over its event-timed launches."""
    import torch
    from paper_1301_4539_gb300 import sophie as so
    from paper_1301_4539_gb300 import workloads as wl
    w = wl.sphere_cavity_graded(n)
    g = so.Grid(n, n, n, w["dx"], w["dt"])
    g.set_stream(stream.cuda_stream)
    g.set_materials(w["eps"], w["sigma"])
    g.set_spacing(*w["widths"])
    for src in w["sources"]:
        g.add_source(*src)
    for p in w["probes"]:
        g.add_probe(*p)

    def one(kk):
        if kk == 0:
            kk, _ = g.autotune()
        else:
            g.configure(temporal_k=kk)
        g.reset()
        g.step(50)  # (a fixed k tunes its tilings at the first step)
        g.profile(True)
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        ev0.record(stream)
        energy = None
        torch.cuda.nvtx.range_push("timed")
        for _ in range(reps):
            g.reset()
            g.step(tsteps)
            energy = g.energy()
        torch.cuda.nvtx.range_pop()
        ev1.record(stream)
        torch.cuda.synchronize()
        ms = ev0.elapsed_time(ev1)
        prof = {kid: g.profile_read(kid) for kid in (so.KERNEL_PLAIN, so.KERNEL_BLOCKED)}
        g.profile(False)
        kid = max(prof, key=lambda q: prof[q][1])
        kl, kms = prof[kid]
        name = "yee_blocked (non-uniform)" if kid == so.KERNEL_BLOCKED else "yee_plain (non-uniform)"
        achieved = n ** 3 * ALG_BYTES / (kms / max(kl, 1) / 1e3) / 1e9
        cfg = g.launch_config()
        traffic, cfgs = ncu_traffic("yee_plain_nu" if kid == so.KERNEL_PLAIN else "yee_blocked_nu",
                                    1 if kid == so.KERNEL_PLAIN else kk, cfg)
        return kk, n ** 3 * tsteps * reps / (ms / 1e3) / 1e9, energy, {
            "kernel": name, "steps_per_launch": kk if kid == so.KERNEL_BLOCKED else 1, "bound": "hbm",
            "achieved": achieved, "peak": peaks()[0], "unit": "GB/s", "frac": achieved / peaks()[0],
            "traffic": traffic, "launch_config": cfg, "traffic_captured_configs": cfgs,
            "avg_launch_ms": kms / max(kl, 1), "launches": kl}

    kk, rate, energy, roof = one(k)
    k1, rate1, _, roof1 = one(1) if kk != 1 else (kk, rate, energy, roof)
    g.close()
    return {"workload": f"{n}^3 PEC sphere cavity on a graded mesh (widths 1 mm to 0.5 mm towards the centre "
                        f"along every axis, dt {w['dt']:.4g} s), {tsteps} steps per run",
            "gcell_per_s": rate, "unit": "Gcell-updates/s", "temporal_k": kk, "autotuned": k == 0,
            "roofline": roof, "k1_gcell_per_s": rate1, "k1_roofline": roof1,
            "k1_vs_uniform_k1": rate1 / uniform_k1, "energy_J": energy}


def run_batch(ncav: int = 4096, tsteps: int = 500, packed: bool = False):
    """The batching form on its workload: `ncav` PEC cavities with sizes
    U{16..96}^3, eps_r U(1,12) per 4^3 block, one Gaussian-pulse Ez source
    each; one run = reset + 500 steps replayed from a CUDA graph + the
    per-cavity energies. Work-list layout: one persistent launch per step over
    (cavity, tile, z chunk) items. Packed layout: the cavities in one grid
    between conducting layers, k steps per persistent temporally blocked launch
    (k and tilings autotuned). Device time of the run with CUDA events on the
    batch's stream; the roofline uses the same 49 algorithmic bytes per
    cell-update as the single grid (per cavity cell; the packed grid's own
    cells, conductors included, are in `packed_grid_cells`)."""
    import torch
    from paper_1301_4539_gb300 import sophie as so
    from paper_1301_4539_gb300 import workloads as wl
    t_setup = time.perf_counter()
    dims, eps, srcs = wl.batch_cavities(ncav=ncav)
    dt = wl.cfl_dt()
    b = so.Batch(dims, wl.DX_DEFAULT, dt, packed=packed)
    st = torch.cuda.Stream()
    b.set_stream(st.cuda_stream)
    b.set_materials(eps)
    del eps
    for s in srcs:
        b.add_source(*s)
    tx, ty, zc, tuned_ms = b.autotune()
    setup_s = time.perf_counter() - t_setup
    info = b.info()
    layout = b.layout()
    cells = int(np.prod(dims, axis=1).sum())
    b.reset()
    b.step(tsteps)  # records the graph; warm-up
    b.energy()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    runs = 2
    torch.cuda.synchronize()
    e0.record(st)
    # NVTX range for ncu filtering: "batch_timed" (packed layout) or "timed"
    torch.cuda.nvtx.range_push("batch_timed" if packed else "timed")
    for _ in range(runs):
        b.reset()
        b.step(tsteps)
    torch.cuda.nvtx.range_pop()
    e1.record(st)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / runs
    W = b.energy()
    b.close()
    rate = cells * tsteps / (ms / 1e3) / 1e9
    peak, peak_kind = peaks()
    achieved = rate * ALG_BYTES
    if packed:
        kernel = "yee_blocked (packed grid)" if layout["temporal_k"] >= 2 else "yee_plain (packed grid)"
    else:
        kernel = "yee_plain (batch work list, TMA)" if tx == 64 else "yee_batch (direct loads)"
    kk = layout["temporal_k"] if packed else 1
    return {"workload": f"{ncav} PEC cavities, sizes U{{16..96}}^3 (seed 1304), eps_r U(1,12) per 4^3 block, "
                        f"one Gaussian-pulse Ez source each, {tsteps} steps per run",
            "layout": "packed" if packed else "work list",
            "cells": cells, "value": rate, "unit": "Gcell-updates/s", "ms_per_run": ms,
            "launches_per_run": -(-tsteps // kk), "graph": True, "tiles": [tx, ty], "zchunk": zc,
            "temporal_k": kk, "packed_grid": list(layout["extent"]) if packed else None,
            "packed_grid_cells": info["work_items"] if packed else None,
            "kernel": kernel,
            "work_items": info["work_items"], "autotuned_ms_per_step": tuned_ms,
            "roofline": {"bound": "hbm", "achieved": achieved / kk, "peak": peak, "unit": "GB/s",
                         "frac": achieved / kk / peak, "peak_source": peak_kind,
                         "traffic": None if packed else BATCH_TRAFFIC_PER_CELL * cells,
                         "note": "49 algorithmic bytes per cell-update; explicit coefficient reads not counted; "
                                 "traffic per launch scaled by cells from an ncu capture of a 300-cavity "
                                 "instance of the same generator"},
            "setup_s": setup_s, "energy_sum_J": float(np.sum(W))}


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
