"""Benchmark of the GB300 hybrid thermal LB phase-change step.

Workload: the batched boiling-curve sweep of 32 independent square domains
(sides drawn from {256, 320, 384, 448, 512}, superheats 0.02-0.30 Tc, 3-9
nucleation sites, 25-row conjugate heater, convective top, gravity 3e-5), all
advanced together: per step one flow launch, one energy sub-step launch and one
FP64 reduction launch (split step), or one fused step launch and the reduction.
A step is one coupled update of every cell of every domain.  The metric is
coupled MLUPS over all lattice nodes (fluid and solid).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

With torchrun (N > 1) every rank runs its own replica of the sweep (the
domains are independent: no collective on the data path); the value is the
cells of all ranks divided by the slowest rank's time.  The reference arm
times the FP64 oracle on the host cores on a bounded sample of the same
workload.
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

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "coupled MLUPS (hybrid thermal LB step, batched boiling-curve sweep)"
UNIT = "MLUPS"
WORKLOAD = ("boiling-curve sweep: 32 square domains, sides {256..512} seeded, superheat 0.02-0.30 Tc, "
            "3-9 nucleation sites, 25-row heater, convective top, g = 3e-5; all domains advanced together "
            "by batched launches (step kernels + one FP64 reduction launch per step)")
BYTES_FLUID = 80  # f read 36 + f write 36 + T read 4 + T write 4
BYTES_SOLID = 8   # T read + write (no populations in solid rows)
# the split step's kernels: the flow kernel reads populations and T^n and writes
# populations, rho^n and u^n; an energy sub-step reads T, rho^n, u^n and writes T
FLOW_BYTES_FLUID = 36 + 36 + 4 + 12
ENERGY_BYTES_FLUID = 4 + 12 + 4
ENERGY_BYTES_SOLID = 8
KIND_SPLIT, KIND_FUSED, KIND_MARCH = 0, 1, 2

KERNEL_SOURCES = ("hlb_internal.cuh", "hlb_kernels.cuh", "hlb_march.cuh", "hlb_split.cuh",
                  "hlb_energy_walk.cuh")  # step kernels' device code


def kernel_source_hash() -> str:
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_1812_10375_gb300", "csrc")
    for fn in KERNEL_SOURCES:
        with open(os.path.join(csrc, fn), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def energy_kernel_name(erows):
    """The split step's energy kernel: the row-walking one (segments of erows
    rows) or the tiled one (erows = 0)."""
    return "k_energy_walk_batch" if erows > 0 else "k_energy_batch"


def kernel_name(tile, kind=KIND_FUSED, erows=-1):
    """The step kernel(s) a variant launches: the split step's flow and energy
    kernels, the fused tiled kernel, or the row-marching kernel (tile width 0)."""
    if kind == KIND_SPLIT:
        return "k_flow_batch+" + energy_kernel_name(erows)
    return "k_march_batch" if tile[0] == 0 else "k_step_batch"


def variant_key(tile, kind=KIND_FUSED, erows=-1):
    """Suffix naming a variant in the committed ncu summary: the tile, and for a
    split variant its energy kernel (walk<rows> or tile)."""
    key = "x".join(str(t) for t in tile)
    if kind == KIND_SPLIT:
        key += "_walk%d" % erows if erows > 0 else "_tile"
    return key


def profile_name(tile, kind=KIND_FUSED):
    """File stem of the committed ncu summary for a variant's step kernels."""
    return "k_flow_energy_batch" if kind == KIND_SPLIT else kernel_name(tile, kind)


def step_launches(cases, tile, kind=KIND_FUSED, nsub=1):
    """Step-kernel launches per step (the reduction aside): a flow launch and N
    energy launches for a split variant, one for a fused tiled variant, one per
    distinct row stride (width rounded up to 32) for a row-marching variant."""
    if kind == KIND_SPLIT:
        return 1 + nsub
    if tile[0] != 0:
        return 1
    return len({(c.nx + 31) // 32 for c in cases})


def read_traffic(tile, kind=KIND_FUSED, erows=-1):
    """DRAM bytes per step of the step kernel(s) from the committed ncu summary, if
    it was taken on the current kernel source and the same tile variant."""
    path = os.path.join(ROOT, "profiles", profile_name(tile, kind) + "_sweep32.md")
    if not os.path.exists(path):
        return None
    vals = {}
    with open(path) as fh:
        for line in fh:
            if line.startswith("- ") and ":" in line:
                k, v = line[2:].split(":", 1)
                vals[k.strip()] = v.strip().strip("`")
    if vals.get("kernel_source_hash") != kernel_source_hash():
        return None
    key = "dram_bytes_per_launch_full_sweep_" + variant_key(tile, kind, erows)
    try:
        return float(vals[key])
    except (KeyError, ValueError):
        return None


class ClockSampler:
    """nvidia-smi samples of the SM clock and throttle reasons during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)
        return parse_clock_lines(self.lines)


def parse_clock_lines(lines):
    """Median SM clock, the maximum clock and the throttle reasons seen active
    in nvidia-smi CSV samples of ClockSampler.FIELDS (malformed lines skipped)."""
    sm, smax, reasons = [], None, set()
    names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
    for ln in lines:
        parts = [p.strip() for p in ln.split(",")]
        if len(parts) < 7:
            continue
        # throttle reasons count whenever the line has its seven fields, even
        # if a clock field is not a number ("[N/A]")
        for nm, v in zip(names, parts[3:7]):
            if v.lower() == "active":
                reasons.add(nm)
        try:
            clk = float(parts[0])
        except ValueError:
            continue
        sm.append(clk)
        try:
            smax = float(parts[1])
        except ValueError:
            pass
    return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax,
            "reasons": sorted(reasons), "samples": len(sm)}


def aggregate(elapsed_ms: float, cells_per_rank: int, steps: int, dist=None):
    """Whole-job throughput of independent replicas: the slowest rank's time and
    the cells of all ranks.  Returns (ms_per_step, MLUPS)."""
    world = 1
    if dist is not None and dist.is_initialized():
        import torch
        world = dist.get_world_size()
        t = torch.tensor([elapsed_ms], dtype=torch.float64)
        if dist.get_backend() == "nccl":
            t = t.cuda()
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        elapsed_ms = float(t.item())
    ms_per_step = elapsed_ms / steps
    return ms_per_step, world * cells_per_rank / (ms_per_step * 1e-3) / 1e6


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def oracle_cpu_rate(seconds: float, domain_index: int = 0) -> dict:
    """Time the FP64 oracle single-threaded on one sweep domain for about `seconds`
    (run in a child process with the BLAS/OpenMP pools at one thread)."""
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
    code = f"""
import sys, time, json
sys.path.insert(0, {ROOT!r}); sys.path.insert(0, {os.path.join(ROOT, 'tests')!r})
from helpers import coexistence, oracle_domain
from paper_1812_10375_gb300 import workloads as wl
coex = coexistence()
case = wl.sweep()[{domain_index}]
d = oracle_domain(case, coex)
d.step(1)
t0 = time.perf_counter(); n = 0
while True:
    d.step(1); n += 1
    el = time.perf_counter() - t0
    if el > {seconds} and n >= 2:
        break
print(json.dumps(dict(cells=case.nx * case.ny, steps=n, seconds=el, nx=case.nx, ny=case.ny)))
"""
    out = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env, timeout=seconds * 4 + 600)
    if out.returncode != 0:
        raise RuntimeError(out.stderr[-2000:])
    r = json.loads(out.stdout.strip().splitlines()[-1])
    r["mlups"] = r["cells"] * r["steps"] / r["seconds"] / 1e6
    return r


def run_reference(args):
    """The reference arm: the FP64 oracle as it stands, on the host cores.  Each
    step is one oracle step of one domain of the sweep (cycling through the 32
    domains), so K + W steps stay within a few minutes."""
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
    code = f"""
import sys, time, json
sys.path.insert(0, {ROOT!r}); sys.path.insert(0, {os.path.join(ROOT, 'tests')!r})
from helpers import coexistence, oracle_domain
from paper_1812_10375_gb300 import workloads as wl
coex = coexistence()
cases = wl.sweep()
doms = {{}}
out = []
for k in range({args.warmup + args.steps}):
    i = k % len(cases)
    if i not in doms:
        doms[i] = oracle_domain(cases[i], coex)
    t0 = time.perf_counter()
    doms[i].step(1)
    out.append((cases[i].nx * cases[i].ny, time.perf_counter() - t0, cases[i].nx))
print(json.dumps(out))
"""
    res = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env, timeout=3600)
    if res.returncode != 0:
        print(json.dumps({"impl": "reference", "unavailable": "oracle run failed: " + res.stderr[-300:]}))
        return 0
    rows = json.loads(res.stdout.strip().splitlines()[-1])[args.warmup:]
    cells = sum(r[0] for r in rows)
    secs = sum(r[1] for r in rows)
    value = cells / secs / 1e6
    sides = sorted(set(r[2] for r in rows))
    sample = (f"{len(rows)} FP64 oracle steps, one sweep domain per step cycling over the 32 domains "
              f"(sides {sides}), one thread")
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * secs / len(rows),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD + " (reference arm: FP64 oracle, one domain per step)"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        "gpu_launches": 0,
    }
    print(json.dumps(line), flush=True)
    return 0


def build_sweep(hlb, wl, params_for, coex_lib, n_domains=None):
    import torch
    cases = wl.sweep()
    if n_domains:
        cases = cases[:n_domains]
    plist, fields, n_fluid, n_solid = [], [], 0, 0
    for c in cases:
        p, Tc = params_for(c)
        plist.append(p)
        rho0, T0 = wl.initial_fields(c, p.rho_l, p.rho_v, Tc)
        fields.append((rho0.astype("float32"), T0.astype("float32")))
        n_solid += c.wall_rows * c.nx
        n_fluid += (c.ny - c.wall_rows) * c.nx
    return cases, plist, fields, n_fluid, n_solid


def run_ours(args):
    import numpy as np
    import torch

    rank, world, local = dist_env()
    dist = None
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)

    import __graft_entry__
    __graft_entry__.build()
    from paper_1812_10375_gb300 import hlb, workloads as wl
    from paper_1812_10375_gb300.config import params_for

    cases, plist, fields, n_fluid, n_solid = build_sweep(hlb, wl, params_for, None, args.domains)
    cells = n_fluid + n_solid
    bytes_per_step = BYTES_FLUID * n_fluid + BYTES_SOLID * n_solid

    batch = hlb.Batch(plist)
    stream = batch.stream
    dev_fields = []
    for i, (r, T) in enumerate(fields):
        rt = torch.from_numpy(r).cuda()
        Tt = torch.from_numpy(T).cuda()
        batch.set_fields(i, rt, Tt)
        batch.set_nucleation_sites(i, cases[i].sites)
        dev_fields.append((rt, Tt))
    torch.cuda.synchronize()

    # warm-up
    n_ev = min(args.steps, 500)
    ev_b = [torch.cuda.Event(enable_timing=True) for _ in range(n_ev)]
    ev_f = [torch.cuda.Event(enable_timing=True) for _ in range(n_ev)]
    ev_a = [torch.cuda.Event(enable_timing=True) for _ in range(n_ev)]
    with torch.cuda.stream(stream):
        for e in ev_b + ev_f + ev_a:
            e.record(stream)  # creates the underlying cudaEvent_t
    # warm-up: the tile-shape autotuner times every compiled variant on the
    # sweep itself (ordinary steps), then the remaining warm-up steps; a fixed
    # --tile-variant skips the tuning (profiler runs, where tuning times are distorted)
    variants = hlb.tile_variants()
    kinds = hlb.variant_kinds()
    erows_all = hlb.variant_energy_rows()
    if args.tile_variant is None:
        chosen, tune_ms = batch.autotune(steps_per_variant=4)
    else:
        chosen, tune_ms = args.tile_variant, []
        batch.set_tile_variant(chosen)
    for _ in range(args.warmup):
        batch.step_profiled(None, None)
    torch.cuda.synchronize()

    kind = kinds[chosen]
    erows = erows_all[chosen]
    # timed region: K steps as the library takes them (CUDA-graph replay of
    # 16-step chunks, each step the step kernels and a reduction launch), CUDA
    # events on the batch stream around the whole region
    start = torch.cuda.Event(enable_timing=True)
    end = torch.cuda.Event(enable_timing=True)
    clocks = ClockSampler(torch.cuda.current_device())
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    time.sleep(0.3)
    start.record(stream)
    batch.step(args.steps)
    end.record(stream)
    torch.cuda.synchronize()
    # the step kernels alone for the roofline: the same steps launched one at a
    # time, with events on the batch stream before the step kernels, between
    # the flow and energy kernels (split step) and after them
    for k in range(n_ev):
        batch.step_phases(ev_b[k], ev_f[k], ev_a[k])
    torch.cuda.synchronize()
    clk = clocks.stop()
    if dist:
        dist.barrier()
    elapsed_ms = start.elapsed_time(end)
    kern_ms = [ev_b[k].elapsed_time(ev_a[k]) for k in range(n_ev)]
    ms_per_step, value = aggregate(elapsed_ms, cells, args.steps, dist)
    kern_avg_ms = sum(kern_ms) / len(kern_ms)
    kernels = None
    if kind == KIND_SPLIT:
        flow_ms = sum(ev_b[k].elapsed_time(ev_f[k]) for k in range(n_ev)) / n_ev
        en_ms = sum(ev_f[k].elapsed_time(ev_a[k]) for k in range(n_ev)) / n_ev
        fb = FLOW_BYTES_FLUID * n_fluid
        eb = ENERGY_BYTES_FLUID * n_fluid + ENERGY_BYTES_SOLID * n_solid
        kernels = {"k_flow_batch": {"ms": flow_ms, "bytes_per_launch": fb, "gbs": fb / (flow_ms * 1e-3) / 1e9},
                   energy_kernel_name(erows): {"ms": en_ms, "bytes_per_launch": eb,
                                               "gbs": eb / (en_ms * 1e-3) / 1e9}}
    diag0 = batch.diag(0, check_flags=False)

    # end to end through the public API with host buffers (skipped by --quick,
    # which profiler runs use)
    e2e = None if args.quick else run_e2e(args, hlb, plist, fields, cases, cells, dist)
    probe = probe_2048(hlb, wl, params_for, peak_gbs()) if rank == 0 and not args.quick else None
    pph = points_per_hour() if rank == 0 and not args.quick else None

    peak, peak_src = peak_gbs()
    achieved = bytes_per_step / (kern_avg_ms * 1e-3) / 1e9
    traffic = read_traffic(variants[chosen], kind, erows)
    if kernels:
        for kv in kernels.values():
            kv["frac"] = kv["gbs"] / peak

    line = None
    if rank == 0:
        cpu = (oracle_cpu_rate(seconds=12.0, domain_index=0) if not args.quick else
               {"mlups": None, "nx": None, "ny": None, "steps": 0, "seconds": 0.0})
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": WORKLOAD, "domains": len(cases), "cells_per_step": cells,
                       "fluid_cells": n_fluid, "solid_cells": n_solid,
                       "l2": "inputs larger than L2 (state %.0f MB per buffer set)" % (
                           (36 + 4) * cells / 1e6),
                       "timing": "CUDA events on the batch stream around K graph-replayed steps; the step "
                                 "kernel bracketed per step over %d further launches for the roofline" % n_ev,
                       "tile": {"chosen": list(variants[chosen]), "chosen_index": chosen,
                                "chosen_energy_walk_rows": erows,
                                "candidates_w_h_threads": [list(v) for v in variants],
                                "tuning_ms_per_step": [round(m, 4) for m in tune_ms]}},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": traffic,
                         "kernel": kernel_name(variants[chosen], kind, erows), "bytes_per_launch": bytes_per_step,
                         "bytes_note": "the step's algorithmic bytes (80 B per fluid cell, 8 B per solid cell) "
                                       "over the step kernels' time per step",
                         "kernel_ms": kern_avg_ms, "peak_source": peak_src, "per_kernel": kernels},
            "cpu_baseline": {"value": cpu["mlups"], "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": f"FP64 oracle, sweep domain 0 ({cpu['nx']}x{cpu['ny']}), "
                                       f"{cpu['steps']} steps in {cpu['seconds']:.1f} s, one thread"},
            "e2e": e2e,
            "gpu_launches": (step_launches(cases, variants[chosen], kind) + 1) * args.steps,
            "clocks": clk,
            "points_per_hour": pph,
            "probe_2048": probe,
            "diag_domain0": {"step": diag0.step, "q_bottom": diag0.q_bottom, "error_flags": diag0.error_flags},
        }
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()
    return 0


def peak_gbs():
    """The measured HBM copy bandwidth (MEASURED_PEAKS.json), else the fallback."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            peaks = json.load(fh)
        return float(peaks["hbm_gbs"]), "of measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "of fallback"


def probe_2048(hlb, wl, params_for, peak, steps=200):
    """The large single-domain roofline probe: one 2048 x 2048 pool shaped like
    the 400 x 400 case (25-row heater at Ts + 0.1 Tc, 5 seeded sites,
    convective top), advanced by the single-domain step (graph-captured), timed
    with CUDA events on the domain's stream over `steps` steps after 32 warm-up
    steps.  State 336 MB per buffer set, larger than L2."""
    import torch
    case = wl.pool(nx=2048, ny=2048, n_sites=5)
    p, Tc = params_for(case)
    rho0, T0 = wl.initial_fields(case, p.rho_l, p.rho_v, Tc)
    d = hlb.Domain(p)
    d.set_fields(torch.from_numpy(rho0.astype("float32")).cuda(), torch.from_numpy(T0.astype("float32")).cuda())
    d.set_nucleation_sites(case.sites)
    d.step(32)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(d.stream)
    d.step(steps)
    e1.record(d.stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / steps
    n_fluid = (case.ny - case.wall_rows) * case.nx
    nbytes = BYTES_FLUID * n_fluid + BYTES_SOLID * case.wall_rows * case.nx
    gbs = nbytes / (ms * 1e-3) / 1e9
    err = d.diag(check_flags=False).error_flags
    d.close()
    return {"workload": "2048 x 2048 pool, 25-row heater at Ts + 0.1 Tc, 5 sites, convective top; single-domain "
                        "step + FP64 reduction per step (graph-captured), CUDA events over %d steps" % steps,
            "ms_per_step": ms, "mlups": case.nx * case.ny / (ms * 1e-3) / 1e6,
            "achieved_gbs": gbs, "frac": gbs / peak[0], "peak": peak[0], "peak_source": peak[1],
            "bytes_per_step": nbytes, "error_flags": err}


def run_e2e(args, hlb, plist, fields, cases, cells, dist):
    """Same metric through the public API: initial fields uploaded from pinned host
    memory, K steps, then the flux histories and the final rho/T read back to host."""
    import torch
    pinned = [(torch.from_numpy(r).pin_memory(), torch.from_numpy(T).pin_memory()) for r, T in fields]
    outs = [(torch.empty(r.shape, dtype=torch.float32).pin_memory(),
             torch.empty(T.shape, dtype=torch.float32).pin_memory()) for r, T in fields]
    b = hlb.Batch(plist)
    dev = [(torch.empty(r.shape, dtype=torch.float32, device="cuda"),
            torch.empty(r.shape, dtype=torch.float32, device="cuda")) for r, _ in fields]
    for i, c in enumerate(cases):
        b.set_nucleation_sites(i, c.sites)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    t0 = time.perf_counter()
    h2d = d2h = 0
    with torch.cuda.stream(b.stream):
        for i, ((rh, Th), (rd, Td)) in enumerate(zip(pinned, dev)):
            rd.copy_(rh, non_blocking=True)
            Td.copy_(Th, non_blocking=True)
            h2d += rh.numel() * 4 + Th.numel() * 4
    for i, (rd, Td) in enumerate(dev):
        b.set_fields(i, rd, Td)
    b.step(args.steps)
    hist = [b.flux_history(i) for i in range(len(cases))]
    d2h += sum(h.nbytes for h in hist)
    for i, (ro, To) in enumerate(outs):
        rd, Td = dev[i]
        b.read_into(i, rho=rd, T=Td)
        with torch.cuda.stream(b.stream):
            ro.copy_(rd, non_blocking=True)
            To.copy_(Td, non_blocking=True)
        d2h += ro.numel() * 4 + To.numel() * 4
    torch.cuda.synchronize()
    el = time.perf_counter() - t0
    if dist:
        t = torch.tensor([el], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        el = float(t.item())
    world = int(os.environ.get("WORLD_SIZE", "1"))
    b.close()
    return {"value": world * cells * args.steps / el / 1e6, "unit": UNIT,
            "h2d_bytes_per_step": h2d / args.steps, "d2h_bytes_per_step": d2h / args.steps,
            "seconds": el}


def points_per_hour(n_points=16, full_steps=40000):
    """Boiling-curve points per hour, measured in full (no extrapolation): a
    fresh seeded set of n_points C4-shaped points (sides 256-512, 3-9 sites,
    superheats 0.02-0.30 Tc), each run to full_steps steps unless the frozen
    early-stop policy stops it at 5,000, in three arms (sweep.pph_study):
    one domain at a time, a slot-refilled batch, and the same batch with the
    policy in the loop.  Allocation is excluded from every arm; per-point
    initial fields, steps, history reads and policy calls are counted.  The
    surrogate arm's accepted points are checked against their full runs in
    the batched arm."""
    from paper_1812_10375_gb300 import sweep
    r = sweep.pph_study(n=n_points, full=full_steps)
    r["accuracy_bar"] = 0.03
    r["meets_accuracy_bar"] = bool(r["accepted_max_error"] <= 0.03)
    return r


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--tile-variant", type=int, default=None,
                    help="index into the compiled tile variants; default: autotune during warm-up")
    ap.add_argument("--domains", type=int, default=None,
                    help="run only the first N domains of the sweep (profiling on a smaller case)")
    ap.add_argument("--quick", action="store_true",
                    help="skip the end-to-end leg, the 2048 probe, points/hour and the CPU baseline")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
