#!/usr/bin/env python
"""D2Q9 + NSBC throughput on one GB300: MLUPS and the HBM roofline.

One "step" is one lattice-Boltzmann time step of the whole domain: either
the staged step kernel (one producer/consumer launch: interior tiles staged
into shared memory by bulk copies, and the NSBC perimeter chunks) or the fused
pull-stream + BGK collide kernel over the interior with the NSBC kernel over
the perimeter beside it, whichever the autotuner finds faster.  Default workload: 8192 x 8192 nodes, tau 0.55, four Gaussian
acoustic pulses (amplitude 1e-3, half-width 64) at seeded centres, NSBC on
all four edges, FP32 shifted storage.

Prints ONE JSON line (rank 0).  --impl reference times the FP64 CPU oracle
(the reference for this method) on the host cores instead.
Under torchrun with N > 1 every rank runs an independent replica (a single
domain does not shard without a halo exchange); value = sum over ranks.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import re
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "D2Q9+NSBC MLUPS"
UNIT = "MLUPS"
BYTES_PER_CELL = {"f64": 144, "f32": 72, "f16": 36, "bf16": 36}
CPU_SAMPLE_N = 2048


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=2000)
    p.add_argument("--warmup", type=int, default=5)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--workload", default="pulse-8192")
    p.add_argument("--storage", default="f32", choices=list(BYTES_PER_CELL))
    p.add_argument("--no-variants", action="store_true")
    p.add_argument("--no-cpu", action="store_true")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--cpu-seconds", type=float, default=12.0)
    p.add_argument("--launch", default="",
                   help="'threads_x,rows[,prefetch]' (bulk + NSBC kernel pair), 'fused[:threads_x,rows,prefetch]' "
                        "(both in one launch), 'staged3' / 'staged4' or 'twostep' instead of autotuning")
    p.add_argument("--batched-only", action="store_true", help="time only the batched workload")
    p.add_argument("--batch-launch", default="", help="batched launch 'threads_x,rows,blocks,prefetch,split[,tma_tile]' or 'twostep'")
    p.add_argument("--batch-count", type=int, default=256,
                   help="instances of the batched workload (--batched-only; fewer for profiling captures)")
    return p.parse_args()


def workload(name: str):
    from paper_2005_08674_gb300 import inputs
    m = re.fullmatch(r"pulse-(\d+)", name)
    if not m:
        raise SystemExit(f"unknown workload {name}")
    n = int(m.group(1))
    if n == 8192:
        return inputs.pulse_8192()
    return inputs.pulse_square(n, margin=max(8, min(256, n // 4)), half_width=min(64.0, n / 16))


def describe(w, storage):
    p = w.params
    return (f"{w.name}: {w.nx}x{w.ny} D2Q9 BGK tau={w.tau}, {len(p['centres'])} Gaussian pulses "
            f"A={p['amplitude']} HWHM={p['half_width']} at seeded centres, NSBC (gamma 0.6, beta 0) "
            f"on all edges, {storage} shifted storage")


# --- clocks -------------------------------------------------------------------

class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.sel = []
        try:
            import torch
            u = str(torch.cuda.get_device_properties(device_index).uuid)
            if u:
                self.sel = ["-i", u if u.startswith("GPU-") else "GPU-" + u]
        except Exception:
            self.sel = []
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits", *self.sel,
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
        time.sleep(0.3)

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        out, _ = self.proc.communicate(timeout=10)
        sm, smax, power, reasons = [], [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 8:
                continue
            try:
                sm.append(float(f[0]))
                smax.append(float(f[1]))
                power.append(float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[4:8]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        srt = sorted(sm)
        busy = [s for s in srt if s > 0.5 * max(srt)] or srt
        return {"sm_mhz": busy[len(busy) // 2], "sm_max_mhz": max(smax), "power_w_max": max(power),
                "samples": len(sm), "reasons": sorted(reasons)}


# --- roofline inputs ------------------------------------------------------------

def measured_peak_gbs():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def kernel_source_sha() -> str:
    h = hashlib.sha256()
    for name in ("lbm_kernels.cuh", "lbm_device.cuh", "lbm_staged.cuh", "lbm_twostep.cuh"):
        with open(os.path.join(ROOT, "paper_2005_08674_gb300", "csrc", name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def step_kernel(sim, nx, ny):
    """(kernel description, traffic summary file stem, nodes whose state one
    timed launch reads and writes once) of the kernel that carries the step:
    the staged kernel updates every node, the bulk kernel the interior (the
    NSBC kernel the perimeter, beside it); a two-step pass moves every node's
    state once for two steps (one launch)."""
    if sim.twostep:
        return ("two-step pass: pass_kernel, one launch per two steps (step n+1 on the width-3 frame into a "
                "frame buffer, steps n+1 and n+2 on nodes 2..n-3 by warps rolling down 128-column strips with "
                "step n+1 in registers, step n+2 on the width-2 frame)", "twostep_traffic", nx * ny)
    if sim.staged:
        return ("batch_ws_kernel (staged step: interior tiles by bulk copies + NSBC chunks, "
                f"{sim.staged} stages)", "staged_step_traffic", nx * ny)
    if sim.fused:
        return "fused_step_kernel (bulk rows + NSBC quads in one launch)", "fused_step_traffic", nx * ny
    return "bulk_kernel (fused pull-stream + BGK collide)", "bulk_kernel_traffic", (nx - 2) * (ny - 2)


def profiled_traffic(stem: str, storage: str, cells: int):
    """DRAM bytes per launch from the committed ncu summary, scaled by the
    cells one launch processes, if the kernel source is unchanged since then."""
    path = os.path.join(ROOT, "profiles", f"{stem}_{storage}.md")
    if not os.path.exists(path):
        return None
    text = open(path).read()
    m_sha = re.search(r"kernel_source_sha:\s*([0-9a-f]+)", text)
    m_b = re.search(r"dram_bytes_per_cell:\s*([0-9.]+)", text)
    if not m_sha or not m_b or m_sha.group(1) != kernel_source_sha():
        return None
    return float(m_b.group(1)) * cells


# --- CPU oracle (baseline / reference arm) --------------------------------------

def oracle_sample_workload():
    from paper_2005_08674_gb300 import inputs
    return inputs.pulse_square(CPU_SAMPLE_N, steps=0)


def cpu_threads() -> int:
    v = os.environ.get("OMP_NUM_THREADS")
    return int(v) if v and v.isdigit() else (os.cpu_count() or 1)


def time_oracle(seconds: float, warmup: int = 1, fixed_steps: int | None = None, openmp: bool = True):
    import oracle
    w = oracle_sample_workload()
    o = oracle.Oracle(w.nx, w.ny, w.tau, openmp=openmp).init(*w.fields())
    o.step(warmup)
    steps, t0 = 0, time.perf_counter()
    while True:
        o.step(1)
        steps += 1
        el = time.perf_counter() - t0
        if (fixed_steps is not None and steps >= fixed_steps) or (fixed_steps is None and el >= seconds):
            break
    mlups = w.cells * steps / el / 1e6
    how = "OpenMP over rows, all host cores" if openmp else "one thread"
    sample = (f"FP64 C oracle ({how}) on the same pulse recipe at {w.nx}x{w.ny} "
              f"(4 pulses, tau 0.55), {steps} steps after {warmup} warm-up")
    return mlups, steps, el, sample


def run_reference(args, rank, world):
    if rank != 0:
        return
    w = workload(args.workload)
    mlups, steps, el, sample = time_oracle(0.0, warmup=args.warmup, fixed_steps=args.steps)
    cores = cpu_threads()
    line = {
        "impl": "reference", "metric": METRIC, "value": mlups, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": el / steps * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": describe(w, args.storage), "sample": f"{CPU_SAMPLE_N}x{CPU_SAMPLE_N}"},
        "cpu_baseline": {"value": mlups, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
        "e2e": {"value": mlups, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# --- GPU arm ------------------------------------------------------------------

def max_over_ranks(x: float, device: str) -> float:
    """Largest value of x over the ranks of the default process group (the
    whole job is as slow as its slowest rank)."""
    import torch
    import torch.distributed as td
    t = torch.tensor([float(x)], device=device, dtype=torch.float64)
    td.all_reduce(t, op=td.ReduceOp.MAX)
    return float(t.item())


def aggregate_mlups(cells_per_rank: int, steps: int, ms_max: float, world: int) -> float:
    """Whole-job MLUPS: every rank advanced its own replica of `cells_per_rank`
    nodes by `steps` steps; the job took the slowest rank's time."""
    return world * cells_per_rank * steps / (ms_max * 1e-3) / 1e6


def batch_what(count: int = 256) -> str:
    return (f"{count} instances 64..1024 per side, tau 0.51..0.8, pulses and vortices, "
            "one persistent launch per step replayed from a CUDA graph")


def shard(cells, rank: int, world: int, partition):
    """Indices of the instances this rank steps: a node-balanced split of the
    independent instances over the ranks (no data moves between ranks)."""
    if world == 1:
        return list(range(len(cells)))
    owner = partition(cells, world)
    return [k for k, r in enumerate(owner) if r == rank]


def run_batched(lbm, ws, bfields, storage, steps, warmup, world, peak, launch=None, rank=0, device="cuda"):
    """The batched workload: MLUPS over all instances, CUDA events on the
    stream.  With several ranks the instances are sharded (lbm_partition_
    instances) and the job time is the slowest rank's."""
    import torch
    all_ws = ws
    total_cells = sum(w.nx * w.ny for w in ws)
    mine = shard([w.nx * w.ny for w in ws], rank, world, lbm.lbm_partition_instances)
    ws, bfields = [ws[k] for k in mine], [bfields[k] for k in mine]
    bt = lbm.Batch(ws, storage=storage)
    for k, f in enumerate(bfields):
        bt.init(k, *f)
    if launch == "twostep":
        tb = tr = tg = tp = ts = tt = None
        bt.set_twostep(True)
    elif launch:
        tb, tr, tg, tp, ts, tt = (list(launch) + [0, 0])[:6]
        bt.set_launch(tb, tr, tg, tp, ts, tt)
    else:
        tb, tr, tg, tp, ts, tt, _ = bt.autotune()
    bt.step(warmup)
    torch.cuda.synchronize()
    a0 = torch.cuda.Event(enable_timing=True)
    a1 = torch.cuda.Event(enable_timing=True)
    a0.record(bt.stream)
    bt.step(steps)
    a1.record(bt.stream)
    torch.cuda.synchronize()
    bms = a0.elapsed_time(a1)
    bt.status()  # raises if a bounded device-side wait gave up
    bad = sum(bt.unstable_nodes(k) for k in range(len(ws)))
    gbs = BYTES_PER_CELL[storage] * bt.cells * steps / (bms * 1e-3) / 1e9
    ms_max = max_over_ranks(bms, device) if world > 1 else bms
    out = {"mlups": total_cells * steps / (ms_max * 1e-3) / 1e6, "steps": steps, "ms_per_step": ms_max / steps,
           "instances": len(ws), "cells": bt.cells, "step_gbs": gbs, "step_frac": gbs / peak,
           "sharding": (f"{world} ranks, instances split by nodes (lbm_partition_instances), no exchange; "
                        f"rank {rank} steps {len(ws)} instances, {bt.cells} nodes of {total_cells}")
           if world > 1 else "one rank, all instances",
           "launch": ({"twostep": True} if bt.twostep else
                      {"threads_x": tb, "rows": tr, "blocks": tg, "prefetch_rows": tp, "split": ts,
                       "tma_tile": tt}),
           "unstable_nodes": bad, "what": batch_what(len(all_ws))}
    bt.close()
    del bt
    torch.cuda.empty_cache()
    return out


def run_one_at_a_time(lbm, ws, bfields, storage, steps):
    """The same instances stepped one after another as single domains (graph
    replays, default launch shape): MLUPS over the summed device times."""
    import torch
    total_ms, cells = 0.0, 0
    for w, f in zip(ws, bfields):
        s = lbm.Simulation(w.nx, w.ny, w.tau, w.farfield_rho, w.farfield_u, storage=storage)
        s.init(*f)
        s.step(16)
        a0 = torch.cuda.Event(enable_timing=True)
        a1 = torch.cuda.Event(enable_timing=True)
        a0.record(s.stream)
        s.step(steps)
        a1.record(s.stream)
        torch.cuda.synchronize()
        total_ms += a0.elapsed_time(a1)
        cells += w.nx * w.ny
        s.close()
    torch.cuda.empty_cache()
    return {"mlups": cells * steps / (total_ms * 1e-3) / 1e6, "steps_each": steps,
            "what": "each instance alone as a single domain (CUDA graphs of 16 steps), device times summed"}


def run_batched_only(args, rank, world, local_rank):
    """--batched-only: the batched workload alone (for profiling runs)."""
    import torch
    from paper_2005_08674_gb300 import build
    build.build()
    from paper_2005_08674_gb300 import inputs, lbm
    torch.cuda.set_device(local_rank)
    ws = inputs.batch_instances(count=args.batch_count)
    bfields = [w.fields() for w in ws]
    peak, _ = measured_peak_gbs()
    launch = (args.batch_launch if args.batch_launch == "twostep" else
              [int(v) for v in args.batch_launch.split(",")] if args.batch_launch else None)
    r = run_batched(lbm, ws, bfields, args.storage, args.steps, args.warmup, world, peak, launch, rank)
    if rank == 0:
        print(json.dumps({"metric": METRIC, "value": r["mlups"], "unit": UNIT, "n_gpus": world,
                          "steps": args.steps, "warmup": args.warmup, "ms_per_step": r["ms_per_step"],
                          "higher_is_better": True, "scaling": "strong" if world > 1 else "weak",
                          "vs_baseline": None, "dtype": args.storage, "data": "synthetic",
                          "config": {"workload": "batched: " + batch_what(len(ws)),
                                     "parallelism": "instances sharded by nodes" if world > 1 else "single-gpu"},
                          "batched": r}), flush=True)


def run_ours(args, rank, world, local_rank):
    import numpy as np
    import torch
    from paper_2005_08674_gb300 import build
    build.build()
    from paper_2005_08674_gb300 import lbm

    torch.cuda.set_device(local_rank)
    dist = world > 1
    if dist:
        import torch.distributed as td

    w = workload(args.workload)
    cells = w.cells
    interior = (w.nx - 2) * (w.ny - 2)
    fields = w.fields()

    sim = lbm.Simulation(w.nx, w.ny, w.tau, w.farfield_rho, w.farfield_u, storage=args.storage)
    sim.init(*fields)
    if args.launch == "twostep":
        bx, rows, pf = 0, 0, 0
        sim.set_twostep(True)
    elif args.launch.startswith("staged"):
        bx, rows, pf = 0, 0, 0
        sim.set_staged(int(args.launch[len("staged"):] or 3))
    elif args.launch.startswith("fused"):
        parts = [int(v) for v in args.launch[len("fused"):].lstrip(":").split(",") if v] or [128, 1, 0]
        bx, rows, pf = (parts + [0, 0])[:3]
        sim.set_launch(bx, rows, pf)
        sim.set_fused(True)
    elif args.launch:
        parts = [int(v) for v in args.launch.split(",")]
        bx, rows, pf = (parts + [0])[:3]
        sim.set_launch(bx, rows, pf)
    else:
        bx, rows, pf, _ = sim.autotune()
    stream = sim.stream

    def barrier():
        torch.cuda.synchronize()
        if dist:
            td.barrier()
        torch.cuda.synchronize()

    # warm-up (also captures the step graphs)
    sim.step(args.warmup)
    barrier()

    clocks = ClockSampler(local_rank)
    clocks.start()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    barrier()
    e0.record(stream)
    sim.step(args.steps)
    e1.record(stream)
    barrier()
    ms = e0.elapsed_time(e1)
    clk = clocks.stop()
    ms_max = max_over_ranks(ms, "cuda") if dist else ms
    value = aggregate_mlups(cells, args.steps, ms_max, world)
    out = sim.reduce(allow_unstable=True)
    stable = out[3] == 0

    # kernel-timing region: same step, per-launch CUDA events on the launching stream
    kprof = min(args.steps, 400)
    lbm.lbm_profile(sim.h, True)
    sim.step(kprof)
    bulk_ms, nb, nsbc_ms, nn = lbm.lbm_profile_read(sim.h)
    lbm.lbm_profile(sim.h, False)
    bulk_avg = bulk_ms / max(nb, 1)
    nsbc_avg = nsbc_ms / max(nn, 1)
    peak, peak_kind = measured_peak_gbs()
    kname, kstem, kcells = step_kernel(sim, w.nx, w.ny)
    alg_bytes = BYTES_PER_CELL[args.storage] * kcells
    achieved = alg_bytes / (bulk_avg * 1e-3) / 1e9
    traffic = profiled_traffic(kstem, args.storage, kcells)

    line = None
    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": args.storage, "data": "synthetic",
            "config": {"workload": describe(w, args.storage), "nx": w.nx, "ny": w.ny,
                       "step_kernel": ({"twostep": True} if sim.twostep else
                                       {"staged_stages": sim.staged} if sim.staged else
                                       {"bulk_threads_x": bx, "bulk_rows": rows, "prefetch_rows": pf,
                                        "fused": sim.fused}),
                       "l2": f"inputs larger than L2: {lbm.lbm_buffer_bytes(sim.h) / 1e9:.2f} GB per population buffer",
                       "parallelism": "replicas" if world > 1 else "single-gpu",
                       "stable": bool(stable)},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": traffic,
                         "frac_of": "measured copy bandwidth (a torch copy: read + write bytes)",
                         # the same launch time against the DRAM bytes ncu counted for this kernel:
                         # what the memory system actually moved, beside the algorithmic rate
                         "dram_gbs": traffic / (bulk_avg * 1e-3) / 1e9 if traffic else None,
                         "dram_frac": traffic / (bulk_avg * 1e-3) / 1e9 / peak if traffic else None,
                         "kernel": kname,
                         "bytes_per_cell": BYTES_PER_CELL[args.storage], "cells_per_launch": kcells,
                         "steps_per_launch": 2 if sim.twostep else 1,
                         "avg_launch_ms": bulk_avg, "peak_source": f"{peak_kind} (MEASURED_PEAKS.json hbm_gbs)",
                         "nsbc_avg_launch_ms": nsbc_avg if nn else None,
                         "timing": f"per-launch CUDA events over {kprof} steps after the timed region"},
            "gpu_launches": (args.steps // 2 + 2 * (args.steps % 2) if sim.twostep else
                             (1 if sim.staged or sim.fused else 2) * args.steps),
            "clocks": clk,
        }

    # end to end through the C ABI with host buffers (pinned)
    if not args.no_e2e:
        pinned = [torch.empty((w.ny, w.nx), dtype=torch.float64, pin_memory=True) for _ in range(6)]
        for t, a in zip(pinned[:3], fields):
            t.numpy()[...] = a
        for t in pinned[3:]:
            t.numpy()[...] = 0.0  # the result buffers exist (and are touched) before the job, like the inputs
        host_in = [t.numpy() for t in pinned[:3]]
        host_out = [t.numpy() for t in pinned[3:]]
        barrier()
        t0 = time.perf_counter()
        lbm.lbm_init(sim.h, *host_in)
        lbm.lbm_step(sim.h, args.steps)
        lbm.lbm_get_macros(sim.h, *host_out)
        t1 = time.perf_counter()
        barrier()
        e2e_s = t1 - t0
        if dist:
            e2e_s = max_over_ranks(e2e_s, "cuda")
        if line is not None:
            nbytes = 3 * cells * 8
            line["e2e"] = {"value": world * cells * args.steps / e2e_s / 1e6, "unit": UNIT,
                           "h2d_bytes_per_step": nbytes / args.steps, "d2h_bytes_per_step": nbytes / args.steps,
                           "what": "lbm_init (host fields) + lbm_step(steps) + lbm_get_macros (host), wall clock",
                           "seconds": e2e_s}
        del pinned, host_in, host_out
    sim.close()
    del sim
    torch.cuda.empty_cache()

    # other storage types on the same workload
    if not args.no_variants:
        variants = {}
        vsteps = min(args.steps, 1000)
        for st in ("f32", "f16", "bf16", "f64"):
            if st == args.storage:
                continue
            s2 = lbm.Simulation(w.nx, w.ny, w.tau, w.farfield_rho, w.farfield_u, storage=st)
            s2.init(*fields)
            vb, vr, vp, _ = s2.autotune()
            s2.step(args.warmup)
            torch.cuda.synchronize()
            a0 = torch.cuda.Event(enable_timing=True)
            a1 = torch.cuda.Event(enable_timing=True)
            a0.record(s2.stream)
            s2.step(vsteps)
            a1.record(s2.stream)
            torch.cuda.synchronize()
            vms = a0.elapsed_time(a1)
            lbm.lbm_profile(s2.h, True)
            s2.step(min(vsteps, 200))
            bms, bn, _, _ = lbm.lbm_profile_read(s2.h)
            bavg = bms / max(bn, 1)
            vname, _, vcells = step_kernel(s2, w.nx, w.ny)
            gbs = BYTES_PER_CELL[st] * vcells / (bavg * 1e-3) / 1e9
            variants[st] = {"mlups": world * cells * vsteps / (vms * 1e-3) / 1e6, "steps": vsteps,
                            "kernel_gbs": gbs, "kernel_frac": gbs / peak, "kernel": vname,
                            "bulk_launch": None if (s2.staged or s2.twostep) else [vb, vr, vp]}
            s2.close()
            del s2
            torch.cuda.empty_cache()
        # the convected-vortex and small-pulse workloads at their own sizes
        # (their populations fit in the 129 MB L2, so these are not HBM rates)
        from paper_2005_08674_gb300 import inputs as _inp
        for label, wl, st, kw in (
                ("vortex-400_mrt_f32", _inp.vortex_400(), "f32",
                 dict(collision="mrt", mrt_rates=(1.4, 1.4, 1.2))),
                ("pulse-200_f64", _inp.pulse_200(), "f64", {})):
            s3 = lbm.Simulation(wl.nx, wl.ny, wl.tau, wl.farfield_rho, wl.farfield_u, storage=st, **kw)
            s3.init(*wl.fields())
            s3.autotune()
            s3.step(args.warmup)
            torch.cuda.synchronize()
            a0 = torch.cuda.Event(enable_timing=True)
            a1 = torch.cuda.Event(enable_timing=True)
            a0.record(s3.stream)
            s3.step(wl.steps)
            a1.record(s3.stream)
            torch.cuda.synchronize()
            vms = a0.elapsed_time(a1)
            variants[label] = {"mlups": world * wl.cells * wl.steps / (vms * 1e-3) / 1e6, "steps": wl.steps,
                               "cells": wl.cells, "storage": st,
                               "note": f"{lbm.lbm_buffer_bytes(s3.h) / 1e6:.1f} MB per buffer: L2-resident"}
            s3.close()
            del s3
        # the same pulse recipe at smaller sizes (f32, autotuned): where the
        # populations start to fit in L2 and launch gaps start to count
        sizes = {}
        for n in (1024, 2048, 4096):
            wn = workload(f"pulse-{n}")
            s4 = lbm.Simulation(wn.nx, wn.ny, wn.tau, wn.farfield_rho, wn.farfield_u, storage="f32")
            s4.init(*wn.fields())
            s4.autotune()
            s4.step(args.warmup)
            nsteps = min(args.steps, 400)
            torch.cuda.synchronize()
            a0 = torch.cuda.Event(enable_timing=True)
            a1 = torch.cuda.Event(enable_timing=True)
            a0.record(s4.stream)
            s4.step(nsteps)
            a1.record(s4.stream)
            torch.cuda.synchronize()
            vms = a0.elapsed_time(a1)
            mlups = world * wn.cells * nsteps / (vms * 1e-3) / 1e6
            sizes[f"pulse-{n}"] = {"mlups": mlups, "steps": nsteps, "frac_of_72B_roofline": mlups * 1e6 * 72 / 1e9 / peak,
                                   "step_kernel": ("twostep" if s4.twostep else f"staged {s4.staged}" if s4.staged
                                                   else "fused" if s4.fused else "bulk + NSBC pair"),
                                   "mb_per_buffer": lbm.lbm_buffer_bytes(s4.h) / 1e6}
            s4.close()
            del s4
            torch.cuda.empty_cache()
        variants["sizes_f32"] = sizes
        # batched: 256 independent instances, one persistent launch per step
        from paper_2005_08674_gb300 import inputs
        ws = inputs.batch_instances()
        bfields = [w.fields() for w in ws]
        bsteps = min(args.steps, 1000)
        for st in ("f32", "f16"):
            variants[f"batched_{st}"] = run_batched(lbm, ws, bfields, st, bsteps, args.warmup, world, peak,
                                                    rank=rank)
            one = run_one_at_a_time(lbm, ws, bfields, st, 64)
            one["batched_speedup"] = variants[f"batched_{st}"]["mlups"] / world / one["mlups"]  # per GPU
            variants[f"batched_{st}"]["one_at_a_time"] = one
        del bfields
        if line is not None:
            line["variants"] = variants

    if line is not None and not args.no_cpu:
        mlups, steps, el, sample = time_oracle(args.cpu_seconds)
        line["cpu_baseline"] = {"value": mlups, "unit": UNIT, "cores": cpu_threads(), "kind": "oracle",
                                "sample": sample, "seconds": el}
        m1, _, el1, sample1 = time_oracle(args.cpu_seconds / 3, openmp=False)
        line["cpu_baseline"]["single_thread"] = {"value": m1, "unit": UNIT, "cores": 1, "sample": sample1,
                                                 "seconds": el1}
    return line


def main():
    args = parse()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    if world > 1:
        import torch
        import torch.distributed as td
        torch.cuda.set_device(local_rank)
        td.init_process_group("nccl")
    if args.batched_only:
        run_batched_only(args, rank, world, local_rank)
        line = None
    else:
        line = run_ours(args, rank, world, local_rank)
    if line is not None:
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as td
        td.destroy_process_group()


if __name__ == "__main__":
    main()
