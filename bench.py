#!/usr/bin/env python3
"""Throughput of the SoA particle hot path on B300, one JSON line on stdout.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl soax|reference] [--no-rows]

Workload (one "step" of this benchmark): the 16,777,216-particle set {i32 id, f64 pos[3],
f32 vel[3]} in the ABC flow (A = B = C = 1, tau = 0.1, dt = 1e-3); one bench step is one
sort interval: 10 midpoint-RK2 steps and a cell sort on the 32^3 grid.  The steps run in
one pass over the planes (soax_permute_step_fused: each particle gathered once through
the permutation the previous sort computed, advanced 10 steps in registers, stored in
sorted order with its new cell key), then the stable radix sort of the keys gives the
next permutation (soax_sort_perm); so every bench step does the steps, the keys, the
radix sort and the permute-gather of every plane, with the gather riding on the next
step's pass.  K bench steps = 10 K RK2 steps; the default K = 100 is the full 1000-step
run.

Metric: particle-steps/s (whole job, all ranks).  The dominant kernel is the fused step;
with the planes moved once per 10 steps it is bound by instruction issue, not by HBM.  Its
roofline is the issue rate, one warp-instruction per clock per SM sub-partition (4 per SM,
148 SMs, 32 lanes, 2032 MHz: 38.5 T thread-instructions/s), against the instructions per
particle-step that ncu counts for the current sources (profiles/ncu_traffic.json).  The
one-pass-per-step kernel (soax_step, 72 algorithmic bytes per particle-step against the
measured copy bandwidth in MEASURED_PEAKS.json) is timed as a secondary row.

Also measured in the same run ("rows"): the AoS <-> SoA round trip and the AoS step on the
same set, the sort's share, the forward+adjoint of the 1M-particle K = 1000 problem against
the plain step, and the batched persistent launch over 512 uneven ensembles against 512
separate plain launches per step (a few steps each, reported per particle-step).

--impl reference times the CPU oracle on the host cores on a bounded sample of the same
workload (the only other place that runs oracle/ besides the cpu_baseline leg).

Multi-GPU (torchrun): every rank advances its own replica of the workload (weak scaling,
no collective on the data path); time = max over ranks; value = all ranks' particle-steps
/ that time.
"""
import argparse
import ctypes
import hashlib
import glob
import json
import os
import re
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import soax_inputs  # noqa: E402

WL = soax_inputs.WORKLOADS["sorted_n16M"]
RK2_PER_STEP = WL["sort_every"]
BYTES_PER_PARTICLE_STEP = 72  # pos 3 x f64 + vel 3 x f32, read and written
METRIC = "particle-steps/s"
L2_BYTES = 126 * 2 ** 20
# Issue-rate peak of B300: 1 warp-instruction per clock per SM sub-partition, 4 per SM,
# 148 SMs, 32 lanes, at the 2032 MHz maximum SM clock (thread-instructions per second).
SMSP_PER_SM = 4
MAX_SM_MHZ = 2032.0
# The bench step's dominant kernel: 10 steps with the previous sort's permute-gather and
# the new cell keys in one pass.  Its algorithmic bytes per particle per launch: perm 4,
# gathered record 40 (id, pos, vel), written record 40, key 4.
STEP_KERNEL = "k_step_soa_fused_gather"
STEP_LAUNCH_BYTES = 88


def parse_args(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="soax", choices=["soax", "reference"])
    ap.add_argument("--no-rows", action="store_true", help="skip the secondary rows")
    ap.add_argument("--only", choices=["euler", "euler_sweep", "adjoint", "batched", "aos", "fixed", "plain", "wide",
                                       "sort"],
                    help="run only this secondary row (profiling captures)")
    ap.add_argument("--n", type=int, default=None, help="particles (default: the row's workload)")
    ap.add_argument("--e2e-chunks", type=int, default=16, help="pieces per soax_step_host call in the e2e loop")
    ap.add_argument("--e2e-no-defer", action="store_true",
                    help="e2e: each call downloads its own result (no interleaving with the next call's uploads)")
    ap.add_argument("--nens", type=int, default=None, help="--only batched: the first NENS ensembles")
    ap.add_argument("--fixed-tune", action="store_true", help="--only batched: a fixed launch shape, no autotuning")
    ap.add_argument("--intervals", type=int, default=None, help="--only wide: sort intervals to time")
    ap.add_argument("--sizes", type=int, nargs="*", default=None, help="--only euler: AoS_SIZE record sizes")
    ap.add_argument("--nsteps", type=int, nargs="*", default=None,
                    help="--only fixed: steps per launch (default 10 and 20)")
    return ap.parse_args(argv)


def dist_env():
    return int(os.environ.get("RANK", "0")), int(os.environ.get("LOCAL_RANK", "0")), int(os.environ.get("WORLD_SIZE", "1"))


def aggregate(local_units, local_seconds, device=None):
    """(sum of units over ranks, max of seconds over ranks); works for any backend."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(local_units), float(local_seconds)
    u = torch.tensor([float(local_units)], dtype=torch.float64, device=device)
    s = torch.tensor([float(local_seconds)], dtype=torch.float64, device=device)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    dist.all_reduce(s, op=dist.ReduceOp.MAX)
    return float(u.item()), float(s.item())


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as fh:
            j = json.load(fh)
        return float(j["hbm_gbs"]), "measured"
    except (OSError, ValueError, KeyError):
        return 6400.0, "fallback"


CSRC = os.path.join(ROOT, "paper_1710_03462_b300", "csrc")


def unit_sources(unit):
    """The files a kernel's code comes from: its translation unit under csrc/, every
    local header it includes (transitively), and the build script (compiler flags)."""
    seen, todo = [], [os.path.join(CSRC, unit)]
    while todo:
        f = os.path.normpath(todo.pop())
        if f in seen:
            continue
        seen.append(f)
        with open(f) as fh:
            for line in fh:
                line = line.strip()
                if line.startswith("#include \""):
                    todo.append(os.path.join(os.path.dirname(f), line.split('"')[1]))
    return sorted(seen) + [os.path.join(ROOT, "paper_1710_03462_b300", "build.py")]


def code_only(text):
    """A source without its comments and blank lines: what the compiler sees (the
    counters of a kernel depend on its code, not on the words around it)."""
    text = re.sub(r"/\*.*?\*/", " ", text, flags=re.S)
    lines = []
    for line in text.splitlines():
        if line.lstrip().startswith("#") and not line.lstrip().startswith(("#include", "#define", "#pragma", "#if",
                                                                            "#else", "#endif", "#ifdef", "#ifndef")):
            line = ""  # a Python comment line (the build script)
        line = re.sub(r"//.*$", "", line).rstrip()
        if line:
            lines.append(line)
    return "\n".join(lines)


def source_hash(unit):
    """Hash of the code (comments dropped) of a kernel's translation unit, its headers and
    the build script."""
    h = hashlib.sha1()
    for f in unit_sources(unit):
        with open(f, encoding="utf-8", errors="replace") as fh:
            h.update(code_only(fh.read()).encode())
    return h.hexdigest()[:16]


def ncu_record(kernel):
    """The committed ncu figures of kernel (profiles/ncu_traffic.json) if they were taken
    on the current sources of its translation unit; else None."""
    path = os.path.join(ROOT, "profiles", "ncu_traffic.json")
    try:
        with open(path) as fh:
            j = json.load(fh)
        e = j.get(kernel)
        if e and e.get("source_hash") == source_hash(e["unit"]):
            return e
    except (OSError, ValueError, KeyError, TypeError):
        pass
    return None


def ncu_traffic(kernel):
    """DRAM bytes per full-size launch of kernel from the committed ncu record, or None."""
    e = ncu_record(kernel)
    try:
        return float(e["dram_bytes_per_launch_full_size"]) if e else None
    except (KeyError, TypeError, ValueError):
        return None


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 50 ms during the timed region
    (the sampler's first line is awaited, and dropped, before the region starts)."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits", "-lms", "50",
                 "-i", str(self.gpu)], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.proc.stdout.readline()  # sampling is live (or nvidia-smi has exited)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *a):
        self.out = ""
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                self.out, _ = self.proc.communicate()

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in (self.out or "").splitlines():
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[1]))
                mx = float(parts[2])
            except ValueError:
                continue
            for nm, v in zip(names, parts[4:8]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


# ---------------------------------------------------------------------------- oracle timing
def oracle_interval(oracle, st, wl, threads, aos=False):
    """One sort interval of the oracle on the sample st (in place): sort_every RK2 steps,
    the cell keys, the stable argsort and the permute of every plane.  st holds "planes"
    (id, pos[3], vel[3], and for the wide record acc[3], mass, tag) or, with aos, "rec"
    (the natural AoS records) plus the layout to step them."""
    steps = wl["sort_every"]
    tau_scale = wl.get("tau_scale", 0.0)
    if aos:
        L = st["layout"]
        oracle.step_aos(st["rec"], L["rb"], L["pos"], L["vel"], wl["A"], wl["B"], wl["C"], wl.get("tau", 0.0),
                        wl["dt"], steps, acc_off=L.get("acc", -1), mass_off=L.get("mass", -1), tau_scale=tau_scale,
                        threads=threads)
        return
    pl = st["planes"]
    pos, vel = pl["pos"], pl["vel"]
    oracle.step_soa(pos, vel, wl["A"], wl["B"], wl["C"], wl.get("tau", 0.0), wl["dt"], steps, acc=pl.get("acc"),
                    mass=pl["mass"][0] if "mass" in pl else None, tau_scale=tau_scale, threads=threads)
    keys = oracle.cell_keys(*pos, wl["grid"])
    perm, _ = oracle.stable_argsort(keys)
    names = list(pl)
    flat = [a for k in names for a in pl[k]]
    out = oracle.permute(flat, perm)
    k = 0
    for name in names:
        m = len(pl[name])
        pl[name] = out[k:k + m]
        k += m


def oracle_sample(name, ns, aos=False):
    """The first ns particles of a workload's set (seeded as the GPU run's), as oracle
    planes or as AoS records."""
    wl = soax_inputs.WORKLOADS[name]
    d = soax_inputs.wide_set(ns, wl["seed"]) if name == "wide_n64M" else soax_inputs.basic_set(ns, wl["seed"])
    planes = {k: [a.copy() for a in v] for k, v in d.items()}
    if not aos:
        return {"planes": planes}
    import oracle
    eb = {"i32": 4, "i64": 8, "u8": 1, "f32": 4, "f64": 8}
    schema = WIDE_FIELDS if name == "wide_n64M" else BASIC_FIELDS
    rb, offs = oracle.aos_layout([eb[t] for _, t, _ in schema], [c for _, _, c in schema])
    rec = oracle.soa_to_aos([a for f, _, _ in schema for a in planes[f]], [eb[t] for _, t, _ in schema],
                            [c for _, _, c in schema])
    layout = {"rb": rb}
    for (f, _, _), o in zip(schema, offs):
        layout[f] = o
    return {"rec": rec, "layout": layout}


BASIC_FIELDS = [("id", "i32", 1), ("pos", "f64", 3), ("vel", "f32", 3)]
WIDE_FIELDS = [("id", "i64", 1), ("pos", "f64", 3), ("vel", "f32", 3), ("acc", "f32", 3), ("mass", "f32", 1),
               ("tag", "u8", 1)]


def time_oracle(name, ns, threads, reps=1, warmup=1, aos=False, sort=True):
    """Seconds per sort interval of the oracle (mean of reps after warmup untimed ones)
    on ns particles of the workload with `threads` threads; the sample is drawn before
    and the warm-up runs on it, so neither page faults on fresh arrays nor thread start-up
    land in the timed region."""
    import oracle
    wl = dict(soax_inputs.WORKLOADS[name])
    wl.setdefault("sort_every", wl.get("steps"))
    st = oracle_sample(name, ns, aos=aos)
    if not sort:
        wl["grid"] = None

    def one():
        if sort:
            oracle_interval(oracle, st, wl, threads, aos=aos)
        elif aos:
            oracle_interval(oracle, st, wl, threads, aos=True)
        else:
            pl = st["planes"]
            oracle.step_soa(pl["pos"], pl["vel"], wl["A"], wl["B"], wl["C"], wl.get("tau", 0.0), wl["dt"],
                            wl["sort_every"], acc=pl.get("acc"), mass=pl["mass"][0] if "mass" in pl else None,
                            tau_scale=wl.get("tau_scale", 0.0), threads=threads)
    for _ in range(warmup):
        one()
    t0 = time.perf_counter()
    for _ in range(reps):
        one()
    return (time.perf_counter() - t0) / reps


def oracle_baseline(name, n, reps=1, warmup=1, single_core=True, aos=True, sort=True):
    """The oracle timed on the host cores on a bounded sample of a workload: all cores
    (the reported value: SoA planes, RK2 steps of one sort interval plus its cell sort),
    one core on a smaller sample, and the AoS records on all cores (steps only: the AoS
    form has no sort here).  Returns the cpu_baseline object."""
    cores = os.cpu_count() or 1
    wl = soax_inputs.WORKLOADS[name]
    steps = wl.get("sort_every", wl.get("steps"))
    ns = min(n, 1 << 22)
    el = time_oracle(name, ns, cores, reps=reps, warmup=warmup, sort=sort)
    out = {"value": ns * steps / el, "unit": "particle-steps/s", "cores": cores, "kind": "oracle",
           "sample": f"{ns} of {n} particles x {steps} RK2 steps" + (" + one cell sort" if sort else "") +
                     f" per timed interval, {reps} timed after {warmup} warm-up, SoA planes, {cores} threads "
                     f"({el:.2f} s per interval)"}
    if single_core:
        n1 = max(1024, ns // max(cores, 1))
        e1 = time_oracle(name, n1, 1, reps=1, warmup=1, sort=sort)
        out["single_core"] = {"value": n1 * steps / e1, "unit": "particle-steps/s", "cores": 1,
                              "sample": f"{n1} particles, same interval, 1 thread ({e1:.2f} s)"}
    if aos:
        ea = time_oracle(name, ns, cores, reps=1, warmup=1, aos=True, sort=False)
        out["aos"] = {"value": ns * steps / ea, "unit": "particle-steps/s", "cores": cores,
                      "sample": f"{ns} AoS records x {steps} RK2 steps, {cores} threads ({ea:.2f} s)"}
        es = time_oracle(name, ns, cores, reps=1, warmup=1, sort=False)
        out["soa_steps_only"] = {"value": ns * steps / es, "unit": "particle-steps/s", "cores": cores,
                                 "sample": f"{ns} particles x {steps} RK2 steps, no sort ({es:.2f} s)"}
    return out


# ---------------------------------------------------------------------------- reference arm
def run_reference(args):
    """The CPU oracle as the reference arm: each bench step is a bounded sample of the
    workload (a quarter of the particles: 10 RK2 steps + the cell sort of that sample),
    timed by the same procedure as the GPU arm's cpu_baseline (oracle_baseline)."""
    rank, _, world = dist_env()
    if rank != 0:
        return 0
    steps = max(1, min(args.steps, 5))
    warm = max(1, min(args.warmup, 2))
    base = oracle_baseline("sorted_n16M", args.n, reps=steps, warmup=warm)
    value = base["value"]
    ms = WL["sort_every"] * min(args.n, 1 << 22) / value * 1e3
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "particle-steps/s", "n_gpus": args.gpus,
            "steps": steps, "warmup": warm, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "sorted_n16M", "n": args.n, "grid": WL["grid"], "sort_every": RK2_PER_STEP},
            "cpu_baseline": base,
            "e2e": {"value": value, "unit": "particle-steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


def cpu_baseline(n):
    """The oracle on the host cores (oracle_baseline on the bench workload)."""
    return oracle_baseline("sorted_n16M", n)


# ---------------------------------------------------------------------------- GPU arm
def run_soax(args):
    import torch
    import torch.distributed as dist
    import paper_1710_03462_b300 as sx

    rank, local, world = dist_env()
    if world > 1:
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    dev = torch.device("cuda", local if world > 1 else torch.cuda.current_device())
    torch.cuda.set_device(dev)
    n = args.n
    flow = sx.Flow(A=WL["A"], B=WL["B"], C=WL["C"], tau=WL["tau"], dt=WL["dt"])
    d = soax_inputs.basic_set(n, WL["seed"] + rank)
    p = sx.Particles(sx.BASIC_SCHEMA, n, device=dev)
    p.load(d)
    ws = p.sort_workspace(WL["grid"])
    stream = torch.cuda.current_stream(dev)

    keys = torch.empty(n, dtype=torch.int32, device=dev)
    pending = {"perm": None}  # the permutation the last sort left, gathered by the next step

    def bench_step(ev=None):
        if ev is not None:
            ev[0].record(stream)
        p.step_fused(flow, RK2_PER_STEP, grid=WL["grid"], keys=keys, perm=pending["perm"])
        if ev is not None:
            ev[1].record(stream)
        pending["perm"] = p.sort_perm(WL["grid"], keys, ws)[1]
        if ev is not None:
            ev[2].record(stream)

    for _ in range(args.warmup):
        bench_step()
    torch.cuda.synchronize(dev)
    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(args.steps)]
    start, stop = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize(dev)
    with ClockSampler(dev.index) as clk:
        start.record(stream)
        for s in range(args.steps):
            bench_step(evs[s])
        stop.record(stream)
        torch.cuda.synchronize(dev)
    if world > 1:
        dist.barrier()
    elapsed = start.elapsed_time(stop) / 1e3
    fused_ms = [evs[s][0].elapsed_time(evs[s][1]) for s in range(args.steps)]
    sort_ms = [evs[s][1].elapsed_time(evs[s][2]) for s in range(args.steps)]
    units = n * RK2_PER_STEP * args.steps
    tot_units, max_el = aggregate(units, elapsed, dev)

    # e2e through the C ABI with host buffers: the state lives in pinned host memory and
    # every bench step is one soax_step_host call, which uploads it, steps it, sorts it
    # and downloads it in pieces (uploads overlap the steps of the pieces already up;
    # downloads overlap the next call's uploads).  Calls are queued back to back: the
    # library orders each piece's upload after the previous call's download of it.
    host = {k: [torch.from_numpy(a).pin_memory() for a in v] for k, v in d.items()}
    e2e_steps = max(1, min(args.steps, 20))  # the run's first upload and last download amortised over 20 steps
    h2d = sum(t.numel() * t.element_size() for v in host.values() for t in v)
    planes = [(k, c) for k, v in host.items() for c in range(len(v))]
    s_up, s_dn = torch.cuda.Stream(dev), torch.cuda.Stream(dev)
    e2e_ws = p.sort_workspace(WL["grid"])
    p.step_host(host, flow, 0, WL["grid"], nchunks=args.e2e_chunks, ws=e2e_ws, stream=stream, up_stream=s_up,
                down_stream=s_dn)  # creates the call's events outside the timed region
    torch.cuda.synchronize(dev)
    for k, c in planes:  # the host home holds the set the device run started from
        host[k][c].copy_(torch.from_numpy(d[k][c]))
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        p.step_host(host, flow, RK2_PER_STEP, WL["grid"], nchunks=args.e2e_chunks, ws=e2e_ws, stream=stream,
                    up_stream=s_up, down_stream=s_dn, defer=not args.e2e_no_defer)
    p.step_host_finish(down_stream=s_dn)  # the last interval's downloads
    torch.cuda.synchronize(dev)
    e2e_el = time.perf_counter() - t0
    e2e_units, e2e_max = aggregate(n * RK2_PER_STEP * e2e_steps, e2e_el, dev)
    link = host_link(torch, dev, host, p, planes, s_up, s_dn)

    rows = {} if args.no_rows else secondary_rows(sx, torch, p, d, dev)
    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return 0
    fused_s = statistics.mean(fused_ms) / 1e3
    roofline = alu_roofline(torch, dev, STEP_KERNEL, n * RK2_PER_STEP, fused_s)
    roofline["hbm_GB/s"] = STEP_LAUNCH_BYTES * n / fused_s / 1e9
    # Algorithmic fractions beside the issue rate: the plain step's 72 B per particle-step
    # at this speed against the copy peak, and the FP32 work against the FP32 pipes.
    roofline["hbm_equivalent"] = hbm_equivalent(BYTES_PER_PARTICLE_STEP, n * RK2_PER_STEP, fused_s)
    roofline["fp32"] = fp32_fraction(torch, dev, STEP_KERNEL, n * RK2_PER_STEP, fused_s)
    sort_launches = sort_kernel_launches(WL["grid"])  # keys and permute-gather ride on the step
    line = {
        "metric": METRIC, "value": tot_units / max_el, "unit": "particle-steps/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": max_el / args.steps * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        # The step computes in FP32 float pairs (binary64-accurate) with positions as
        # 64-bit fixed-point turns; f64 is only the positions' storage type.
        "dtype": "f32 float-float + u64 fixed-point", "data": "synthetic",
        "config": {"workload": "sorted_n16M", "n": n, "fields": "i32 id, f64 pos[3], f32 vel[3]",
                   "rk2_steps_per_step": RK2_PER_STEP, "grid": WL["grid"], "flow": "ABC A=B=C=1 tau=0.1 dt=1e-3",
                   "parallelism": f"replicas x{world}",
                   "l2": f"inputs larger than L2 ({n * 40 / 2**20:.0f} MiB of planes > 126 MiB)"},
        "roofline": roofline,
        "sort_ms": statistics.mean(sort_ms),
        "e2e": {"value": e2e_units / e2e_max, "unit": "particle-steps/s", "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": h2d, "steps": e2e_steps,
                "copies": f"soax_step_host, {args.e2e_chunks} pieces per call: piece uploads overlap the "
                          "steps of the pieces already up; " + ("each call's downloads overlap the next call's uploads"
                          if args.e2e_no_defer else "each call's downloads are interleaved with the next call's "
                          "uploads piece by piece (defer), the last call's by soax_step_host_finish"),
                "link": link,
                "floor": e2e_floor(n * RK2_PER_STEP, e2e_steps, statistics.mean(sort_ms) / 1e3, h2d, link)},
        "gpu_launches": args.steps * (1 + sort_launches),
        "clocks": clk.summary(),
        "cpu_baseline": cpu_baseline(n) if world == 1 or rank == 0 else None,
        "rows": rows,
    }
    print(json.dumps(line))
    if world > 1:
        dist.destroy_process_group()
    return 0


def sort_kernel_launches(grid):
    """Kernels one soax_sort_perm launches on a grid^3 grid: for up to 18 key bits the
    cell counting sort's graph, six kernels (probe, count, chunk totals, scan, scatter,
    order) and the one that opens its conditional node (the radix passes in its body run
    only for keys the counting sort cannot take); beyond, the radix passes' three kernels
    each (upsweep, scan, downsweep)."""
    bits = max(1, int(grid ** 3 - 1).bit_length())
    passes = (bits + 8) // 9
    return 7 if bits <= 18 else 3 * passes


def e2e_floor(units_per_step, steps, gap_seconds, state_bytes, link):
    """The best e2e rate (units/s) the host link allows for `steps` sort intervals that
    each move state_bytes up and back: the first upload and the last download overlap
    nothing, the k - 1 round trips between them move at most at the two directions'
    combined rate, and in every interval the link waits gap_seconds of device work that
    needs all of the upload and precedes all of the download (the sort: every key before
    it, every sorted particle after it)."""
    both = 2 * state_bytes / (link["both_GB/s"] * 1e9)
    total = (steps * gap_seconds + (steps - 1) * both + state_bytes / (link["h2d_GB/s"] * 1e9)
             + state_bytes / (link["d2h_GB/s"] * 1e9))
    return units_per_step * steps / total


def host_link(torch, dev, host, p, planes, s_up, s_dn):
    """The host link's rates for the e2e state (pinned memory, one soax_copy_plane per plane): all
    planes up alone, down alone, and both directions at once (GB/s, total bytes moved).
    The e2e loop overlaps one call's downloads with the next call's uploads, so "both"
    uploads the planes while downloading the same number of bytes from a separate device
    buffer into a separate pinned buffer."""
    nbytes = sum(t.numel() * t.element_size() for v in host.values() for t in v)
    dev_scratch = torch.empty(nbytes, dtype=torch.uint8, device=dev)
    host_scratch = torch.empty(nbytes, dtype=torch.uint8).pin_memory()

    def up():
        for k, c in planes:
            p.copy_plane(k, c, host[k][c], True, stream=s_up)

    def down():
        for k, c in planes:
            p.copy_plane(k, c, host[k][c], False, stream=s_dn)

    def down_scratch():
        with torch.cuda.stream(s_dn):
            host_scratch.copy_(dev_scratch, non_blocking=True)

    out = {}
    for name, fn, moved in (("h2d_GB/s", up, nbytes), ("d2h_GB/s", down, nbytes),
                            ("both_GB/s", lambda: (up(), down_scratch()), 2 * nbytes)):
        fn()
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        for _ in range(3):
            fn()
        torch.cuda.synchronize(dev)
        out[name] = moved * 3 / (time.perf_counter() - t0) / 1e9
    # Each direction's own rate while both run, started together (CUDA events on the two
    # copy streams): the e2e pipeline waits on the slower one, piece by piece.
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
    torch.cuda.synchronize(dev)
    ev[0].record(s_up)
    s_dn.wait_event(ev[0])
    up()
    down_scratch()
    ev[1].record(s_up)
    ev[2].record(s_dn)
    torch.cuda.synchronize(dev)
    out["both_h2d_GB/s"] = nbytes / (ev[0].elapsed_time(ev[1]) / 1e3) / 1e9
    out["both_d2h_GB/s"] = nbytes / (ev[0].elapsed_time(ev[2]) / 1e3) / 1e9
    return out


def _time(torch, fn, reps=1):
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    fn()
    torch.cuda.synchronize()
    e0.record()
    for _ in range(reps):
        fn()
    e1.record()
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / 1e3 / reps


def euler_replica(sx, torch, n, dev, sizes=(0, 32)):
    """The paper's experiment on B300 (Sec. 2-3): Eq. 1 in single precision on SoA planes
    (fused; and one launch per component, as the paper's GPU code) and on Listing 4's
    AoS_SIZE records; time per particle and the AoS/SoA ratios the paper reports."""
    rng = np.random.default_rng(1)
    out = {"n": n, "algorithmic_bytes_per_particle": 36}
    q = sx.Particles([("x", "f32", 3, "P"), ("v", "f32", 3, "V")], n, device=dev, shadow=False)
    for name in ("x", "v"):
        for t in q.field(name):
            t.normal_()
    t_fused = _time(torch, lambda: q.euler(1e-3), reps=10)
    t_comp = _time(torch, lambda: q.euler(1e-3, per_component=True), reps=10)
    out["soa_fused_ns_per_particle"] = t_fused / n * 1e9
    out["soa_fused_GB/s"] = 36 * n / t_fused / 1e9
    out["roofline"] = hbm_roofline(36, n, t_fused)
    out["soa_per_component_ns_per_particle"] = t_comp / n * 1e9
    del q
    for size in sizes:
        rb = 24 + 4 * size
        rec = torch.empty(n * rb // 4, dtype=torch.float32, device=dev).normal_()
        t_aos = _time(torch, lambda: sx.euler_aos(rec, n, rb, 0, 12, 1e-3), reps=10)
        out[f"aos{size}_ns_per_particle"] = t_aos / n * 1e9
        out[f"aos{size}_over_soa_per_component"] = t_aos / t_comp
        del rec
    torch.cuda.empty_cache()
    return out


def euler_sweep(sx, torch, dev, ns=None, sizes=(0, 1, 2, 4, 8, 16, 32), max_bytes=48 << 30):
    """The paper's GPU experiment (Sec. 3.2, Figs. of the M2050 benchmark) on B300: the
    single-precision Euler step x += dt*v (Eq. 1) for N from 1e2 to 1e9 particles, on SoA
    planes (one fused launch over all components, and the paper's three launches, one per
    component) and on Listing 4's AoS_SIZE records for SIZE in sizes (24 + 4 SIZE bytes;
    sizes whose buffer would exceed max_bytes are skipped at that N).  Each form is timed
    per step with CUDA events over a CUDA graph of many steps (kernel time, as the paper
    measured with the profiler), in ns per particle; the ratios AoS_SIZE / SoA (the
    paper's three-launch SoA) and the smallest N from which SoA is ahead of AoS_0."""
    ns = ns or [100, 300, 1000, 2000, 5000, 10000, 100000, 1000000, 10000000, 100000000, 1000000000]
    stream = torch.cuda.current_stream(dev)
    rows = []
    for n in ns:
        reps = max(2, min(200, int(2e8 // max(n, 1))))
        row = {"n": n, "steps_per_graph": reps}
        q = sx.Particles([("x", "f32", 3, "P"), ("v", "f32", 3, "V")], n, device=dev, shadow=False)
        for name in ("x", "v"):
            for t in q.field(name):
                t.normal_()
        for key, fn in (("soa_fused", lambda s: q.euler(1e-3, stream=s)),
                        ("soa_per_component", lambda s: q.euler(1e-3, per_component=True, stream=s))):
            g = _graph(torch, dev, lambda s: [fn(s) for _ in range(reps)])
            row[key + "_ns"] = _events(torch, stream, g.replay, reps=3) / reps / n * 1e9
            del g
        del q
        for size in sizes:
            rb = 24 + 4 * size
            if n * rb > max_bytes:
                continue
            rec = torch.empty(n * rb // 4, dtype=torch.float32, device=dev).normal_()
            g = _graph(torch, dev, lambda s: [sx.euler_aos(rec, n, rb, 0, 12, 1e-3, stream=s) for _ in range(reps)])
            row[f"aos{size}_ns"] = _events(torch, stream, g.replay, reps=3) / reps / n * 1e9
            row[f"aos{size}_over_soa"] = row[f"aos{size}_ns"] / row["soa_per_component_ns"]
            del g, rec
        row["soa_fused_GB/s"] = 36 / row["soa_fused_ns"]
        rows.append(row)
        torch.cuda.empty_cache()
    cross = next((r["n"] for r in rows if r.get("aos0_ns", 0) > r["soa_per_component_ns"]), None)
    cross_fused = next((r["n"] for r in rows if r.get("aos0_ns", 0) > r["soa_fused_ns"]), None)
    return {"rows": rows, "sizes": list(sizes), "units": "ns per particle per step (kernel time, CUDA graph)",
            "soa3_ahead_of_aos0_from_n": cross, "soa_fused_ahead_of_aos0_from_n": cross_fused}


def issue_peak(torch, dev):
    """Issue-rate peak in T thread-instructions/s and its description."""
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    return (sms * SMSP_PER_SM * 32 * MAX_SM_MHZ * 1e6 / 1e12,
            f"issue rate: 1 warp-instruction/clock per SM sub-partition x {SMSP_PER_SM} x {sms} SMs x 32 lanes "
            f"at {MAX_SM_MHZ:.0f} MHz")


def hbm_roofline(bytes_per_unit, units, seconds, kernel=None):
    """Roofline entry of an HBM-bound launch: algorithmic bytes / time against the copy peak."""
    peak, kind = measured_peaks()
    achieved = bytes_per_unit * units / seconds / 1e9
    return {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
            "peak_kind": f"{kind} copy", "bytes_per_unit": bytes_per_unit,
            "traffic": ncu_traffic(kernel) if kernel else None, "kernel": kernel}


def hbm_equivalent(bytes_per_unit, units, seconds):
    """The rate a kernel that is not HBM-bound would need from HBM to do the same work in
    one pass per step (the plain step's algorithmic bytes per particle-step), against the
    copy peak: the algorithmic fraction beside an issue-rate roofline."""
    peak, kind = measured_peaks()
    achieved = bytes_per_unit * units / seconds / 1e9
    return {"achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
            "peak_kind": f"{kind} copy", "bytes_per_unit": bytes_per_unit}


def fp32_fraction(torch, dev, kernel, units, seconds):
    """FP32 lane operations per particle-step that ncu counted for the current sources
    (FADD + FMUL + FFMA thread instructions, each packed FP32x2 instruction counted as two)
    x units / time, against the FP32 pipes' peak: 128 FP32 lanes per SM per clock x SMs at
    the maximum SM clock.  None figures when no record matches the sources."""
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    peak = sms * 128 * MAX_SM_MHZ * 1e6 / 1e12
    rec = ncu_record(kernel)
    ops = float(rec["fp32_ops_per_particle_step"]) if rec and "fp32_ops_per_particle_step" in rec else None
    achieved = ops * units / seconds / 1e12 if ops else None
    return {"achieved": achieved, "peak": peak, "unit": "T FP32 lane-ops/s", "frac": achieved / peak if achieved else None,
            "ops_per_unit": ops, "peak_kind": f"128 FP32 lanes/SM/clock x {sms} SMs at {MAX_SM_MHZ:.0f} MHz"}


def alu_roofline(torch, dev, kernel, units, seconds):
    """Roofline entry of an issue-bound launch: the thread-instructions per unit that ncu
    counted for the current sources x units / time, against the issue-rate peak.  None
    figures when no record matches the sources."""
    peak, kind = issue_peak(torch, dev)
    rec = ncu_record(kernel)
    inst = float(rec["inst_per_particle_step"]) if rec and "inst_per_particle_step" in rec else None
    achieved = inst * units / seconds / 1e12 if inst else None
    return {"bound": "alu", "kernel": kernel, "achieved": achieved, "peak": peak, "unit": "Tinst/s",
            "frac": achieved / peak if achieved else None, "peak_kind": kind, "work_per_unit": inst,
            "work_unit": "thread-instructions per particle-step (ncu counter)", "units_per_launch": units,
            "traffic": ncu_traffic(kernel), "launch_ms": seconds * 1e3}


def _events(torch, stream, fn, reps=1):
    """Mean time in seconds of fn() over reps calls, with CUDA events on stream, after one
    untimed call."""
    fn()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(reps):
        fn()
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / 1e3 / reps


def row_one_pass(sx, torch, p, flow):
    """The one-pass-per-step kernel (soax_step): HBM roofline at 72 bytes per particle-step."""
    n = p.n
    t1 = _time(torch, lambda: p.step(flow, 1), reps=10)
    tf = _time(torch, lambda: p.step_fused(flow, RK2_PER_STEP), reps=3)
    rl = hbm_roofline(BYTES_PER_PARTICLE_STEP, n, t1, "k_step_soa")
    return {"kernel": "k_step_soa", "launch_ms": t1 * 1e3, "particle-steps/s": n / t1, "bound": "hbm",
            "achieved_GB/s": rl["achieved"], "peak_GB/s": rl["peak"], "frac": rl["frac"],
            "peak_kind": rl["peak_kind"], "traffic": rl["traffic"], "fused_over_one_pass": t1 * RK2_PER_STEP / tf,
            "roofline": rl}


def row_aos(sx, torch, p, flow):
    """AoS <-> SoA round trip (176 algorithmic bytes per particle) and the AoS step (72
    algorithmic bytes per particle-step, 96 moved in whole 48-B records)."""
    n = p.n
    aos = p.to_aos()
    t_rt = _time(torch, lambda: (p.to_aos(aos), p.from_aos(aos)), reps=5)
    rt = {"ms": t_rt * 1e3, "GB/s": 176 * n / t_rt / 1e9, "bytes_per_particle": 176,
          "roofline": hbm_roofline(176, n, t_rt, "aos_soa_roundtrip")}
    t_aos = _time(torch, lambda: p.step_aos(aos, flow, 1), reps=3)
    t_soa = _time(torch, lambda: p.step(flow, 1), reps=3)
    st = {"particle-steps/s": n / t_aos, "algorithmic_GB/s": 72 * n / t_aos / 1e9,
          "record_GB/s": 96 * n / t_aos / 1e9, "soa_over_aos": t_aos / t_soa,
          "roofline": hbm_roofline(72, n, t_aos, "k_step_aos")}
    del aos
    torch.cuda.empty_cache()
    return rt, st


def row_adjoint(sx, torch, dev, n=None):
    """Forward (checkpoints every 32 steps) + adjoint of the 1M-particle K = 1000 problem,
    against the plain step; each launch timed on its own and set against the issue rate
    with the instructions per particle-step ncu counted (k_adj_forward: one forward step
    with its checkpoint traffic; k_adj_reverse: one recomputed step and its reverse)."""
    wa = soax_inputs.WORKLOADS["adjoint_n1M"]
    n = wa["n"] if n is None else n
    da = soax_inputs.basic_set(n, wa["seed"])
    pa = sx.Particles([("pos", "f64", 3, "P"), ("vel", "f32", 3, "V")], n, device=dev, shadow=False)
    fa = sx.Flow(A=wa["A"], B=wa["B"], C=wa["C"], tau=wa["tau"], dt=wa["dt"])
    K, C = wa["K"], wa["ckpt_every"]
    wsa = pa.adjoint_workspace(K, C)
    xt = [torch.from_numpy(a).to(dev) for a in da["pos"]]
    stream = torch.cuda.current_stream(dev)

    def reset():
        pa.load({"pos": da["pos"], "vel": da["vel"]})

    reset()
    t_plain = _time(torch, lambda: pa.step(fa, K))
    reset()
    t_plain_fused = _time(torch, lambda: pa.step_fused(fa, K))
    reset()
    # Forward and adjoint timed apart (CUDA events on the launching stream), then together.
    t_fwd = _events(torch, stream, lambda: pa.step_checkpointed(fa, K, C, wsa))
    _, xb = pa.minimage_loss(xt, wsa)
    t_rev = _events(torch, stream, lambda: pa.step_adjoint(fa, K, C, wsa, xb))

    def fwd_adj():
        pa.step_checkpointed(fa, K, C, wsa)
        _, xb = pa.minimage_loss(xt, wsa)
        pa.step_adjoint(fa, K, C, wsa, xb)
    t_fa = _time(torch, fwd_adj)
    out = {"n": n, "K": K, "ckpt_every": C, "plain_ms": t_plain * 1e3, "plain_fused_ms": t_plain_fused * 1e3,
           "fwd_adj_ms": t_fa * 1e3, "fwd_ms": t_fwd * 1e3, "adj_ms": t_rev * 1e3,
           "ratio_vs_plain": t_fa / t_plain, "ratio_vs_plain_fused": t_fa / t_plain_fused,
           "roofline": {"k_adj_forward": alu_roofline(torch, dev, "k_adj_forward", n * K, t_fwd),
                        "k_adj_reverse": alu_roofline(torch, dev, "k_adj_reverse", n * K, t_rev)}}
    del pa, wsa, xt
    torch.cuda.empty_cache()
    return out


def row_batched(sx, torch, dev, nens=None, fixed_tune=False):
    """512 uneven ensembles (or the first nens of them): one persistent launch per step,
    all 200 steps in one fused launch, and 512 plain launches per step in a CUDA graph.
    fixed_tune: 2 particles per thread, 512 threads, 128-bit loads (the autotuner's usual
    pick) instead of autotuning, so the launches are the same on every run (profiling)."""
    wb = soax_inputs.WORKLOADS["batched_512"]
    sizes, taus, abc = soax_inputs.ensembles(wb["nens"], wb["nmin"], wb["nmax"], wb["seed"])
    nens = wb["nens"] if nens is None else nens
    parts, flows = [], []
    for e in range(nens):
        ne, tau = int(sizes[e]), float(taus[e])
        q = sx.Particles(sx.BASIC_SCHEMA, ne, device=dev, shadow=False)
        rng = np.random.default_rng(1000 + e)
        pos = np.minimum(rng.uniform(0.0, soax_inputs.TWO_PI, (3, ne)), np.nextafter(soax_inputs.TWO_PI, 0))
        vel = rng.normal(0.0, 0.1, (3, ne)).astype(np.float32)
        q.load({"pos": list(pos), "vel": list(vel)})
        parts.append(q)
        flows.append(sx.Flow(A=abc[e, 0], B=abc[e, 1], C=abc[e, 2], tau=tau, dt=wb["dt"]))
    total = int(sizes[:nens].sum())
    nst = wb["steps"]  # the workload's 200 steps for every form
    stream = torch.cuda.current_stream(dev)
    # One persistent launch per step (autotuned), over the workload's steps.
    tune = sx.Tune(2, 512, 128, 0) if fixed_tune else sx.autotune(parts, flows, nsteps_probe=1)
    wsb = sx.step_batched(parts, flows, 1, tune)
    t_b = _events(torch, stream, lambda: sx.step_batched(parts, flows, nst, tune, ws=wsb))
    # The workload's form: all its steps in ONE fused persistent launch (autotuned), called
    # directly and replayed from a CUDA graph.
    tf = sx.Tune(2, 512, 128, 1) if fixed_tune else sx.autotune(parts, flows, nsteps_probe=10, fuse=True)
    wsf = sx.batched_workspace(parts)
    sx.step_batched(parts, flows, 1, tf, ws=wsf)
    kf = wb["steps"]
    t_f = _events(torch, stream, lambda: sx.step_batched(parts, flows, kf, tf, ws=wsf))
    sx.step_batched(parts, flows, kf, tf, ws=wsf)  # the plan for these arguments is in place before capture
    torch.cuda.synchronize(dev)
    g_f = _graph(torch, dev, lambda s: sx.step_batched(parts, flows, kf, tf, ws=wsf, stream=s))
    t_fg = _events(torch, stream, g_f.replay)
    # Baseline: separate plain launches per step, one CUDA graph per step of all ensembles.
    g = _graph(torch, dev, lambda s: [q.step(f, 1, stream=s) for q, f in zip(parts, flows)])
    t_plain_b = _events(torch, stream, lambda: [g.replay() for _ in range(nst)])
    out = {"ensembles": len(parts), "particles": total,
           "persistent": {"steps": nst, "launches": nst, "tune": tune.__dict__, "ms": t_b * 1e3,
                          "particle-steps/s": total * nst / t_b,
                          "roofline": hbm_roofline(BYTES_PER_PARTICLE_STEP, total * nst, t_b, "k_step_batched")},
           "fused": {"steps": kf, "launches": 1, "tune": tf.__dict__, "ms": t_f * 1e3,
                     "particle-steps/s": total * kf / t_f,
                     "roofline": alu_roofline(torch, dev, "k_step_batched_fused", total * kf, t_f)},
           "fused_graph": {"steps": kf, "launches": 1, "ms": t_fg * 1e3, "particle-steps/s": total * kf / t_fg,
                           "how": "the fused launch captured in a CUDA graph and replayed"},
           "plain_launches": {"launches_per_step": len(parts), "steps": nst, "ms": t_plain_b * 1e3,
                              "particle-steps/s": total * nst / t_plain_b},
           "persistent_over_plain": t_plain_b / t_b,
           "fused_over_plain": (t_plain_b / nst) / (t_f / kf),
           "fused_graph_over_plain": (t_plain_b / nst) / (t_fg / kf)}
    del parts, g, g_f
    torch.cuda.empty_cache()
    return out


def _graph(torch, dev, fn):
    """fn captured in a CUDA graph on a side stream; returns the graph."""
    s = torch.cuda.Stream(dev)
    s.wait_stream(torch.cuda.current_stream(dev))
    g = torch.cuda.CUDAGraph()
    with torch.cuda.stream(s):
        with torch.cuda.graph(g, stream=s):
            fn(s)
    torch.cuda.current_stream(dev).wait_stream(s)
    return g


def row_plain_n65536(sx, torch, dev):
    """The 65,536-particle set, 100 RK2 steps, SoA and AoS, on the device (2.5 MiB of
    planes: L2-resident, so an HBM fraction means nothing here and the one-pass forms are
    launch-bound; the 100 launches are captured in one CUDA graph).  Forms: 100 one-pass
    SoA launches, the 100 steps in one fused launch, 100 AoS launches on the 48-B records;
    the oracle runs the full 100 steps beside them (SoA and AoS, all cores and one)."""
    w = soax_inputs.WORKLOADS["plain_n65536"]
    n, K = w["n"], w["steps"]
    d = soax_inputs.basic_set(n, w["seed"])
    flow = sx.Flow(A=w["A"], B=w["B"], C=w["C"], tau=w["tau"], dt=w["dt"])
    p = sx.Particles(sx.BASIC_SCHEMA, n, device=dev, shadow=False)
    p.load(d)
    aos = p.to_aos()
    stream = torch.cuda.current_stream(dev)
    g_soa = _graph(torch, dev, lambda s: p.step(flow, K, stream=s))
    g_aos = _graph(torch, dev, lambda s: p.step_aos(aos, flow, K, stream=s))
    t_soa = _events(torch, stream, g_soa.replay, reps=5)
    t_fused = _events(torch, stream, lambda: p.step_fused(flow, K), reps=5)
    t_aos = _events(torch, stream, g_aos.replay, reps=5)
    units = n * K
    out = {"n": n, "steps": K, "l2_resident": True,
           "note": "2.5 MiB of planes stay in the 126 MB L2: HBM fractions are not meaningful; one-pass forms are "
                   "bound by launch and per-step latency (100 launches in one CUDA graph)",
           "soa_one_pass_graph": {"ms": t_soa * 1e3, "particle-steps/s": units / t_soa,
                                  "launches": K, "hbm_equivalent_GB/s": 72 * units / t_soa / 1e9},
           "soa_fused_one_launch": {"ms": t_fused * 1e3, "particle-steps/s": units / t_fused, "launches": 1},
           "aos_one_pass_graph": {"ms": t_aos * 1e3, "particle-steps/s": units / t_aos, "launches": K},
           "soa_over_aos": t_aos / t_soa, "fused_over_one_pass": t_soa / t_fused}
    out["roofline"] = alu_roofline(torch, dev, "k_step_soa", units, t_soa)
    out["roofline"]["note"] = "one-pass kernel's ncu instruction count at its 16.7M-particle capture"
    out["cpu_baseline"] = oracle_baseline("plain_n65536", n, sort=False)
    del p, aos, g_soa, g_aos
    torch.cuda.empty_cache()
    return out


def row_wide_n64M(sx, torch, dev, n=None, intervals=None):
    """The wide record at its full size: 67,108,864 particles {i64 id, f64 pos[3], f32
    vel[3], f32 acc[3], f32 mass, u8 tag}, tau = 0.1 mass, dt = 5e-4, acc written, 200 RK2
    steps with a cell sort on the 64^3 grid every 20: each interval is one fused launch of
    20 steps that gathers every plane through the previous sort's permutation and writes
    the new 18-bit keys, then the stable radix sort of those keys (2 passes).  Also: the
    one-pass step (88 algorithmic bytes per particle-step), the 64-B record AoS <-> SoA
    round trip, and the oracle on a sample."""
    w = soax_inputs.WORKLOADS["wide_n64M"]
    n = w["n"] if n is None else n
    every, grid = w["sort_every"], w["grid"]
    nint = w["steps"] // every if intervals is None else intervals
    d = soax_inputs.wide_set(n, w["seed"])
    p = sx.Particles(sx.WIDE_SCHEMA, n, device=dev)
    p.load(d)
    del d
    flow = sx.Flow(A=w["A"], B=w["B"], C=w["C"], tau=0.0, dt=w["dt"], tau_field="mass",
                   tau_scale=w["tau_scale"], acc="acc")
    ws = p.sort_workspace(grid)
    keys = torch.empty(n, dtype=torch.int32, device=dev)
    stream = torch.cuda.current_stream(dev)
    pending = {"perm": None}

    def interval(ev=None):
        if ev is not None:
            ev[0].record(stream)
        p.step_fused(flow, every, grid=grid, keys=keys, perm=pending["perm"])
        if ev is not None:
            ev[1].record(stream)
        pending["perm"] = p.sort_perm(grid, keys, ws)[1]
        if ev is not None:
            ev[2].record(stream)

    for _ in range(2):
        interval()
    torch.cuda.synchronize(dev)
    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(nint)]
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for k in range(nint):
        interval(evs[k])
    e1.record(stream)
    torch.cuda.synchronize(dev)
    total = e0.elapsed_time(e1) / 1e3
    fused = statistics.mean(ev[0].elapsed_time(ev[1]) for ev in evs) / 1e3
    srt = statistics.mean(ev[1].elapsed_time(ev[2]) for ev in evs) / 1e3
    units = n * every * nint
    out = {"workload": "wide_n64M", "n": n, "rk2_steps": every * nint, "sort_every": every, "grid": grid,
           "fields": "i64 id, f64 pos[3], f32 vel[3], f32 acc[3], f32 mass, u8 tag",
           "flow": "ABC A=B=C=1, tau = 0.1 mass, dt = 5e-4, acc written",
           "ms": total * 1e3, "particle-steps/s": units / total, "interval_ms": total / nint * 1e3,
           "fused_launch_ms": fused * 1e3, "sort_ms": srt * 1e3,
           "l2": f"inputs larger than L2 ({n * 61 / 2**20:.0f} MiB of planes)"}
    rl = alu_roofline(torch, dev, "k_step_soa_fused_gather/wide", n * every, fused)
    rl["hbm_equivalent"] = hbm_equivalent(88, n * every, fused)
    out["roofline"] = rl
    # H1 as the workload states it: one pass over the planes per step.
    t1 = _time(torch, lambda: p.step(flow, 1), reps=5)
    out["step_one_pass"] = {"launch_ms": t1 * 1e3, "particle-steps/s": n / t1,
                            "roofline": hbm_roofline(88, n, t1, "k_step_soa/wide")}
    # The 64-B record round trip: SoA -> AoS reads 61 B of planes and writes 64 B, and back.
    aos = p.to_aos()
    t_rt = _time(torch, lambda: (p.to_aos(aos), p.from_aos(aos)), reps=3)
    out["aos_soa_roundtrip"] = {"ms": t_rt * 1e3, "bytes_per_particle": 250,
                                "roofline": hbm_roofline(250, n, t_rt, None)}
    del aos, p, ws, keys
    torch.cuda.empty_cache()
    out["cpu_baseline"] = oracle_baseline("wide_n64M", n)
    return out


def row_sort(sx, torch, dev, name, n=None):
    """The cell sort of a workload's near-sorted keys (its bench interval: a set sorted by
    cell, stepped sort_every steps, keyed again in that order), timed as the library's
    soax_sort_perm (the cell counting sort, with the radix passes gated behind it) and as
    the plain LSD radix sort of the same keys (soax_radix_sort_pairs, 2 passes), which
    must give the same permutation; algorithmic bytes: keys read twice and the
    permutation written (12 B per particle) for the counting sort, 32 B for the radix."""
    w = soax_inputs.WORKLOADS[name]
    n = w["n"] if n is None else n
    grid = w["grid"]
    wide = name == "wide_n64M"
    d = soax_inputs.wide_set(n, w["seed"]) if wide else soax_inputs.basic_set(n, w["seed"])
    schema = sx.WIDE_SCHEMA if wide else sx.BASIC_SCHEMA
    p = sx.Particles(schema, n, device=dev)
    p.load(d)
    del d
    f = (sx.Flow(A=w["A"], B=w["B"], C=w["C"], tau=0.0, dt=w["dt"], tau_field="mass", tau_scale=w["tau_scale"],
                 acc="acc") if wide else sx.Flow(A=w["A"], B=w["B"], C=w["C"], tau=w["tau"], dt=w["dt"]))
    ws = p.sort_workspace(grid)
    p.sort_by_cell(grid, ws)
    keys = p.step_fused(f, w["sort_every"], grid=grid)
    bits = int(grid ** 3 - 1).bit_length()
    stream = torch.cuda.current_stream(dev)
    t_cell = _events(torch, stream, lambda: p.sort_perm(grid, keys, ws), reps=10)
    perm_cell = p.sort_results(grid, ws)[1].clone()
    nb = ctypes.c_size_t()  # the radix sort's own workspace
    sx._check(sx.lib().soax_radix_workspace_bytes(n, bits, ctypes.byref(nb)))
    rws = torch.empty(max(nb.value, 16), dtype=torch.uint8, device=dev)
    vo = torch.empty(n, dtype=torch.int32, device=dev)
    t_radix = _events(torch, stream, lambda: sx.radix_sort_pairs(keys, None, bits, want_keys=False, ws=rws, out=vo),
                      reps=10)
    same = bool(torch.equal(perm_cell, vo))
    out = {"workload": name, "n": n, "grid": grid, "key_bits": bits, "same_permutation": same,
           "cell_sort_ms": t_cell * 1e3, "radix_sort_ms": t_radix * 1e3, "radix_over_cell": t_radix / t_cell,
           "cell_roofline": hbm_roofline(12, n, t_cell, None), "radix_roofline": hbm_roofline(32, n, t_radix, None)}
    del p, ws, keys, rws, vo
    torch.cuda.empty_cache()
    return out


def row_fixed(sx, torch, dev, n, nsteps_list):
    """Per-step and per-launch costs of the fused step: the bench's gather step (through
    a near-identity permutation), the fused step with keys and the plain fused step, each
    timed at every steps-per-launch in nsteps_list; with two or more, the slope and the
    intercept of the first two (ms per step, ms per launch)."""
    d = soax_inputs.basic_set(n, WL["seed"])
    p = sx.Particles(sx.BASIC_SCHEMA, n, device=dev)
    p.load(d)
    ws = p.sort_workspace(WL["grid"])
    f = sx.Flow(A=WL["A"], B=WL["B"], C=WL["C"], tau=WL["tau"], dt=WL["dt"])
    keys = p.step_fused(f, RK2_PER_STEP, grid=WL["grid"])
    perm = p.sort_perm(WL["grid"], keys, ws)[1]
    keys = p.step_fused(f, RK2_PER_STEP, grid=WL["grid"], keys=keys, perm=perm)
    perm = p.sort_perm(WL["grid"], keys, ws)[1]  # near-identity from here on
    forms = (("gather+keys", lambda ns: p.step_fused(f, ns, grid=WL["grid"], keys=keys, perm=perm)),
             ("fused+keys", lambda ns: p.step_fused(f, ns, grid=WL["grid"], keys=keys)),
             ("fused", lambda ns: p.step_fused(f, ns)))
    out = {}
    for name, fn in forms:
        ms = {ns: _time(torch, lambda: fn(ns), reps=5) * 1e3 for ns in nsteps_list}
        row = {"ms_per_launch": ms}
        if len(nsteps_list) >= 2:
            a, b = nsteps_list[0], nsteps_list[1]
            per = (ms[b] - ms[a]) / (b - a)
            row.update(ms_per_step=per, ms_fixed=ms[a] - a * per)
        out[name] = row
    return out


def secondary_rows(sx, torch, p, d, dev):
    n = p.n
    flow = sx.Flow(A=WL["A"], B=WL["B"], C=WL["C"], tau=WL["tau"], dt=WL["dt"])
    rows = {"euler_replica": euler_replica(sx, torch, n, dev), "step_one_pass": row_one_pass(sx, torch, p, flow)}
    rows["aos_soa_roundtrip"], rows["aos_step"] = row_aos(sx, torch, p, flow)
    rows["fwd_adjoint"] = row_adjoint(sx, torch, dev)
    rows["batched"] = row_batched(sx, torch, dev)
    rows["sort_sorted_n16M"] = row_sort(sx, torch, dev, "sorted_n16M")
    rows["plain_n65536"] = row_plain_n65536(sx, torch, dev)
    rows["wide_n64M"] = row_wide_n64M(sx, torch, dev)
    rows["sort_wide_n64M"] = row_sort(sx, torch, dev, "wide_n64M")
    return rows


def run_only(args):
    """One secondary row on its own, at a chosen size (for profiling captures)."""
    import torch
    import paper_1710_03462_b300 as sx
    dev = torch.device("cuda", torch.cuda.current_device())
    if args.only == "euler":
        row = euler_replica(sx, torch, args.n or WL["n"], dev, sizes=args.sizes or (0, 32))
    elif args.only == "euler_sweep":
        row = euler_sweep(sx, torch, dev, ns=[args.n] if args.n else None)
    elif args.only == "adjoint":
        row = row_adjoint(sx, torch, dev, args.n)
    elif args.only == "batched":
        row = row_batched(sx, torch, dev, args.nens, args.fixed_tune)
    elif args.only == "sort":
        row = {"sorted_n16M": row_sort(sx, torch, dev, "sorted_n16M", args.n),
               "wide_n64M": row_sort(sx, torch, dev, "wide_n64M", args.n)}
    elif args.only == "plain":
        row = row_plain_n65536(sx, torch, dev)
    elif args.only == "wide":
        row = row_wide_n64M(sx, torch, dev, args.n, args.intervals)
    elif args.only == "fixed":
        row = row_fixed(sx, torch, dev, args.n or WL["n"], args.nsteps or [RK2_PER_STEP, 2 * RK2_PER_STEP])
    else:
        n = args.n or WL["n"]
        flow = sx.Flow(A=WL["A"], B=WL["B"], C=WL["C"], tau=WL["tau"], dt=WL["dt"])
        p = sx.Particles(sx.BASIC_SCHEMA, n, device=dev)
        p.load(soax_inputs.basic_set(n, WL["seed"]))
        row = dict(zip(("aos_soa_roundtrip", "aos_step"), row_aos(sx, torch, p, flow)))
    print(json.dumps({"only": args.only, "n": args.n, "nens": args.nens, "fixed_tune": args.fixed_tune, "row": row}))
    return 0


def main(argv=None):
    args = parse_args(argv)
    if args.only:
        return run_only(args)
    if args.n is None:
        args.n = WL["n"]
    if args.impl == "reference":
        return run_reference(args)
    return run_soax(args)


if __name__ == "__main__":
    sys.exit(main())
