"""Benchmark of the SBS chemical stage on one GB300 (or N independent replicas).

Workload: single pulse of synthetic proton tracks, 5 um periodic cube, 200 straight
tracks of Gaussian spurs (sigma 2 nm), ~1e6 species arriving at t = 0, log-growing dt
from 1 ps (20 steps per decade) to 1 us. One benchmark step is one whole trajectory
(every SBS step from 1 ps to 1 us: release, diffusion, hash, sort, pair search,
matching, products, tallies) with a fresh seed.

Prints one JSON line. ``value`` is species-steps/s of the FP32-local form with the
species already resident in HBM (CUDA events around chem_run_until on the library's
stream, L2 flushed before every timed trajectory); the FP64 form, the matched G-values
and the end-to-end number through host buffers are reported beside it.

``--impl reference`` times the FP64 reference (the plain C++ program, one
single-threaded process per host core) instead: whole trajectories of the same workload
in a smaller box at the same track and species density, one per process and step.
"""
from __future__ import annotations

import argparse
import json
import math
import multiprocessing as mp
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "species-steps/s (diffuse+search+react) FP32-local vs FP64 at matched G(H2O2)"
UNIT = "species-steps/s"
WORKLOAD = ("single pulse of 200 synthetic proton tracks (Gaussian spurs, sigma 2 nm), "
            "5 um periodic cube, ~1e6 species at t=0, log dt 1 ps -> 1 us (20 steps/decade)")
# Algorithmic bytes per species and launch of each phase kernel: one read + one write of
# the state where the phase rewrites it, one read where it only reads it; sort passes
# read and write one (key, value) pair.
STATE_BYTES = {"fp32l": 16, "fp64": 28}
# Minimum lane instructions of the pair search's two kinds of work (FP32-local mode): a
# tested neighbour pair is one 16-byte load, three subtractions, a squared norm (one
# multiply, two fused multiply-adds), the type pair's cutoff and a compare; a pair
# inside its cutoff adds one acceptance test: the Philox4x32-10 block (ten rounds of two
# wide multiplies and two three-input XORs), the start separation from the two stored
# displacements (two loads, six adds, a squared norm), the two square roots and the
# exp(-a) bound, and the compare with the uniform.
ALU_OPS_TESTED = 9
ALU_OPS_IN_CUTOFF = 66
ISSUE_LANE_OPS_PER_S = 152 * 4 * 32 * 2.07e9
PHASE_BYTES = {"diffuse": lambda s: 2 * s, "gather": lambda s: 2 * s, "search": lambda s: s,
               "sort": lambda s: 16, "release": lambda s: 0, "begin": lambda s: 0, "react": lambda s: 0}


TRAFFIC_FILE = os.path.join(ROOT, "profiles", "traffic_tracks_1e6_fp32l.json")


def sources_digest():
    """SHA-256 over the device-code sources and the C header, to tell whether a recorded
    ncu measurement still describes the kernels that run (chem_api.cu holds host code
    only and is left out). Comments and white space are dropped first: editing them
    changes no kernel."""
    import hashlib
    import re
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2509_03313_gb300", "csrc")
    files = sorted(os.path.join(csrc, f) for f in os.listdir(csrc)
                   if f.endswith((".cu", ".cuh", ".h")) and f != "chem_api.cu")
    for f in files + [os.path.join(ROOT, "include", "chem.h")]:
        with open(f, encoding="utf-8") as fh:
            text = fh.read()
        text = re.sub(r"/\*.*?\*/", " ", text, flags=re.S)
        text = re.sub(r"//[^\n]*", " ", text)
        h.update(os.path.basename(f).encode() + b"\0" + " ".join(text.split()).encode())
    return h.hexdigest()


def recorded_traffic(kernel):
    """Mean DRAM bytes per launch of `kernel` from the committed ncu capture, or None when
    there is none or the sources changed since it was taken."""
    try:
        with open(TRAFFIC_FILE) as f:
            rec = json.load(f)
    except (OSError, ValueError):
        return None
    if rec.get("sources_sha256") != sources_digest():
        return None
    return rec.get("dram_bytes_per_launch", {}).get(kernel)


def shard_trains(sizes, world):
    """Trains of the batched sweep per rank: largest first to the least-loaded rank (by
    species count), so ranks get similar work; every train goes to exactly one rank."""
    loads = [0] * world
    out = [[] for _ in range(world)]
    for b in sorted(range(len(sizes)), key=lambda q: (-sizes[q], q)):
        r = min(range(world), key=lambda q: (loads[q], q))
        out[r].append(b)
        loads[r] += sizes[b]
    return [sorted(x) for x in out]


def gather_batched(species_steps, seconds, counts, device=None):
    """Whole-sweep species-steps (sum), time (slowest rank) and per-train final counts
    (each train's row comes from the one rank that ran it): the only exchange of the
    sharded sweep, once at the end."""
    import torch
    import torch.distributed as dist
    c = torch.as_tensor(np.asarray(counts, dtype=np.int64), device=device)
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(species_steps), float(seconds), c.cpu().numpy()
    a = torch.tensor([float(species_steps)], dtype=torch.float64, device=device)
    b = torch.tensor([float(seconds)], dtype=torch.float64, device=device)
    dist.all_reduce(a, op=dist.ReduceOp.SUM)
    dist.all_reduce(b, op=dist.ReduceOp.MAX)
    dist.all_reduce(c, op=dist.ReduceOp.SUM)
    return float(a[0]), float(b[0]), c.cpu().numpy()


def dist_env():
    return int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")), \
        int(os.environ.get("LOCAL_RANK", "0"))


def aggregate_over_ranks(species_steps, seconds, device=None):
    """Whole-job species-steps (sum over ranks) and the slowest rank's time (max): the
    ranks run independent replicas, so this is the only exchange."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(species_steps), float(seconds)
    a = torch.tensor([float(species_steps)], dtype=torch.float64, device=device)
    b = torch.tensor([float(seconds)], dtype=torch.float64, device=device)
    dist.all_reduce(a, op=dist.ReduceOp.SUM)
    dist.all_reduce(b, op=dist.ReduceOp.MAX)
    return float(a[0]), float(b[0])


# ------------------------------------------------------------------- CPU reference arm
# The reference is timed on whole trajectories (every SBS step from 1 ps to 1 us) of the
# benchmark workload in a smaller box with the same track density, species density and
# time-step schedule (workloads.tracks_same_density): its species-steps cost what the
# 1e6-species trajectory's cost, early and late steps alike, in seconds of CPU time.
ORACLE_L_NM = 1600.0
ORACLE_KINDS = {
    "cxx": "oracle (plain FP64 C++ program, one single-threaded process per core)",
    "numpy": "oracle (numpy/scipy FP64, one process per core)",
}


def _oracle_module(name: str):
    if name == "cxx":
        from oracle import cxx
        cxx.load()
        return cxx
    from oracle import sbs
    return sbs


def _oracle_worker(args):
    seed, L, n_warm, n_timed, impl = args
    from paper_2509_03313_gb300 import workloads as W
    ref = _oracle_module(impl)
    ss, busy = 0, 0.0
    for k in range(n_warm + n_timed):
        wl = W.tracks_same_density(seed + 7919 * k, L)
        o = ref.from_workload(wl, seed=seed + 7919 * k, record=False)
        t0 = time.perf_counter()
        o.run_until(wl.t_end)
        if k >= n_warm:
            busy += time.perf_counter() - t0
            ss += o.species_steps
    return ss, busy


def oracle_rate(n_proc: int, L: float, n_warm: int, n_timed: int, impl: str = "cxx"):
    """Aggregate species-steps/s of n_proc reference processes (one per core), each timing
    n_timed whole trajectories after n_warm untimed ones."""
    _oracle_module(impl)  # the C++ program is compiled once, before the workers start
    ctx = mp.get_context("spawn")
    with ctx.Pool(n_proc) as pool:
        t0 = time.perf_counter()
        res = pool.map(_oracle_worker, [(1000 + i, L, n_warm, n_timed, impl) for i in range(n_proc)])
        wall = time.perf_counter() - t0
    ss = sum(r[0] for r in res)
    busy = max(r[1] for r in res)
    return ss / busy, ss, busy, wall


def oracle_sample_text(n_proc, n_traj, L):
    from paper_2509_03313_gb300 import workloads as W
    n = W.tracks_same_density(1, L).n_species
    return (f"{n_proc} processes x {n_traj} whole trajectories (1 ps -> 1 us, all SBS steps) of the track "
            f"workload at the benchmark's density in a {L / 1000:g} um box ({n} species, "
            f"{max(1, int(round(200 * (L / 5000) ** 2)))} tracks)")


def run_reference_arm(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    cores = os.cpu_count() or 1
    n_proc = max(1, min(cores, args.ref_procs or cores))
    # each benchmark step: every process runs one whole trajectory
    rate, ss, busy, wall = oracle_rate(n_proc, ORACLE_L_NM, args.warmup, args.steps, args.cpu_oracle)
    sample = oracle_sample_text(n_proc, args.steps, ORACLE_L_NM)
    line = {"impl": "reference", "metric": METRIC, "value": rate, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * busy / max(1, args.steps),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": WORKLOAD, "species": args.species, "L_nm": 5000.0, "sample": sample},
            "cpu_baseline": {"value": rate, "unit": UNIT, "cores": n_proc,
                             "kind": ORACLE_KINDS[args.cpu_oracle], "sample": sample},
            "e2e": {"value": rate, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------------- GPU arm helpers
class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons while running."""

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.rows = []
        self.proc = None

    def __enter__(self):
        q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
             "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
             "clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 7:
                self.rows.append(parts)

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        if not self.rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        sm = [float(r[0]) for r in self.rows if r[0].replace(".", "").isdigit()]
        mx = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in self.rows for i in range(4) if r[3 + i].lower() == "active"})
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.rows)}


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured (MEASURED_PEAKS.json hbm_gbs)"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback 6.8 TB/s"


def nvtx_push(torch, name):
    try:
        torch.cuda.nvtx.range_push(name)
    except (AttributeError, RuntimeError):
        pass


def nvtx_pop(torch):
    try:
        torch.cuda.nvtx.range_pop()
    except (AttributeError, RuntimeError):
        pass


def make_ctx(chem, wl, precision, seed, cap, stream, alloc, profiling=False):
    s = wl.schedule
    cfg, keep = chem.make_config(
        wl.L, wl.D, wl.reactions, seed=seed, precision=precision, dt_min=s.dt_min, dt_max=s.dt_max,
        dt_growth=s.dt_growth, reset_on_release=s.reset_on_release, cutoff_c=s.cutoff_c,
        capacity_species=cap, capacity_pending=cap, capacity_candidates=max(1 << 16, cap // 4),
        stream=stream, allocator=alloc)
    ctx = chem.chem_init(cfg)
    if profiling:
        chem.chem_set_profiling(ctx, True)
    return ctx, keep


def trajectory(chem, ctx, pulse, seed, t_end, torch, stream, flush, timed_events):
    """Reset, inject (host -> device, outside the timed region), flush L2, time the run."""
    chem.chem_reset(ctx, seed)
    chem.chem_inject_pulse(ctx, pulse.types, pulse.xyz, pulse.t_arrival, pulse.energy_eV)
    with torch.cuda.stream(stream):
        flush.zero_()
        a, b = timed_events
        a.record(stream)
    chem.chem_run_until(ctx, t_end)
    with torch.cuda.stream(stream):
        b.record(stream)
    b.synchronize()
    return a.elapsed_time(b) * 1e-3


def run_gpu_arm(args):
    import torch

    from paper_2509_03313_gb300 import chem, workloads as W
    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    dev = local if world > 1 else 0
    torch.cuda.set_device(dev)
    stream = torch.cuda.Stream(device=dev)
    alloc = chem.torch_allocator(dev, stream)
    # CPU baseline first (spawned workers, before heavy GPU work), rank 0 only, N = 1 only
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cores = os.cpu_count() or 1
        n_proc = max(1, min(cores, args.ref_procs or cores))
        rate, ss, busy, wall = oracle_rate(n_proc, ORACLE_L_NM, 0, args.cpu_trajectories, args.cpu_oracle)
        cpu = {"value": rate, "unit": UNIT, "cores": n_proc, "kind": ORACLE_KINDS[args.cpu_oracle],
               "sample": oracle_sample_text(n_proc, args.cpu_trajectories, ORACLE_L_NM) + f"; {busy:.1f} s"}
    seed0 = 10_000 * (rank + 1)
    wl = W.single_pulse_tracks(seed0, n_species=args.species, n_tracks=args.tracks)
    pulse = wl.pulses[0]
    cap = int(pulse.n * 1.3) + 4096
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)  # > 129 MB L2
    ev = (torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
    peak, peak_src = measured_peaks()
    results = {}
    modes = [("fp32l", chem.CHEM_FP32_LOCAL, args.steps)]
    if not args.no_fp64:
        modes.append(("fp64", chem.CHEM_FP64, args.fp64_steps if args.fp64_steps > 0 else args.steps))
    for name, prec, k_steps in modes:
        # the timed trajectories run without phase events (recorded around every phase of
        # every step they cost about 13 % of the step); the phase times come from
        # profiled trajectories right after the timed and end-to-end ones
        ctx, keep = make_ctx(chem, wl, prec, seed0, cap, stream.cuda_stream, alloc, profiling=False)
        tuned = None
        try:
            if name == "fp32l" and args.tuned:
                tuned = tuple(int(v) for v in args.tuned.split(","))
                chem.chem_set_tuning(ctx, *tuned)
            elif name == "fp32l" and not args.no_autotune:
                chem.chem_reset(ctx, seed0 + 3)
                chem.chem_inject_pulse(ctx, pulse.types, pulse.xyz, pulse.t_arrival, pulse.energy_eV)
                tuned = chem.chem_autotune(ctx, args.autotune_ms)
            for w in range(args.warmup):
                trajectory(chem, ctx, pulse, seed0 + 7 + w, wl.t_end, torch, stream, flush, ev)
            st0 = chem.chem_get_stats(ctx)
            times, ss, g_h2o2, g_oh, g_e = [], 0, [], [], []
            if world > 1:
                torch.distributed.barrier()
            torch.cuda.synchronize()
            nvtx_push(torch, f"timed_{name}")  # lets a profiler select the timed launches
            with ClockSampler(dev) as clk:
                for k in range(k_steps):
                    dt = trajectory(chem, ctx, pulse, seed0 + 100 + k, wl.t_end, torch, stream, flush, ev)
                    tal = chem.chem_tally(ctx, 7, 9)
                    times.append(dt)
                    ss += tal["species_steps"]
                    g_h2o2.append(tal["G"][W.H2O2]); g_oh.append(tal["G"][W.OH]); g_e.append(tal["G"][W.E_AQ])
            torch.cuda.synchronize()
            nvtx_pop(torch)
            st1 = chem.chem_get_stats(ctx)
            # end to end through the public API with host buffers
            e2e_t, e2e_ss = [], 0
            h2d_per = pulse.n * (4 + 8 * 4)
            for k in range(max(1, k_steps // 2)):
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                chem.chem_reset(ctx, seed0 + 500 + k)
                chem.chem_inject_pulse(ctx, pulse.types, pulse.xyz, pulse.t_arrival, pulse.energy_eV)
                chem.chem_run_until(ctx, wl.t_end)
                tal = chem.chem_tally(ctx, 7, 9)
                e2e_t.append(time.perf_counter() - t0)
                e2e_ss += tal["species_steps"]
            # untimed trajectories on further seeds for the G comparison of the two modes
            for k in range(max(0, args.g_seeds - len(g_h2o2))):
                chem.chem_reset(ctx, seed0 + 2000 + k)
                chem.chem_inject_pulse(ctx, pulse.types, pulse.xyz, pulse.t_arrival, pulse.energy_eV)
                chem.chem_run_until(ctx, wl.t_end)
                tal = chem.chem_tally(ctx, 7, 9)
                g_h2o2.append(tal["G"][W.H2O2]); g_oh.append(tal["G"][W.OH]); g_e.append(tal["G"][W.E_AQ])
            # profiled trajectories: CUDA events around every phase on the library's stream
            prof_times, prof_ss, stp0, stp1 = [], 0, st1, st1
            if not args.no_phase_events:
                chem.chem_set_profiling(ctx, True)  # recaptures with phase events, timers zeroed
                stp0 = chem.chem_get_stats(ctx)
                for k in range(args.profiled):
                    prof_times.append(trajectory(chem, ctx, pulse, seed0 + 100 + k, wl.t_end, torch, stream,
                                                 flush, ev))
                    prof_ss += chem.chem_tally(ctx, 7, 9)["species_steps"]
                stp1 = chem.chem_get_stats(ctx)
        finally:
            chem.chem_destroy(ctx)
        tot = float(np.sum(times))
        per_phase = {}
        for ph in ("diffuse", "sort", "gather", "search", "react", "begin", "release"):
            ms = stp1["phase_ms"][ph]
            nl = stp1["phase_launches"][ph]
            per_phase[ph] = {"ms_total": ms, "launches": nl}
        keys = ("pairs_tested", "pairs_in_cutoff", "pairs_accepted", "steps_advanced")
        work = {k: st1[k] - st0[k] for k in keys}
        work_prof = {k: stp1[k] - stp0[k] for k in keys}
        results[name] = dict(times=times, ss=ss, tot=tot, G_H2O2=g_h2o2, G_OH=g_oh, G_e=g_e, work=work,
                             work_prof=work_prof, prof_times=prof_times, prof_ss=prof_ss,
                             launches=st1["kernel_launches"] - st0["kernel_launches"],
                             phases=per_phase, clocks=clk.summary(), e2e_t=e2e_t, e2e_ss=e2e_ss,
                             tuned=tuned,
                             h2d=h2d_per, d2h=8 * 7 + 8 * 7 + 8 * 9 + 16)
    # aggregate over ranks (replicas): sum of species-steps over the max time
    r = results["fp32l"]
    ss_all, t_max = aggregate_over_ranks(r["ss"], r["tot"], device=dev)
    # the batched sweep: every rank runs its share of the trains
    bres = None if args.no_batched else run_batched(args, chem, W, torch, stream, alloc, flush, rank, world, dev)
    # the same sweep with every pulse and the beam-off stages (rate equations), 10 s tail
    hres = None if args.no_hybrid else run_hybrid(args, chem, W, torch, stream, alloc, rank, world, dev,
                                                  tuned=bres.get("autotuned") if bres else None)
    vres = None if args.no_volume else run_volume_scaling(args, chem, W, torch, stream, alloc, rank, world, dev)
    lres = run_large(args, chem, W, torch, stream, alloc) if not args.no_large and rank == 0 else None
    mres = run_multi_pulse(args, chem, W, torch, stream, alloc) if not args.no_multi_pulse and rank == 0 else None
    rres = (run_replicas(args, chem, W, torch, stream, alloc, flush, r["tuned"])
            if args.replicas > 1 and rank == 0 else None)
    xres = (run_beyond_l2(args, chem, W, torch, stream, alloc, flush)
            if not args.no_beyond_l2 and rank == 0 else None)
    if rank != 0:
        return 0
    value = ss_all / t_max
    # roofline of the dominant phase kernel of the FP32-local run
    phases = r["phases"]
    dom = max(phases, key=lambda p: phases[p]["ms_total"])
    have_phases = phases[dom]["ms_total"] > 0.0
    sb = STATE_BYTES["fp32l"]
    dom_bytes = PHASE_BYTES[dom](sb) * r["prof_ss"]
    n_launch = max(1, phases[dom]["launches"])
    if dom == "sort":
        # species-steps per pass launch: every pass moves every species once
        dom_bytes = PHASE_BYTES["sort"](sb) * r["prof_ss"] * (phases["sort"]["launches"] / max(1, phases["diffuse"]["launches"]))
    achieved = dom_bytes / max(1e-12, phases[dom]["ms_total"] * 1e-3) / 1e9
    tuned = list(r["tuned"]) if r["tuned"] is not None else None

    def traffic_of(phase):
        # DRAM bytes per phase launch from the committed capture of the same tuning and
        # sources; the search phase launches both search kernels every step
        kerns = {"search": ("k_search_tps", "k_search"), "diffuse": ("k_diffuse",),
                 "sort": ("k_sort_pass",), "gather": ("k_gather",)}.get(phase)
        try:
            with open(TRAFFIC_FILE) as fh:
                rec_tuning = json.load(fh).get("tuning")
        except (OSError, ValueError):
            return None
        # same search mapping and launch form (the hash limit the autotuner picks varies
        # from run to run and moves the traffic little)
        same = rec_tuning is not None and tuned is not None and rec_tuning[2:] == tuned[2:]
        if not kerns or not same:
            return None
        vals = [recorded_traffic(k) for k in kerns]
        return None if any(v is None for v in vals) else sum(vals)

    def search_alu_roofline(res):
        # The search is bound by instruction issue, not by memory: its algorithmic work is
        # counted in lane instructions, ALU_OPS_TESTED per neighbour pair whose separation
        # is tested and ALU_OPS_IN_CUTOFF per pair inside its cutoff (one acceptance test),
        # against the issue ceiling of the part (one warp instruction per cycle and
        # scheduler: 152 SMs x 4 x 32 lanes x the maximum SM clock).
        ph = res["phases"]["search"]
        w = res["work_prof"]
        if ph["ms_total"] <= 0.0 or w["pairs_tested"] <= 0:
            return None
        ops = ALU_OPS_TESTED * w["pairs_tested"] + ALU_OPS_IN_CUTOFF * w["pairs_in_cutoff"]
        ach = ops / (ph["ms_total"] * 1e-3)
        peak_alu = ISSUE_LANE_OPS_PER_S
        return {"bound": "alu", "kernel": "search", "achieved": ach, "peak": peak_alu,
                "unit": "lane-instr/s (algorithmic)", "frac": ach / peak_alu, "traffic": traffic_of("search"),
                "peak_source": "152 SMs x 4 schedulers x 32 lanes x 2.07 GHz (one warp instruction per cycle "
                               "per scheduler)",
                "algorithmic_ops": f"{ALU_OPS_TESTED} lane-instr per tested pair + {ALU_OPS_IN_CUTOFF} per pair "
                                   "inside the cutoff",
                "pairs_tested_per_launch": w["pairs_tested"] / max(1, ph["launches"]),
                "pairs_in_cutoff_per_launch": w["pairs_in_cutoff"] / max(1, ph["launches"]),
                "pairs_tested_per_s": w["pairs_tested"] / (ph["ms_total"] * 1e-3),
                "pairs_in_cutoff_per_s": w["pairs_in_cutoff"] / (ph["ms_total"] * 1e-3),
                "avg_launch_ms": ph["ms_total"] / max(1, ph["launches"])}

    def roofline_of(phase):
        ph = phases[phase]
        if ph["ms_total"] <= 0.0:
            return None
        nb = PHASE_BYTES[phase](sb) * r["prof_ss"]
        if phase == "sort":
            nb *= phases["sort"]["launches"] / max(1, phases["diffuse"]["launches"])
        ach = nb / (ph["ms_total"] * 1e-3) / 1e9
        return {"bound": "hbm", "kernel": phase, "achieved": ach, "peak": peak, "unit": "GB/s",
                "frac": ach / peak, "traffic": traffic_of(phase), "peak_source": peak_src,
                "algorithmic_bytes": f"{PHASE_BYTES[phase](sb)} B per live species per launch",
                "avg_launch_ms": ph["ms_total"] / max(1, ph["launches"])}
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * r["tot"] / len(r["times"]),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": WORKLOAD, "species": int(pulse.n), "L_nm": wl.L,
                   "t_end_s": wl.t_end, "sbs_steps_per_trajectory": r["work"]["steps_advanced"] / len(r["times"]),
                   "mode": "FP32-local positions, FP64 clock/probabilities/tallies",
                   "l2": "flushed (256 MiB write) before every timed trajectory",
                   "phase_events": ("none in the timed trajectories; CUDA events around every phase in "
                                    f"{len(r['prof_times'])} profiled trajectories after them (rooflines, phases_ms)")
                   if not args.no_phase_events else "off",
                   "profiled_ms_per_trajectory": (1e3 * float(np.mean(r["prof_times"])) if r["prof_times"] else None),
                   "autotuned": None if r["tuned"] is None else
                   dict(zip(("steps_per_launch", "cells_per_axis_limit", "species_per_item", "launch_mode"), r["tuned"])),
                   "parallelism": "replicas" if world > 1 else "1 GPU"},
        "e2e": {"value": (r["e2e_ss"] / sum(r["e2e_t"])) if r["e2e_t"] else None, "unit": UNIT,
                "h2d_bytes_per_step": r["h2d"], "d2h_bytes_per_step": r["d2h"],
                "includes": "chem_reset + chem_inject_pulse (host arrays) + chem_run_until + chem_tally"},
        "gpu_launches": int(r["launches"]),
        "roofline": (search_alu_roofline(r) if dom == "search" else roofline_of(dom)) if have_phases else None,
        "roofline_hbm_search": roofline_of("search") if have_phases else None,
        "roofline_diffuse": roofline_of("diffuse") if have_phases else None,
        "search_work_per_trajectory": {k: v / len(r["times"]) for k, v in r["work"].items()},
        "phases_ms": {p: round(v["ms_total"], 3) for p, v in phases.items()},
        "phases_ms_over": f"{len(r['prof_times'])} profiled trajectories",
        "clocks": r["clocks"],
        "G_per_100eV_fp32l": {"H2O2": float(np.mean(r["G_H2O2"])), "OH": float(np.mean(r["G_OH"])),
                              "e_aq": float(np.mean(r["G_e"]))},
    }
    if "fp64" in results:
        f = results["fp64"]
        v64 = f["ss"] / f["tot"]
        line["fp64"] = {"value": v64, "unit": UNIT, "ms_per_step": 1e3 * f["tot"] / len(f["times"]),
                        "steps": len(f["times"]),
                        "phases_ms": {p: round(v["ms_total"], 3) for p, v in f["phases"].items()},
                        "G_per_100eV": {"H2O2": float(np.mean(f["G_H2O2"])), "OH": float(np.mean(f["G_OH"])),
                                        "e_aq": float(np.mean(f["G_e"]))}}
        line["speedup_fp32l_over_fp64"] = value / v64
        g32, g64 = np.array(r["G_H2O2"]), np.array(f["G_H2O2"])
        line["G_H2O2_match"] = {"seeds": [len(g32), len(g64)],
                                "fp32l_mean": float(g32.mean()), "fp64_mean": float(g64.mean()),
                                "rel_diff": float(abs(g32.mean() - g64.mean()) / g64.mean()),
                                "sigma_rel": float(math.sqrt(g32.var(ddof=1) / len(g32) + g64.var(ddof=1) / len(g64)) / g64.mean())
                                if len(g32) > 1 and len(g64) > 1 else None}
    if bres is not None:
        line["batched"] = bres
        if "fp64" in line and bres.get("value"):
            line["speedup_batched_fp32l_over_plain_fp64"] = bres["value"] / line["fp64"]["value"]
    if hres is not None:
        line["hybrid"] = hres
    if vres is not None:
        line["volume_scaling"] = vres
    if lres is not None:
        line["large"] = lres
    if mres is not None:
        line["multi_pulse"] = mres
    if rres is not None:
        line["batched_replicas"] = rres
        if "fp64" in line:
            line["speedup_batched_replicas_over_plain_fp64"] = rres["value"] / line["fp64"]["value"]
    if xres is not None:
        line["beyond_l2"] = xres
    line["cpu_baseline"] = cpu
    print(json.dumps(line), flush=True)
    return 0


def run_batched(args, chem, W, torch, stream, alloc, flush, rank=0, world=1, device=None):
    """64 independent pulse trains of the dose-rate sweep (10 us window) advanced
    together in one context per rank: one hash for the rank's trains, the launch form,
    steps per replay, hash limit and search mapping chosen by chem_autotune. With
    several ranks the trains are split between them (no exchange until the end)."""
    wls_all = W.batched_sweep(scale=args.batch_scale)
    mine = shard_trains([w.n_species for w in wls_all], world)[rank]
    wls = [wls_all[b] for b in mine]
    cfgs, keep = [], []
    for b, wl in zip(mine, wls):
        s = wl.schedule
        n = wl.n_species
        cfg, k = chem.make_config(
            wl.L, wl.D, wl.reactions, seed=77 + b, train_id=b, precision=chem.CHEM_FP32_LOCAL,
            dt_min=s.dt_min, dt_max=s.dt_max, dt_growth=s.dt_growth, sbs_horizon=s.sbs_horizon,
            capacity_species=int(n * 1.3) + 4096, capacity_pending=n + 16,
            capacity_candidates=max(4096, n // 2), stream=stream.cuda_stream, allocator=alloc)
        cfgs.append(cfg)
        keep.append(k)
    ctx = chem.chem_batch_init(cfgs)
    ends = [wl.t_end for wl in wls]

    def load(seed_base):
        chem.chem_batch_reset(ctx, [seed_base + b for b in mine])
        for i, wl in enumerate(wls):
            for p in wl.pulses:
                chem.chem_batch_inject(ctx, i, p.types, p.xyz, p.t_arrival, p.energy_eV)

    counts = np.zeros((len(wls_all), 7), dtype=np.int64)
    try:
        load(500)
        if args.batch_tuned:
            tuned = tuple(int(v) for v in args.batch_tuned.split(","))
            chem.chem_set_tuning(ctx, *tuned)
        else:
            tuned = chem.chem_autotune(ctx, args.autotune_ms)
        ev = (torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
        times, ss = [], 0
        for k in range(args.batch_reps + 1):
            load(600 + 100 * k)
            with torch.cuda.stream(stream):
                flush.zero_()
                ev[0].record(stream)
            chem.chem_batch_run_until(ctx, ends)
            with torch.cuda.stream(stream):
                ev[1].record(stream)
            ev[1].synchronize()
            if k == 0:
                continue  # warm-up repetition
            times.append(ev[0].elapsed_time(ev[1]) * 1e-3)
            tal = [chem.chem_batch_tally(ctx, i, 7, 9) for i in range(len(wls))]
            ss += sum(t["species_steps"] for t in tal)
            for i, b in enumerate(mine):
                counts[b] = tal[i]["counts"][:7]
    finally:
        chem.chem_destroy(ctx)
    ss_all, t_all, counts_all = gather_batched(ss, sum(times), counts, device=device)
    return {"value": ss_all / t_all, "unit": UNIT, "trains": len(wls_all),
            "species": int(sum(w.n_species for w in wls_all)), "reps": len(times),
            "ms_per_rep": 1e3 * t_all / len(times), "window_s": wls_all[0].t_end,
            "mode": "FP32-local, one context per rank for its trains (launch form chosen by the autotuner)",
            "scaling": "strong (the 64 trains are split between the ranks)" if world > 1 else "1 GPU",
            "autotuned": dict(zip(("steps_per_launch", "cells_per_axis_limit", "species_per_item", "launch_mode"), tuned)),
            "species_at_end": [int(v) for v in counts_all.sum(axis=0)],
            "workload": "dose-rate sweep: 64 trains, Dav log-spaced 0.01-1e5 Gy/s at Dp 2e5 and 1e6 Gy/s, "
                        "species log-spaced 1e4-2e6 per 10 pulses, pulses of 4 bunches, 10 us window"}


def sum_over_ranks(rows, device=None):
    """Element-wise sum of a float array over the ranks (each train's row is filled on
    the one rank that ran it, zeros elsewhere)."""
    import torch
    import torch.distributed as dist
    a = torch.as_tensor(np.asarray(rows, dtype=np.float64), device=device)
    if dist.is_available() and dist.is_initialized() and dist.get_world_size() > 1:
        dist.all_reduce(a, op=dist.ReduceOp.SUM)
    return a.cpu().numpy()


def run_trains(chem, hybrid, wls_all, plans_all, stream, alloc, rank, world, device, tuned=None):
    """Run the (kind, t_end) plans of this rank's share of the trains in one batched
    FP32-local context. Returns (species-steps, slowest wall seconds, slowest seconds in
    the rate-equation stages, most integrator steps of one stage, rows) with rows[b] =
    post-irradiation counts (7), E_dep, radicals at the end of the second-to-last pulse
    and (real, before rounding) when the last pulse starts: summed over the ranks."""
    import torch
    mine = shard_trains([w.n_species for w in wls_all], world)[rank]
    wls = [wls_all[b] for b in mine]
    plans = [plans_all[b] for b in mine]
    cfgs, keep = [], []
    for b, wl in zip(mine, wls):
        s = wl.schedule
        n = wl.n_species
        cfg, k = chem.make_config(
            wl.L, wl.D, wl.reactions, seed=91 + b, train_id=b, precision=chem.CHEM_FP32_LOCAL,
            dt_min=s.dt_min, dt_max=s.dt_max, dt_growth=s.dt_growth,
            capacity_species=int(n * 0.8) + 4096, capacity_pending=n + 16,
            capacity_candidates=max(4096, n // 4), cells_per_axis_max=128,
            stream=stream.cuda_stream, allocator=alloc)
        cfgs.append(cfg)
        keep.append(k)
    rows = np.zeros((len(wls_all), 10))
    ss, wall, ode, steps_max = 0, 0.0, 0.0, 0
    if wls:
        ctx = chem.chem_batch_init(cfgs)
        try:
            if tuned:
                chem.chem_set_tuning(ctx, *[int(tuned[k]) for k in ("steps_per_launch", "cells_per_axis_limit",
                                                                     "species_per_item", "launch_mode")])
            for i, wl in enumerate(wls):
                for p in wl.pulses:
                    chem.chem_batch_inject(ctx, i, p.types, p.xyz, p.t_arrival, p.energy_eV)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            run = hybrid.run_plans(ctx, plans)
            torch.cuda.synchronize()
            wall = time.perf_counter() - t0
            steps_max = max(chem.chem_batch_homogeneous_report(ctx, i)[2] for i in range(len(wls)))
        finally:
            chem.chem_destroy(ctx)
        ss, ode = run["species_steps"], run["seconds"]["ode"]
        frac = hybrid.buildup_fraction(run, nu=hybrid.stoichiometry(7, wls[0].reactions))
        for i, b in enumerate(mine):
            rows[b, :7] = run["counts"][-1, i]
            rows[b, 7] = sum(p.energy_eV for p in wls[i].pulses)
            rows[b, 8] = frac[i]
    ss_all, wall_all, _ = gather_batched(ss, wall, np.zeros(1, np.int64), device=device)
    _, ode_all, _ = gather_batched(0, ode, np.zeros(1, np.int64), device=device)
    _, steps_all, _ = gather_batched(0, float(steps_max), np.zeros(1, np.int64), device=device)
    return ss_all, wall_all, ode_all, int(steps_all), sum_over_ranks(rows, device=device)


def run_hybrid(args, chem, W, torch, stream, alloc, rank=0, world=1, device=None, tuned=None):
    """Sec. 2.1 alternation on the GPU: step-by-step chemistry while the beam is on, the
    rate equations for the rest of each interval and for 10 s after the last pulse.
    (1) The 64 trains of the dose-rate sweep with all 10 pulses: post-irradiation
    G(H2O2) per train and the radical build-up before the last pulse, whose onset gives
    the SDR/UHDR threshold of Sec. 3.3. (2) Separate irradiations of 1-20 pulses at 1 and
    1e4 Gy/s: the H2O2 yield as the slope of post-irradiation concentration against dose
    (Fig. Concentration-Dose). Timed end to end on the host clock (every call syncs);
    trains are split between the ranks."""
    from paper_2509_03313_gb300 import hybrid
    wls_all, plans_all = W.hybrid_sweep(scale=args.hybrid_scale)
    descs = W.dose_rate_sweep()
    ss, wall, ode, steps, rows = run_trains(chem, hybrid, wls_all, plans_all, stream, alloc, rank, world,
                                            device, tuned)
    g_h2o2 = rows[:, 6] * 100.0 / rows[:, 7]
    per_dp = {}
    for dp in sorted({d["pulse_dose_rate"] for d in descs}):
        idx = [d["train"] for d in descs if d["pulse_dose_rate"] == dp]
        dav = [descs[q]["avg_dose_rate"] for q in idx]
        per_dp[f"{dp:g}"] = {
            "avg_dose_rate_Gy_s": [round(v, 4) for v in dav],
            "G_H2O2_post": [round(float(g_h2o2[q]), 4) for q in idx],
            "radical_buildup": [round(float(rows[q, 8]), 5) for q in idx],
            "threshold_avg_dose_rate": hybrid.threshold_dose_rate(dav, rows[idx, 8]),
        }
    out = {"value": ss / wall, "unit": UNIT, "trains": len(wls_all),
           "species": int(sum(w.n_species for w in wls_all)), "wall_s": wall, "ode_s": ode,
           "integrator_steps_max": steps,
           "mode": "FP32-local SBS while the beam is on; rate equations (GPU) between pulses and for 10 s after",
           "timing": "host clock around the whole alternation, species-steps of the SBS stages",
           "per_pulse_dose_rate": per_dp,
           "workload": "dose-rate sweep: 64 trains, Dav log-spaced 0.01-1e5 Gy/s at Dp 2e5 and 1e6 Gy/s, "
                       "species log-spaced 1e4-2e6 over 10 pulses of 4 bunches each, all pulses, 10 s tail"}
    if not args.no_dose_series:
        wls_d, plans_d, meta = W.dose_series()
        ss_d, wall_d, ode_d, _, rows_d = run_trains(chem, hybrid, wls_d, plans_d, stream, alloc, rank, world,
                                                    device, tuned)
        series = {}
        for dav in sorted({m["avg_dose_rate"] for m in meta}):
            idx = [q for q, m in enumerate(meta) if m["avg_dose_rate"] == dav]
            L = wls_d[idx[0]].L
            dose = rows_d[idx, 7] * 1.602176634e-19 / (L ** 3 * 1e-24)  # J per kg of water
            conc = hybrid.concentration(rows_d[idx, 6], L)
            slope, g = hybrid.dose_slope_yield(dose, conc)
            series[f"{dav:g}"] = {"pulses": [meta[q]["n_pulses"] for q in idx],
                                  "dose_Gy": [round(float(v), 4) for v in dose],
                                  "H2O2_post_M": [float(v) for v in conc],
                                  "yield_mol_per_J": slope, "yield_per_100eV": g}
        out["dose_series"] = {"workload": "1, 5, 10, 15, 20 pulses of 1e5 species (about 1 Gy each) at "
                                          "Dp 1e6 Gy/s, Dav 1 and 1e4 Gy/s, each followed by 10 s",
                              "wall_s": wall_d, "ode_s": ode_d, "species_steps_per_s": ss_d / wall_d,
                              "per_avg_dose_rate": series}
    return out


def run_volume_scaling(args, chem, W, torch, stream, alloc, rank=0, world=1, device=None):
    """Volume-scaling study of Sec. 2.2 / Sec. 3.1 on the GPU: one mixture concentration in boxes of
    0.2, 0.5 and 1.0 um (8, 4 and 2 seeds) followed to 1 ms by the FP32-local SBS in one
    batched context per rank; mean concentrations per box at 1 ms, their largest
    relative spread across the boxes, and the ratio of the SBS to the GPU rate equations
    from the same initial mixture (the paper: SBS above the well-mixed kinetics by up to
    20 % for H2 and 12 % for H2O2)."""
    boxes = {200.0: 8, 500.0: 4, 1000.0: 2}
    trains = [(L, s) for L, n in boxes.items() for s in range(n)]
    wls_all = [W.volume_scaling(L, seed=100 + s) for L, s in trains]
    mine = shard_trains([w.n_species for w in wls_all], world)[rank]
    rows = np.zeros((len(trains), 7))
    ss, wall = 0, 0.0
    if mine:
        cfgs, keep = [], []
        for b in mine:
            wl = wls_all[b]
            sch = wl.schedule
            n = wl.n_species
            c, k = chem.make_config(wl.L, wl.D, wl.reactions, seed=300 + b, train_id=b,
                                    precision=chem.CHEM_FP32_LOCAL, dt_min=sch.dt_min, dt_max=sch.dt_max,
                                    dt_growth=sch.dt_growth, capacity_species=2 * n + 4096,
                                    capacity_pending=n, capacity_candidates=max(4096, n),
                                    stream=stream.cuda_stream, allocator=alloc)
            cfgs.append(c)
            keep.append(k)
        ctx = chem.chem_batch_init(cfgs)
        try:
            for i, b in enumerate(mine):
                p = wls_all[b].pulses[0]
                chem.chem_batch_inject(ctx, i, p.types, p.xyz, p.t_arrival, p.energy_eV)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            chem.chem_batch_run_until(ctx, [wls_all[b].t_end for b in mine])
            torch.cuda.synchronize()
            wall = time.perf_counter() - t0
            for i, b in enumerate(mine):
                tal = chem.chem_batch_tally(ctx, i, 7, 9)
                L = trains[b][0]
                rows[b] = tal["counts"][:7] / (6.02214076e23 * L ** 3 * 1e-24)
                ss += tal["species_steps"]
        finally:
            chem.chem_destroy(ctx)
    ss_all, wall_all, _ = gather_batched(ss, wall, np.zeros(1, np.int64), device=device)
    rows = sum_over_ranks(rows, device=device)
    # the rate equations on the GPU from the 1 um box's initial mixture (deterministic)
    wl = W.volume_scaling(1000.0, seed=100)
    cfg, keep = chem.make_config(wl.L, wl.D, wl.reactions, seed=5, capacity_species=2 * wl.n_species,
                                 capacity_pending=wl.n_species, capacity_candidates=4096,
                                 stream=stream.cuda_stream, allocator=alloc)
    ctx = chem.chem_init(cfg)
    try:
        p = wl.pulses[0]
        chem.chem_inject_pulse(ctx, p.types, p.xyz, p.t_arrival, p.energy_eV)
        chem.chem_run_homogeneous(ctx, wl.t_end)
        ode = chem.chem_tally(ctx, 7, 9)["counts"][:7] / (6.02214076e23 * wl.L ** 3 * 1e-24)
    finally:
        chem.chem_destroy(ctx)
    means = {}
    for L in boxes:
        idx = [b for b, (LL, _) in enumerate(trains) if LL == L]
        means[L] = rows[idx].mean(axis=0)
    m = np.array([means[L] for L in boxes])
    # species with at least 20 molecules per smallest box (fewer is counting noise)
    big = m.min(axis=0) > 20.0 / (6.02214076e23 * min(boxes) ** 3 * 1e-24)
    mb = m[:, big]
    spread = float(((mb.max(axis=0) - mb.min(axis=0)) / mb.mean(axis=0)).max()) if big.any() else None
    return {"value": ss_all / wall_all if wall_all > 0 else None, "unit": UNIT, "wall_s": wall_all,
            "boxes_nm": list(boxes), "seeds": list(boxes.values()),
            "conc_1ms_M": {f"{L:g}": [float(v) for v in means[L]] for L in boxes},
            "max_rel_spread_across_boxes": spread,
            "spread_species": "those with >= 20 molecules in the 0.2 um box at 1 ms",
            "sbs_over_rate_equations_1ms": {"H2": float(means[1000.0][5] / ode[5]),
                                            "H2O2": float(means[1000.0][6] / ode[6])},
            "workload": "2,000 species (e 600, OH 600, H 120, H3O+ 600, OH- 80) per (0.2 um)^3, boxes of "
                        "0.2/0.5/1.0 um, log dt from 1 ps to 1 ms, FP32-local"}


def phase_rooflines(phases, ss, state_bytes, work, peak, peak_src):
    """HBM roofline of every phase kernel over a run (algorithmic bytes of the phase per
    species-step, summed, over the phase's summed device time), and the search's issue
    roofline from the pair counters."""
    out = {}
    diff_launches = max(1, phases["diffuse"]["launches"])
    for ph in ("diffuse", "sort", "gather", "search"):
        ms = phases[ph]["ms_total"]
        if ms <= 0.0:
            continue
        nb = PHASE_BYTES[ph](state_bytes) * ss
        if ph == "sort":
            nb *= phases["sort"]["launches"] / diff_launches
        ach = nb / (ms * 1e-3) / 1e9
        out[ph] = {"bound": "hbm", "achieved": ach, "peak": peak, "unit": "GB/s", "frac": ach / peak,
                   "peak_source": peak_src, "ms_total": ms, "launches": phases[ph]["launches"],
                   "algorithmic_bytes": f"{PHASE_BYTES[ph](state_bytes)} B per species per launch"}
    ms = phases["search"]["ms_total"]
    if ms > 0.0 and work["pairs_tested"] > 0:
        ops = ALU_OPS_TESTED * work["pairs_tested"] + ALU_OPS_IN_CUTOFF * work["pairs_in_cutoff"]
        out["search_alu"] = {"bound": "alu", "achieved": ops / (ms * 1e-3), "peak": ISSUE_LANE_OPS_PER_S,
                             "unit": "lane-instr/s (algorithmic)",
                             "frac": ops / (ms * 1e-3) / ISSUE_LANE_OPS_PER_S,
                             "pairs_tested_per_s": work["pairs_tested"] / (ms * 1e-3),
                             "pairs_in_cutoff_per_s": work["pairs_in_cutoff"] / (ms * 1e-3)}
    return out


def timed_trajectories(chem, torch, wl, precision, seeds, n_warm, stream, alloc, flush, tuning=None):
    """Whole trajectories of a single-pulse workload in one context with per-phase device
    timers: n_warm untimed, then one per seed timed with CUDA events (L2 flushed before
    each). Returns species-steps, seconds, per-phase times, counters and G(H2O2)."""
    pulse = wl.pulses[0]
    cap = int(pulse.n * 1.3) + 4096
    ctx, keep = make_ctx(chem, wl, precision, seeds[0], cap, stream.cuda_stream, alloc, profiling=True)
    ev = (torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
    try:
        if tuning is not None:
            chem.chem_set_tuning(ctx, *tuning)
        for w in range(n_warm):
            trajectory(chem, ctx, pulse, seeds[0] + 31 + w, wl.t_end, torch, stream, flush, ev)
        chem.chem_set_profiling(ctx, True)
        st0 = chem.chem_get_stats(ctx)
        ss, tot, g = 0, 0.0, []
        for sd in seeds:
            tot += trajectory(chem, ctx, pulse, sd, wl.t_end, torch, stream, flush, ev)
            tal = chem.chem_tally(ctx, 7, 9)
            ss += tal["species_steps"]
            g.append(float(tal["G"][6]))
        st1 = chem.chem_get_stats(ctx)
    finally:
        chem.chem_destroy(ctx)
    phases = {ph: {"ms_total": st1["phase_ms"][ph], "launches": st1["phase_launches"][ph]}
              for ph in ("diffuse", "sort", "gather", "search", "react", "begin", "release")}
    work = {k: st1[k] - st0[k] for k in ("pairs_tested", "pairs_in_cutoff", "pairs_accepted", "steps_advanced")}
    return ss, tot, phases, work, g


def run_replicas(args, chem, W, torch, stream, alloc, flush, tuned):
    """The benchmark workload as R independent trajectories (seeds differ) advanced together
    in one batched context: one hash and one graph for all R pulses, the grid limit and
    launch form of the single-train run. Species-steps/s over whole trajectories, L2
    flushed before each."""
    wl = W.single_pulse_tracks(10_000, n_species=args.species, n_tracks=args.tracks)
    pulse = wl.pulses[0]
    s = wl.schedule
    R = args.replicas
    cap = int(pulse.n * 1.3) + 4096
    n_lim = tuned[1] if tuned is not None else 255
    cfgs, keep = [], []
    for b in range(R):
        cfg, k = chem.make_config(wl.L, wl.D, wl.reactions, seed=5 + b, train_id=b,
                                  precision=chem.CHEM_FP32_LOCAL, dt_min=s.dt_min, dt_max=s.dt_max,
                                  dt_growth=s.dt_growth, capacity_species=cap, capacity_pending=cap,
                                  capacity_candidates=max(1 << 16, cap // 4), cells_per_axis_max=n_lim,
                                  stream=stream.cuda_stream, allocator=alloc)
        cfgs.append(cfg)
        keep.append(k)
    ctx = chem.chem_batch_init(cfgs)
    ev = (torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
    times, ss = [], 0
    try:
        chem.chem_set_tuning(ctx, tuned[0] if tuned is not None else 8, n_lim, -1,
                             tuned[3] if tuned is not None else chem.CHEM_LAUNCH_PHASES)
        for rep in range(args.replica_reps + 1):
            chem.chem_batch_reset(ctx, [20_000 + 100 * rep + b for b in range(R)])
            for b in range(R):
                chem.chem_batch_inject(ctx, b, pulse.types, pulse.xyz, pulse.t_arrival, pulse.energy_eV)
            with torch.cuda.stream(stream):
                flush.zero_()
                ev[0].record(stream)
            chem.chem_batch_run_until(ctx, [wl.t_end] * R)
            with torch.cuda.stream(stream):
                ev[1].record(stream)
            ev[1].synchronize()
            if rep == 0:
                continue  # warm-up repetition
            times.append(ev[0].elapsed_time(ev[1]) * 1e-3)
            ss += sum(chem.chem_batch_tally(ctx, b, 7, 9)["species_steps"] for b in range(R))
    finally:
        chem.chem_destroy(ctx)
    return {"value": ss / sum(times), "unit": UNIT, "replicas": R, "species": int(R * pulse.n),
            "ms_per_rep": 1e3 * float(np.mean(times)), "reps": len(times),
            "workload": f"{R} independent trajectories of the benchmark workload (seeds differ) in one "
                        "batched context, FP32-local, 1 ps -> 1 us"}


def run_beyond_l2(args, chem, W, torch, stream, alloc, flush):
    """The benchmark workload at 20x the volume (13.6 um box, same track and species
    density, 2e7 species): state arrays of 320 MB (FP32-local) and 560 MB (FP64), beyond
    the 126 MB L2, so every phase's traffic reaches HBM. Per-phase HBM rooflines and the
    search's issue roofline in both precisions."""
    wl = W.tracks_same_density(seed=4242, L=13572.0)
    peak, peak_src = measured_peaks()
    out = {"workload": f"single pulse of tracks at the benchmark's density, 13.6 um box, "
                       f"{wl.n_species} species, log dt 1 ps -> 1 us", "species": int(wl.n_species)}
    tuning = tuple(int(v) for v in args.tuned.split(",")) if args.tuned else None
    for name, prec, n_timed in (("fp32l", chem.CHEM_FP32_LOCAL, 2), ("fp64", chem.CHEM_FP64, 1)):
        if name == "fp64" and args.no_fp64:
            continue
        seeds = [4300 + k for k in range(n_timed)]
        ss, tot, phases, work, g = timed_trajectories(chem, torch, wl, prec, seeds, 1, stream, alloc, flush,
                                                      tuning if name == "fp32l" else None)
        out[name] = {"value": ss / tot, "unit": UNIT, "ms_per_trajectory": 1e3 * tot / n_timed,
                     "trajectories": n_timed, "G_H2O2": g,
                     "sbs_steps_per_trajectory": work["steps_advanced"] / n_timed,
                     "phases_ms": {p: round(v["ms_total"], 3) for p, v in phases.items()},
                     "rooflines": phase_rooflines(phases, ss, STATE_BYTES[name], work, peak, peak_src)}
    return out


def run_multi_pulse(args, chem, W, torch, stream, alloc):
    """Multi-pulse build-up (10 pulses of 1 us at 1e6 Gy/s pulse dose rate, 0.1 ms apart,
    163 tracks x 1,800 species each, step by step throughout, species carried across the
    intervals), FP32-local: wall time, species-steps/s, live species and G(H2O2) at the
    end of every pulse and before the next."""
    wl = W.multi_pulse(seed=11)
    n = wl.n_species
    period = 1e-4
    stops = sorted({round(k * period + d, 12) for k in range(len(wl.pulses)) for d in (1e-6, period)})
    stops = [t for t in stops if t <= wl.t_end] + ([wl.t_end] if wl.t_end not in stops else [])
    cfg, keep = chem.make_config(wl.L, wl.D, wl.reactions, seed=11, precision=chem.CHEM_FP32_LOCAL,
                                 dt_min=wl.schedule.dt_min, dt_max=wl.schedule.dt_max,
                                 dt_growth=wl.schedule.dt_growth, capacity_species=n + 200_000,
                                 capacity_pending=n, capacity_candidates=max(4096, n // 4),
                                 stream=stream.cuda_stream, allocator=alloc)
    ctx = chem.chem_init(cfg)
    try:
        if args.tuned:
            chem.chem_set_tuning(ctx, *[int(v) for v in args.tuned.split(",")])
        for p in wl.pulses:
            chem.chem_inject_pulse(ctx, p.types, p.xyz, p.t_arrival, p.energy_eV)
        st0 = chem.chem_get_stats(ctx)
        g, live = [], []
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for t in stops:
            chem.chem_run_until(ctx, t)
            tal = chem.chem_tally(ctx, 7, 9)
            g.append(round(float(tal["G"][6]), 4))
            live.append(int(tal["counts"][:7].sum()))
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
        st1 = chem.chem_get_stats(ctx)
        tal = chem.chem_tally(ctx, 7, 9)
    finally:
        chem.chem_destroy(ctx)
    return {"workload": "10 pulses of 1 us (163 tracks x 1,800 species each, arrivals uniform over the "
                        "pulse) every 0.1 ms, 5 um box, step by step throughout (dt reset at every "
                        "arrival, 10 ps -> 1 us)",
            "species_created": int(n), "wall_s": wall, "value": tal["species_steps"] / wall, "unit": UNIT,
            "sbs_steps": st1["steps_advanced"] - st0["steps_advanced"],
            "timing": "host clock around the run_until calls (each syncs)",
            "t_s": stops, "live": live, "G_H2O2": g, "peak_live": max(live)}


def run_large(args, chem, W, torch, stream, alloc):
    """Large build-up (10 um, 20 pulses, 20 Gy, ~7.5e6 species created), step by step
    throughout, FP32-local and FP64: G(H2O2) at the end of every pulse and before the
    next, wall time and species-steps/s of each, and the FP32-local / FP64 G(H2O2) ratio
    at the end (one seed each)."""
    wl = W.large_build_up(seed=1)
    n = wl.n_species
    period = 10e-6
    stops = sorted({round(k * period + d, 12) for k in range(20) for d in (1e-6, period)})
    out = {"workload": "10 um cube, 20 pulses of ~1 Gy (648 tracks, 375,000 species, 4 bunches each) every "
                       "10 us at 1e6 Gy/s pulse dose rate, step by step throughout, to 200 us",
           "species_created": int(n), "t_s": stops}
    precisions = [("fp32l", chem.CHEM_FP32_LOCAL)] + ([] if args.no_large_fp64 else [("fp64", chem.CHEM_FP64)])
    for name, prec in precisions:
        cfg, keep = chem.make_config(wl.L, wl.D, wl.reactions, seed=3, precision=prec,
                                     dt_min=wl.schedule.dt_min, dt_max=wl.schedule.dt_max,
                                     dt_growth=wl.schedule.dt_growth, capacity_species=int(1.2 * n) + 4096,
                                     capacity_pending=n, capacity_candidates=max(4096, n // 4),
                                     stream=stream.cuda_stream, allocator=alloc)
        ctx = chem.chem_init(cfg)
        try:
            if name == "fp32l" and args.tuned:
                chem.chem_set_tuning(ctx, *[int(v) for v in args.tuned.split(",")])
            for p in wl.pulses:
                chem.chem_inject_pulse(ctx, p.types, p.xyz, p.t_arrival, p.energy_eV)
            g = []
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            for t in stops:
                chem.chem_run_until(ctx, t)
                g.append(float(chem.chem_tally(ctx, 7, 9)["G"][6]))
            torch.cuda.synchronize()
            wall = time.perf_counter() - t0
            tal = chem.chem_tally(ctx, 7, 9)
        finally:
            chem.chem_destroy(ctx)
        out[name] = {"wall_s": wall, "value": tal["species_steps"] / wall, "unit": UNIT,
                     "G_H2O2": [round(v, 4) for v in g], "live_at_end": int(tal["counts"][:7].sum())}
    if "fp64" in out:
        out["G_H2O2_end_fp32l_over_fp64"] = out["fp32l"]["G_H2O2"][-1] / out["fp64"]["G_H2O2"][-1]
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--species", type=int, default=1_000_000)
    ap.add_argument("--tracks", type=int, default=200,
                    help="number of tracks (species per track = species / tracks)")
    ap.add_argument("--fp64-steps", type=int, default=0,
                    help="FP64 trajectories (default: as many as --steps, same seeds)")
    ap.add_argument("--cpu-trajectories", type=int, default=4,
                    help="whole reference trajectories per process in the cpu_baseline sample")
    ap.add_argument("--cpu-oracle", default="cxx", choices=["cxx", "numpy"],
                    help="reference timed on the host cores: the plain C++ program or the numpy one")
    ap.add_argument("--ref-procs", type=int, default=0)
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-phase-events", action="store_true")
    ap.add_argument("--profiled", type=int, default=3,
                    help="trajectories with phase events after the timed ones (phase times, rooflines)")
    ap.add_argument("--g-seeds", type=int, default=32,
                    help="seeds per precision for the FP32-local / FP64 G comparison (untimed "
                         "trajectories on other seeds make up the difference)")
    ap.add_argument("--no-autotune", action="store_true")
    ap.add_argument("--autotune-ms", type=float, default=1500.0)
    ap.add_argument("--tuned", default="",
                    help="FP32-local tuning instead of the autotuner: steps_per_launch,"
                         "cells_per_axis_limit,species_per_item,launch_mode (1 phases, 2 persistent)")
    ap.add_argument("--batch-tuned", default="", help="the same for the batched run")
    ap.add_argument("--no-batched", action="store_true")
    ap.add_argument("--batch-scale", type=float, default=1.0)
    ap.add_argument("--batch-reps", type=int, default=2)
    ap.add_argument("--no-hybrid", action="store_true")
    ap.add_argument("--hybrid-scale", type=float, default=1.0)
    ap.add_argument("--no-dose-series", action="store_true")
    ap.add_argument("--no-volume", action="store_true")
    ap.add_argument("--no-large", action="store_true", help="skip the 10 um, 20-pulse build-up")
    ap.add_argument("--no-large-fp64", action="store_true", help="run it in FP32-local mode only")
    ap.add_argument("--no-multi-pulse", action="store_true", help="skip the 10-pulse build-up (0.1 ms apart)")
    ap.add_argument("--no-beyond-l2", action="store_true", help="skip the 2e7-species workload")
    ap.add_argument("--replicas", type=int, default=4,
                    help="trajectories of the benchmark workload batched in one context (1: skip the leg)")
    ap.add_argument("--replica-reps", type=int, default=3)
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference_arm(args)
    return run_gpu_arm(args)


if __name__ == "__main__":
    sys.exit(main())
