"""The benchmark configurations at their full sizes, in the launch configuration the
bench times (FP32-local single trains with the tuning the bench's autotuner picks on
this workload, batched trains autotuned in the test, FP64 runs default):

* 1e6-species track pulse: the first SBS steps in FP64 mode equal the numpy FP64
  reference and the whole trajectory (1 ps to 1 us, about 4e5 events) equals the C++
  FP64 reference (every event, every per-step count, all positions); the whole
  trajectory in FP32-local mode matches FP64-mode G-values over 32 seeds each within
  max(1 %, 3 sigma);
* multi-pulse build-up (10 pulses of 293k species, 0.1 ms apart) and the 64-train
  dose-rate sweep: exact conservation laws and internal consistency, which hold at any
  size (the reference cannot run these within a test)."""
import math

import numpy as np
import pytest

from harness import assert_fp64_parity, cuda_available, gpu_run, oracle_run
from paper_2509_03313_gb300 import chem, workloads as W

pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not cuda_available(), reason="needs a CUDA GPU")]

# steps per graph replay, hash limit, search mapping chosen per step, one kernel per phase
BENCH_TUNING = (8, 255, -1, chem.CHEM_LAUNCH_PHASES)


def _conserved(wl, tally, injected_types):
    """Charge, H and O (products' water counted through each reaction's water change)."""
    c0 = np.bincount(injected_types, minlength=wl.n_types)[:7]
    c = tally["counts"][:7]
    ev = tally["events"][:len(wl.reactions)]
    dw = np.array([r.water_delta for r in wl.reactions], dtype=np.int64)
    water = int((ev * dw).sum())
    assert int((c * W.CHARGE).sum()) == int((c0 * W.CHARGE).sum())
    assert int((c * W.N_H).sum()) + 2 * water == int((c0 * W.N_H).sum())
    assert int((c * W.N_O).sum()) + water == int((c0 * W.N_O).sum())
    stoich = np.zeros((len(wl.reactions), 7), dtype=np.int64)
    for r, rx in enumerate(wl.reactions):
        stoich[r, rx.a] -= 1
        stoich[r, rx.b] -= 1
        for p in rx.products:
            stoich[r, p] += 1
    assert np.array_equal(c, c0 + ev @ stoich)


def test_tracks_1e6_first_steps_fp64_equal_reference():
    wl = W.single_pulse_tracks(10_000, n_species=1_000_000)
    s = wl.schedule
    t3 = s.dt_min * (1.0 + s.dt_growth + s.dt_growth ** 2)  # three SBS steps
    o = oracle_run(wl, 10_000, t_end=t3)
    g = gpu_run(wl, 10_000, t_end=t3, capacity=1_400_000)
    assert len(o.step_log) == 3
    assert_fp64_parity(g, o, wl.L)


def test_tracks_1e6_whole_trajectory_fp64_equals_cxx_reference():
    wl = W.single_pulse_tracks(10_001, n_species=1_000_000)
    o = oracle_run(wl, 10_001, impl="cxx")
    g = gpu_run(wl, 10_001, capacity=1_400_000)
    assert len(o.step_log) == 102 and o.events_total.sum() > 300_000
    assert_fp64_parity(g, o, wl.L)


def test_tracks_1e6_fp32_local_g_values_match_fp64():
    """G(H2O2), G(OH) and G(e_aq) of whole 1e6-species trajectories: FP32-local in the
    bench's tuning against FP64 mode, 32 SBS seeds each (one context per precision, reset
    between seeds), within max(1 %, 3 sigma); every trajectory conserves charge, H and O."""
    import torch
    wl = W.single_pulse_tracks(10_000, n_species=1_000_000)
    p = wl.pulses[0]
    s = wl.schedule
    g = {}
    for prec in (chem.CHEM_FP32_LOCAL, chem.CHEM_FP64):
        cfg, keep = chem.make_config(
            wl.L, wl.D, wl.reactions, seed=500, precision=prec, dt_min=s.dt_min, dt_max=s.dt_max,
            dt_growth=s.dt_growth, reset_on_release=s.reset_on_release, cutoff_c=s.cutoff_c,
            sbs_horizon=s.sbs_horizon, capacity_species=1_400_000, capacity_pending=wl.n_species,
            capacity_candidates=700_000, stream=torch.cuda.current_stream().cuda_stream,
            allocator=chem.torch_allocator(0))
        ctx = chem.chem_init(cfg)
        try:
            if prec == chem.CHEM_FP32_LOCAL:
                chem.chem_set_tuning(ctx, *BENCH_TUNING)
            rows = []
            for seed in range(32):
                chem.chem_reset(ctx, 500 + seed)
                chem.chem_inject_pulse(ctx, p.types, p.xyz, p.t_arrival, p.energy_eV)
                chem.chem_run_until(ctx, wl.t_end)
                tally = chem.chem_tally(ctx, wl.n_types, len(wl.reactions))
                _conserved(wl, tally, p.types)
                rows.append(tally["G"])
            g[prec] = np.array(rows)
        finally:
            chem.chem_destroy(ctx)
    a, b = g[chem.CHEM_FP32_LOCAL], g[chem.CHEM_FP64]
    for t in (W.H2O2, W.OH, W.E_AQ):
        diff = abs(a[:, t].mean() - b[:, t].mean())
        sigma = math.sqrt(a[:, t].var(ddof=1) / len(a) + b[:, t].var(ddof=1) / len(b))
        assert diff <= max(0.01 * b[:, t].mean(), 3 * sigma), (t, a[:, t].mean(), b[:, t].mean(), sigma)


def test_multi_pulse_build_up_full_size():
    wl = W.multi_pulse(3)
    types = np.concatenate([p.types for p in wl.pulses])
    n_total = types.size
    stops = [k * 1e-4 + 2e-6 for k in range(len(wl.pulses))]  # just after each pulse
    r = gpu_run(wl, 3, precision=chem.CHEM_FP32_LOCAL, record=False, capacity=n_total + 200_000,
                t_stops=stops[:-1], t_end=wl.t_end, tuning=BENCH_TUNING)
    live = [int(t["counts"][:7].sum()) for t in r["tallies"]]
    # species are carried across the 0.1 ms intervals: every pulse adds to what is left
    assert all(b > a for a, b in zip(live, live[1:])), live
    assert r["tally"]["t"] == wl.t_end
    _conserved(wl, r["tally"], types)
    ids, st, _ = r["state"]
    assert np.array_equal(np.bincount(st, minlength=7)[:7], r["tally"]["counts"][:7])
    assert np.unique(ids).size == ids.size


def test_batched_sweep_full_size():
    import torch
    wls = W.batched_sweep(64)
    cfgs, keep = [], []
    for b, wl in enumerate(wls):
        s = wl.schedule
        cap = int(wl.n_species * 1.3) + 4096
        cfg, k = chem.make_config(wl.L, wl.D, wl.reactions, seed=900 + b, train_id=b,
                                  precision=chem.CHEM_FP32_LOCAL, dt_min=s.dt_min, dt_max=s.dt_max,
                                  dt_growth=s.dt_growth, reset_on_release=s.reset_on_release,
                                  sbs_horizon=s.sbs_horizon, capacity_species=cap,
                                  capacity_pending=max(wl.n_species, 1),
                                  capacity_candidates=max(1 << 16, cap // 4),
                                  stream=torch.cuda.current_stream().cuda_stream,
                                  allocator=chem.torch_allocator(0))
        cfgs.append(cfg)
        keep.append(k)
    ctx = chem.chem_batch_init(cfgs)
    try:
        for b, wl in enumerate(wls):
            for p in wl.pulses:
                chem.chem_batch_inject(ctx, b, p.types, p.xyz, p.t_arrival, p.energy_eV)
        chem.chem_autotune(ctx, 1500.0)
        # run a step past every arrival (steps are at most 0.1 us) so that every injected
        # species has been released
        ends = [max(wl.t_end, max(float(p.t_arrival.max()) for p in wl.pulses)) + 1e-6 for wl in wls]
        chem.chem_batch_run_until(ctx, ends)
        for b, wl in enumerate(wls):
            tal = chem.chem_batch_tally(ctx, b, 7, 9)
            assert tal["t"] == ends[b]
            _conserved(wl, tal, np.concatenate([p.types for p in wl.pulses]))
            ids, st, _ = chem.chem_batch_get_state(ctx, b)
            assert np.array_equal(np.bincount(st, minlength=7)[:7], tal["counts"][:7])
            assert np.unique(ids).size == ids.size
    finally:
        chem.chem_destroy(ctx)


def test_large_box_build_up_first_pulses_conserve():
    """The 10 um, 20-pulse build-up at full size for its first two pulses (750,000 species
    created, FP32-local): charge and atoms conserved exactly, counts equal to the injected
    species plus events times stoichiometry, and species carried into the second pulse."""
    import torch
    wl = W.large_build_up(seed=1, n_pulses=2)
    n = wl.n_species
    cfg, keep = chem.make_config(wl.L, wl.D, wl.reactions, seed=3, precision=chem.CHEM_FP32_LOCAL,
                                 dt_min=wl.schedule.dt_min, dt_max=wl.schedule.dt_max,
                                 dt_growth=wl.schedule.dt_growth, capacity_species=int(1.2 * n) + 4096,
                                 capacity_pending=n, capacity_candidates=max(4096, n // 4),
                                 stream=torch.cuda.current_stream().cuda_stream,
                                 allocator=chem.torch_allocator(0))
    ctx = chem.chem_init(cfg)
    try:
        for p in wl.pulses:
            chem.chem_inject_pulse(ctx, p.types, p.xyz, p.t_arrival, p.energy_eV)
        chem.chem_run_until(ctx, 10e-6)
        first = chem.chem_tally(ctx, 7, 9)
        chem.chem_run_until(ctx, wl.t_end)
        tal = chem.chem_tally(ctx, 7, 9)
    finally:
        chem.chem_destroy(ctx)
    injected = np.bincount(np.concatenate([p.types for p in wl.pulses]), minlength=7)
    nu = np.zeros((7, 9), np.int64)
    water = 0
    for r, rx in enumerate(W.WATER_REACTIONS):
        nu[rx.a, r] -= 1
        nu[rx.b, r] -= 1
        for q in rx.products:
            nu[q, r] += 1
        water += int(tal["events"][r]) * rx.water_delta
    counts = tal["counts"][:7]
    np.testing.assert_array_equal(counts, injected + nu @ tal["events"][:9])
    assert int(counts @ W.CHARGE) == int(injected @ W.CHARGE)
    assert int(counts @ W.N_H) + 2 * water == int(injected @ W.N_H)
    assert int(counts @ W.N_O) + water == int(injected @ W.N_O)
    assert first["counts"][:7].sum() > 50_000 and first["t"] == 10e-6
    assert tal["t"] == wl.t_end
