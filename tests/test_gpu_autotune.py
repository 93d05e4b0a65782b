"""The autotuner times trial runs from the live state and restores it after each one:
an FP64 run that is tuned half-way must still reproduce the FP64 reference exactly."""
import numpy as np
import pytest

from harness import assert_fp64_parity, cuda_available, event_matrix, oracle_run, step_matrix
from paper_2509_03313_gb300 import chem, workloads as W

pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not cuda_available(), reason="needs a CUDA GPU")]


def _ctx(wl, seed, precision, **kw):
    import torch
    s = wl.schedule
    cfg, keep = chem.make_config(wl.L, wl.D, wl.reactions, seed=seed, precision=precision,
                                 dt_min=s.dt_min, dt_max=s.dt_max, dt_growth=s.dt_growth,
                                 capacity_species=65536, capacity_event_log=1 << 15,
                                 capacity_step_log=1 << 14,
                                 stream=torch.cuda.current_stream().cuda_stream, **kw)
    return chem.chem_init(cfg), keep


@pytest.mark.parametrize("launch_mode", [chem.CHEM_LAUNCH_PHASES, chem.CHEM_LAUNCH_PERSISTENT])
def test_tuning_mid_run_leaves_fp64_results_unchanged(launch_mode):
    wl = W.uniform_2000(seed=51, L=200.0, n_steps=200)
    ctx, keep = _ctx(wl, 51, chem.CHEM_FP64, launch_mode=launch_mode)
    try:
        p = wl.pulses[0]
        chem.chem_inject_pulse(ctx, p.types, p.xyz, p.t_arrival, p.energy_eV)
        chem.chem_run_until(ctx, 70e-9)
        spl, n_lim, ih, mode = chem.chem_autotune(ctx, 400.0)
        assert spl in (8, 32) and ih == -1 and n_lim >= 3  # the mapping stays chosen per step
        assert mode in (chem.CHEM_LAUNCH_PHASES, chem.CHEM_LAUNCH_PERSISTENT)
        chem.chem_run_until(ctx, wl.t_end)
        ids, types, xyz = chem.chem_get_state(ctx)
        o = np.argsort(ids)
        g = {"tally": chem.chem_tally(ctx, 7, 9), "events": chem.chem_get_events(ctx),
             "steps": chem.chem_get_step_log(ctx),
             "state": (ids[o].astype(np.int64), types[o].astype(np.int64), xyz[o])}
    finally:
        chem.chem_destroy(ctx)
    assert_fp64_parity(g, oracle_run(wl, 51, t_stops=[70e-9]), wl.L)


def test_tuning_fp32_local_keeps_counts_consistent():
    pulse = W.track_pulse(20, 800.0, 1000, seed=52)
    wl = W.Workload("tracks_tune", 800.0, [pulse],
                    W.Schedule(dt_min=1e-12, dt_max=1e-7, dt_growth=W.LOG_GROWTH_20_PER_DECADE),
                    t_end=1e-7)
    ctx, keep = _ctx(wl, 52, chem.CHEM_FP32_LOCAL, capacity_candidates=1 << 14)
    try:
        chem.chem_inject_pulse(ctx, pulse.types, pulse.xyz, pulse.t_arrival, pulse.energy_eV)
        chem.chem_run_until(ctx, 1e-11)
        chem.chem_autotune(ctx, 300.0)
        chem.chem_run_until(ctx, wl.t_end)
        tal = chem.chem_tally(ctx, 7, 9)
        ids, types, _ = chem.chem_get_state(ctx)
    finally:
        chem.chem_destroy(ctx)
    assert tal["t"] == wl.t_end
    assert np.array_equal(np.bincount(types, minlength=7), tal["counts"])
    assert np.unique(ids).size == ids.size
    c0 = np.bincount(pulse.types, minlength=7)
    assert int((tal["counts"] * W.CHARGE).sum()) == int((c0 * W.CHARGE).sum())


@pytest.mark.parametrize("tuning", [(4, 12, 16, chem.CHEM_LAUNCH_PERSISTENT), (32, 200, 32, chem.CHEM_LAUNCH_PHASES),
                                    (8, 200, -1, chem.CHEM_LAUNCH_PHASES), (8, 200, 0, chem.CHEM_LAUNCH_PHASES)])
def test_set_tuning_mid_run_leaves_fp64_results_unchanged(tuning):
    wl = W.uniform_2000(seed=53, L=200.0, n_steps=200)
    ctx, keep = _ctx(wl, 53, chem.CHEM_FP64)
    try:
        p = wl.pulses[0]
        chem.chem_inject_pulse(ctx, p.types, p.xyz, p.t_arrival, p.energy_eV)
        chem.chem_run_until(ctx, 90e-9)
        chem.chem_set_tuning(ctx, *tuning)
        chem.chem_run_until(ctx, wl.t_end)
        ids, types, xyz = chem.chem_get_state(ctx)
        o = np.argsort(ids)
        g = {"tally": chem.chem_tally(ctx, 7, 9), "events": chem.chem_get_events(ctx),
             "steps": chem.chem_get_step_log(ctx),
             "state": (ids[o].astype(np.int64), types[o].astype(np.int64), xyz[o])}
    finally:
        chem.chem_destroy(ctx)
    assert_fp64_parity(g, oracle_run(wl, 53, t_stops=[90e-9]), wl.L)


def test_set_tuning_rejects_out_of_range_values():
    wl = W.uniform_2000(seed=54, L=200.0, n_steps=10)
    ctx, keep = _ctx(wl, 54, chem.CHEM_FP64)
    try:
        for bad in [(0, 12, 16, 1), (8, 2, 16, 1), (8, 12, 33, 1), (8, 12, -2, 1), (8, 12, 16, 0),
                    (8, 12, 16, 3)]:
            with pytest.raises(chem.ChemError) as ei:
                chem.chem_set_tuning(ctx, *bad)
            assert ei.value.status == chem.CHEM_EINVAL
    finally:
        chem.chem_destroy(ctx)


def test_profiling_on_then_off_mid_run_leaves_fp64_results_unchanged():
    # Phase events are recorded only by graphs captured with profiling on; a run after
    # profiling is switched off (and the grid limit changed) must neither query them nor
    # fail, and the results stay the reference's.
    wl = W.uniform_2000(seed=53, L=200.0, n_steps=120)
    ctx, keep = _ctx(wl, 53, chem.CHEM_FP64)
    try:
        p = wl.pulses[0]
        chem.chem_inject_pulse(ctx, p.types, p.xyz, p.t_arrival, p.energy_eV)
        chem.chem_set_profiling(ctx, True)
        chem.chem_set_tuning(ctx, 1, 40, -1, 1)
        chem.chem_run_until(ctx, 40e-9)
        st = chem.chem_get_stats(ctx)
        assert st["phase_launches"]["search"] == 40 and st["phase_ms"]["search"] > 0.0
        chem.chem_set_profiling(ctx, False)
        chem.chem_set_tuning(ctx, 8, 25, -1, 1)
        chem.chem_run_until(ctx, 90e-9)
        chem.chem_set_tuning(ctx, 4, 60, -1, 1)
        chem.chem_run_until(ctx, wl.t_end)
        ids, types, xyz = chem.chem_get_state(ctx)
        o = np.argsort(ids)
        g = {"tally": chem.chem_tally(ctx, 7, 9), "events": chem.chem_get_events(ctx),
             "steps": chem.chem_get_step_log(ctx),
             "state": (ids[o].astype(np.int64), types[o].astype(np.int64), xyz[o])}
    finally:
        chem.chem_destroy(ctx)
    assert_fp64_parity(g, oracle_run(wl, 53, t_stops=[40e-9, 90e-9]), wl.L)


def test_sort_passes_follow_the_grid_limit():
    # A single-train context sorts only the key bits its runtime grid limit needs: at most
    # 15 cells per axis -> 12-bit keys, two radix passes; 200 -> 24 bits, three. Ten steps
    # at each limit differ by ten sort launches, and the results stay the reference's.
    wl = W.uniform_2000(seed=54, L=200.0, n_steps=30)
    ctx, keep = _ctx(wl, 54, chem.CHEM_FP64)
    try:
        p = wl.pulses[0]
        chem.chem_inject_pulse(ctx, p.types, p.xyz, p.t_arrival, p.energy_eV)
        launches = []
        for lim, t in ((15, 10e-9), (200, 20e-9), (15, wl.t_end)):
            chem.chem_set_tuning(ctx, 1, lim, -1, chem.CHEM_LAUNCH_PHASES)
            before = chem.chem_get_stats(ctx)["kernel_launches"]
            chem.chem_run_until(ctx, t)
            launches.append(chem.chem_get_stats(ctx)["kernel_launches"] - before)
        ids, types, xyz = chem.chem_get_state(ctx)
        o = np.argsort(ids)
        g = {"tally": chem.chem_tally(ctx, 7, 9), "events": chem.chem_get_events(ctx),
             "steps": chem.chem_get_step_log(ctx),
             "state": (ids[o].astype(np.int64), types[o].astype(np.int64), xyz[o])}
    finally:
        chem.chem_destroy(ctx)
    # the third run may keep three passes: its species were last sorted on the finer grid
    assert launches[1] - launches[0] == 10, launches
    assert launches[2] in (launches[0], launches[1]), launches
    assert_fp64_parity(g, oracle_run(wl, 54, t_stops=[10e-9, 20e-9]), wl.L)
