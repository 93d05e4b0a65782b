"""GPU homogeneous (beam-off) stage against the reference (Sec. 2.3, Eq. 3 / Eq. 4).

The library integrates the rate equations with its own scheme, so real extents agree
within the integrators' tolerances; whole events, counts, the re-created particles and
every SBS step after a stage agree exactly (FP64 mode), provided no extent's fraction
lies within that tolerance of its rounding uniform, which each test checks first."""
import numpy as np
import pytest

from harness import assert_fp64_parity, event_matrix, step_matrix
from oracle import homogeneous as H
from oracle import sbs
from paper_2509_03313_gb300 import chem, workloads as W

pytestmark = pytest.mark.gpu

EXT_RTOL = 1e-8   # real extents, relative
EXT_ATOL = 1e-5   # real extents, events


def _config(wl, seed, precision, train_id=0, cap=None, launch_mode=chem.CHEM_LAUNCH_AUTO):
    import torch
    s = wl.schedule
    n = wl.n_species
    cap = cap or max(8192, 4 * n)
    return chem.make_config(
        wl.L, wl.D, wl.reactions, seed=seed, train_id=train_id, precision=precision,
        dt_min=s.dt_min, dt_max=s.dt_max, dt_growth=s.dt_growth, reset_on_release=s.reset_on_release,
        cutoff_c=s.cutoff_c, sbs_horizon=s.sbs_horizon, capacity_species=cap,
        capacity_pending=max(n, 1), capacity_candidates=max(4096, cap // 2),
        capacity_event_log=4 * cap + 1024, capacity_step_log=400000, launch_mode=launch_mode,
        stream=torch.cuda.current_stream().cuda_stream, allocator=chem.torch_allocator(0))


def _check_extents(e_gpu, E_gpu, e_ref, u):
    n = e_ref.shape[0]
    np.testing.assert_allclose(e_gpu[:n], e_ref, rtol=EXT_RTOL, atol=EXT_ATOL)
    x = np.maximum(e_ref, 0.0)
    tol = EXT_ATOL + EXT_RTOL * x
    assert np.all(np.abs((x - np.floor(x)) - u) > 2 * tol), \
        "a rounding decision lies within the integrators' tolerance: pick another seed"


def _run_both(wl, seed, plan, precision=chem.CHEM_FP64):
    """Run the (kind, t_end) plan through the library and the reference."""
    cfg, keep = _config(wl, seed, precision)
    ctx = chem.chem_init(cfg)
    o = sbs.from_workload(wl, seed=seed)
    g = {"tallies": [], "reports": []}
    try:
        for p in wl.pulses:
            chem.chem_inject_pulse(ctx, p.types, p.xyz, p.t_arrival, p.energy_eV)
        for kind, t in plan:
            if kind == "sbs":
                chem.chem_run_until(ctx, t)
                o.run_until(t)
            else:
                stage = o.hx_stage
                chem.chem_run_homogeneous(ctx, t)
                e_ref, E_ref = o.run_homogeneous(t)
                e, E, steps = chem.chem_batch_homogeneous_report(ctx, 0)
                if precision == chem.CHEM_FP64:
                    _check_extents(e, E, e_ref, H.rounding_uniforms(len(wl.reactions), stage, o.key))
                g["reports"].append((e, E, steps, e_ref, E_ref))
            g["tallies"].append((chem.chem_tally(ctx, wl.n_types, len(wl.reactions)), o.counts().copy(),
                                 o.events_total.copy(), o.t))
        g["tally"] = g["tallies"][-1][0]
        ids, types, xyz = chem.chem_get_state(ctx)
        order = np.argsort(ids)
        g["state"] = (ids[order].astype(np.int64), types[order].astype(np.int64), xyz[order])
        g["events"] = chem.chem_get_events(ctx)
        g["steps"] = chem.chem_get_step_log(ctx)
    finally:
        chem.chem_destroy(ctx)
    return g, o


def _totals(counts, water=0):
    return (int(counts @ W.CHARGE), int(counts @ W.N_H) + 2 * water, int(counts @ W.N_O) + water)


def test_stage_between_sbs_runs_matches_reference_fp64():
    wl = W.uniform_2000(seed=11, L=400.0, n_steps=50)
    plan = [("sbs", 5e-8), ("ode", 1e-3), ("sbs", 1e-3 + 3e-8)]
    g, o = _run_both(wl, 11, plan)
    e, E, steps, e_ref, E_ref = g["reports"][0]
    np.testing.assert_array_equal(E[:9], E_ref)
    assert 0 < steps < 2000
    # tallies right after the stage: the survivors are counted before they are re-created
    tal, counts, events, t = g["tallies"][1]
    np.testing.assert_array_equal(tal["counts"][:7], counts)
    np.testing.assert_array_equal(tal["events"][:9], events)
    assert tal["t"] == t == 1e-3
    # the SBS after the stage: every event, step, id and position as in the reference
    assert_fp64_parity(g, o, wl.L)


def test_pulse_train_alternates_sbs_and_rate_equations_fp64():
    pulses = W.pulse_train(3, 1e-4, 1e-6, n_tracks=6, L=600.0, species_per_track=120, seed=5)
    wl = W.Workload("hybrid3", 600.0, pulses,
                    W.Schedule(dt_min=1e-11, dt_max=1e-7, dt_growth=W.LOG_GROWTH_20_PER_DECADE),
                    t_end=0.0)
    plan = W.hybrid_stages(3, 1e-4, 1e-6, tail_s=10.0)
    assert [k for k, _ in plan] == ["sbs", "ode"] * 3
    g, o = _run_both(wl, 5, plan)
    for tal, counts, events, t in g["tallies"]:
        np.testing.assert_array_equal(tal["counts"][:7], counts)
        np.testing.assert_array_equal(tal["events"][:9], events)
        assert tal["t"] == t
    assert g["tally"]["t"] == pytest.approx(2e-4 + 1e-6 + 10.0, rel=1e-15)
    assert_fp64_parity(g, o, wl.L)
    # charge and atoms of everything injected, exactly, after 10 s of rate equations
    n_in = np.bincount(np.concatenate([p.types for p in pulses]), minlength=7)
    assert _totals(g["tally"]["counts"][:7], o.water) == _totals(n_in)


def test_due_species_join_the_stage_and_arrivals_inside_it_are_refused():
    wl = W.uniform_2000(seed=4, L=300.0, n_steps=10)
    cfg, keep = _config(wl, 4, chem.CHEM_FP64)
    ctx = chem.chem_init(cfg)
    o = sbs.from_workload(wl, seed=4)
    try:
        for p in wl.pulses:
            chem.chem_inject_pulse(ctx, p.types, p.xyz, p.t_arrival, p.energy_eV)
        chem.chem_run_homogeneous(ctx, 1e-3)  # straight from injection: all species are due
        e_ref, E_ref = o.run_homogeneous(1e-3)
        e, E, _ = chem.chem_batch_homogeneous_report(ctx, 0)
        _check_extents(e, E, e_ref, H.rounding_uniforms(9, 0, o.key))
        np.testing.assert_array_equal(E[:9], E_ref)
        before = chem.chem_tally(ctx, 7, 9)
        xyz = np.zeros((1, 3))
        chem.chem_inject_pulse(ctx, np.array([W.E_AQ], np.int32), xyz, np.array([5e-3]), 0.0)
        with pytest.raises(chem.ChemError) as err:
            chem.chem_run_homogeneous(ctx, 1e-2)
        assert err.value.status == chem.CHEM_EINVAL
        after = chem.chem_tally(ctx, 7, 9)
        np.testing.assert_array_equal(after["counts"], before["counts"])
        assert after["t"] == before["t"] == 1e-3
        chem.chem_run_homogeneous(ctx, 5e-3)  # up to the arrival is fine
        o.inject([W.E_AQ], xyz, [5e-3])
        o.run_homogeneous(5e-3)
        chem.chem_run_until(ctx, 5e-3 + 2e-8)
        o.run_until(5e-3 + 2e-8)
        np.testing.assert_array_equal(chem.chem_tally(ctx, 7, 9)["counts"][:7], o.counts())
        ids, types, pos = chem.chem_get_state(ctx)
        oi, ot, op = o.state()
        order = np.argsort(ids)
        np.testing.assert_array_equal(ids[order], oi)
        d = pos[order] - op
        d -= wl.L * np.round(d / wl.L)
        assert np.abs(d).max() <= 1e-12 * wl.L
    finally:
        chem.chem_destroy(ctx)


def test_batched_trains_take_their_own_stages():
    import torch
    wls = [W.uniform_2000(seed=20 + b, L=L, n_steps=20) for b, L in enumerate((300.0, 500.0, 800.0))]
    cfgs, keep = [], []
    for b, wl in enumerate(wls):
        c, k = _config(wl, 20 + b, chem.CHEM_FP64, train_id=b)
        cfgs.append(c)
        keep.append(k)
    ctx = chem.chem_batch_init(cfgs)
    ors = [sbs.from_workload(wl, seed=20 + b, train_id=b) for b, wl in enumerate(wls)]
    try:
        for b, wl in enumerate(wls):
            for p in wl.pulses:
                chem.chem_batch_inject(ctx, b, p.types, p.xyz, p.t_arrival, p.energy_eV)
        chem.chem_batch_run_until(ctx, [2e-8, 3e-8, 2e-8])
        for b, t in enumerate((2e-8, 3e-8, 2e-8)):
            ors[b].run_until(t)
        # train 1 stays where it is (end time not after its clock)
        ends = [1e-4, 3e-8, 1.0]
        chem.chem_batch_run_homogeneous(ctx, ends)
        for b in (0, 2):
            stage = ors[b].hx_stage
            e_ref, E_ref = ors[b].run_homogeneous(ends[b])
            e, E, _ = chem.chem_batch_homogeneous_report(ctx, b)
            _check_extents(e, E, e_ref, H.rounding_uniforms(9, stage, ors[b].key))
        chem.chem_batch_run_until(ctx, [1e-4 + 2e-8, 6e-8, 1.0 + 2e-8])
        for b, t in enumerate((1e-4 + 2e-8, 6e-8, 1.0 + 2e-8)):
            ors[b].run_until(t)
        for b, wl in enumerate(wls):
            tal = chem.chem_batch_tally(ctx, b, 7, 9)
            np.testing.assert_array_equal(tal["counts"][:7], ors[b].counts())
            np.testing.assert_array_equal(tal["events"][:9], ors[b].events_total)
            assert tal["t"] == ors[b].t and tal["species_steps"] == ors[b].species_steps
            ids, types, pos = chem.chem_batch_get_state(ctx, b)
            oi, ot, op = ors[b].state()
            order = np.argsort(ids)
            np.testing.assert_array_equal(ids[order], oi)
            np.testing.assert_array_equal(types[order], ot)
            d = pos[order] - op
            d -= wl.L * np.round(d / wl.L)
            assert np.abs(d).max() <= 1e-12 * wl.L
    finally:
        chem.chem_destroy(ctx)
    torch.cuda.synchronize()


def test_fp32_local_stage_conserves_and_counts_whole_events():
    pulses = W.pulse_train(2, 1e-4, 1e-6, n_tracks=8, L=800.0, species_per_track=200, seed=9)
    wl = W.Workload("hybrid2", 800.0, pulses,
                    W.Schedule(dt_min=1e-11, dt_max=1e-7, dt_growth=W.LOG_GROWTH_20_PER_DECADE),
                    t_end=0.0)
    cfg, keep = _config(wl, 9, chem.CHEM_FP32_LOCAL)
    ctx = chem.chem_init(cfg)
    nu = H.stoichiometry(7, W.WATER_REACTIONS)
    try:
        for p in wl.pulses:
            chem.chem_inject_pulse(ctx, p.types, p.xyz, p.t_arrival, p.energy_eV)
        n_in = np.bincount(np.concatenate([p.types for p in pulses]), minlength=7)
        water = 0
        for kind, t in W.hybrid_stages(2, 1e-4, 1e-6, tail_s=1.0):
            if kind == "sbs":
                chem.chem_run_until(ctx, t)
                continue
            before = chem.chem_tally(ctx, 7, 9)
            chem.chem_run_homogeneous(ctx, t)
            after = chem.chem_tally(ctx, 7, 9)
            e, E, steps = chem.chem_batch_homogeneous_report(ctx, 0)
            # rounding moves an extent by less than one event; take-backs only lower it
            assert np.all(E[:9] <= np.ceil(np.maximum(e[:9], 0.0)))
            assert np.all(E[:9] >= 0)
            np.testing.assert_array_equal(after["counts"][:7], before["counts"][:7] + nu @ E[:9])
            np.testing.assert_array_equal(after["events"][:9], before["events"][:9] + E[:9])
        # the tally's water balance is internal; charge needs none
        assert int(after["counts"][:7] @ W.CHARGE) == int(n_in @ W.CHARGE)
        ev = after["events"][:9]
        water = int(sum(ev[r] * rx.water_delta for r, rx in enumerate(W.WATER_REACTIONS)))
        assert _totals(after["counts"][:7], water) == _totals(n_in)
    finally:
        chem.chem_destroy(ctx)


def test_ten_second_tail_at_a_million_species():
    # the rate equations at the benchmark's species count: 1e6 species of the track mix
    # uniformly in a 5 um box, straight into a 10 s homogeneous stage
    counts = (W.MIX_COUNTS * (1_000_000 // W.MIX_COUNTS.sum())).astype(np.int64)
    L = 5000.0
    pulse = W.uniform_mixture(counts, L, seed=2)
    wl = W.Workload("mix1e6", L, [pulse], W.Schedule(1e-9, 1e-9), t_end=0.0)
    cfg, keep = _config(wl, 2, chem.CHEM_FP32_LOCAL, cap=2 * int(counts.sum()))
    ctx = chem.chem_init(cfg)
    try:
        chem.chem_inject_pulse(ctx, pulse.types, pulse.xyz, pulse.t_arrival, 0.0)
        chem.chem_run_homogeneous(ctx, 10.0)
        e, E, steps = chem.chem_batch_homogeneous_report(ctx, 0)
    finally:
        chem.chem_destroy(ctx)
    e_ref = H.extents(counts.astype(float), L, 10.0, W.WATER_REACTIONS)
    np.testing.assert_allclose(e[:9], e_ref, rtol=EXT_RTOL, atol=EXT_ATOL)
    assert 0 < steps < 5000


def test_pulse_train_driver_matches_reference_per_call():
    from paper_2509_03313_gb300 import hybrid
    specs = [(2, 1e-4, 500.0, 31), (3, 3e-5, 700.0, 32)]
    wls, plans, cfgs, keep = [], [], [], []
    for b, (n_p, period, L, seed) in enumerate(specs):
        pulses = W.pulse_train(n_p, period, 1e-6, n_tracks=4, L=L, species_per_track=100, seed=seed)
        wl = W.Workload(f"drv{b}", L, pulses,
                        W.Schedule(dt_min=1e-11, dt_max=1e-7, dt_growth=W.LOG_GROWTH_20_PER_DECADE),
                        t_end=0.0)
        wls.append(wl)
        plans.append(W.hybrid_stages(n_p, period, 1e-6, tail_s=0.5))
        c, k = _config(wl, seed, chem.CHEM_FP64, train_id=b)
        cfgs.append(c)
        keep.append(k)
    ctx = chem.chem_batch_init(cfgs)
    try:
        for b, wl in enumerate(wls):
            for p in wl.pulses:
                chem.chem_batch_inject(ctx, b, p.types, p.xyz, p.t_arrival, p.energy_eV)
        run = hybrid.run_plans(ctx, plans)
    finally:
        chem.chem_destroy(ctx)
    for b, (wl, plan) in enumerate(zip(wls, plans)):
        o = sbs.from_workload(wl, seed=specs[b][3], train_id=b)
        for i, (kind, t) in enumerate(plan):
            if kind == "sbs":
                o.run_until(t)
            else:
                o.run_homogeneous(t)
            np.testing.assert_array_equal(run["counts"][i, b], o.counts(), err_msg=f"train {b} call {i}")
            np.testing.assert_array_equal(run["events"][i, b], o.events_total)
            assert run["t"][i, b] == o.t
