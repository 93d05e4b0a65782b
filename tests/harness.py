"""Helpers that run one workload through the CUDA library (via its C ABI) and through
the FP64 reference, and compare them."""
import numpy as np

from paper_2509_03313_gb300 import chem, workloads as W


def cuda_available():
    try:
        import torch
        return torch.cuda.is_available()
    except Exception:  # noqa: BLE001
        return False


def gpu_run(wl, seed, precision=chem.CHEM_FP64, t_end=None, capacity=None, record=True,
            steps_per_launch=0, cells_per_axis_max=0, train_id=0, t_stops=None,
            launch_mode=chem.CHEM_LAUNCH_AUTO, tuning=None):
    import torch
    s = wl.schedule
    n = wl.n_species
    cap = capacity or max(4096, 2 * n)
    cfg, keep = chem.make_config(
        wl.L, wl.D, wl.reactions, seed=seed, train_id=train_id, precision=precision,
        dt_min=s.dt_min, dt_max=s.dt_max, dt_growth=s.dt_growth, reset_on_release=s.reset_on_release,
        cutoff_c=s.cutoff_c, sbs_horizon=s.sbs_horizon, capacity_species=cap,
        capacity_pending=max(n, 1), capacity_candidates=max(4096, cap // 2),
        capacity_event_log=(4 * n + 1024) if record else 0,
        capacity_step_log=200000 if record else 0, steps_per_launch=steps_per_launch,
        cells_per_axis_max=cells_per_axis_max, launch_mode=launch_mode,
        stream=torch.cuda.current_stream().cuda_stream, allocator=chem.torch_allocator(0))
    ctx = chem.chem_init(cfg)
    out = {}
    try:
        if tuning is not None:
            chem.chem_set_tuning(ctx, *tuning)
        for p in wl.pulses:
            chem.chem_inject_pulse(ctx, p.types, p.xyz, p.t_arrival, p.energy_eV)
        stops = list(t_stops or []) + [t_end if t_end is not None else wl.t_end]
        tallies = []
        for t in stops:
            chem.chem_run_until(ctx, t)
            tallies.append(chem.chem_tally(ctx, wl.n_types, len(wl.reactions)))
        out["tally"] = tallies[-1]
        out["tallies"] = tallies
        ids, types, xyz = chem.chem_get_state(ctx)
        o = np.argsort(ids)
        out["state"] = (ids[o].astype(np.int64), types[o].astype(np.int64), xyz[o])
        if record:
            out["events"] = chem.chem_get_events(ctx)
            out["steps"] = chem.chem_get_step_log(ctx)
        out["stats"] = chem.chem_get_stats(ctx)
    finally:
        chem.chem_destroy(ctx)
    return out


def oracle_run(wl, seed, t_end=None, train_id=0, t_stops=None, impl="numpy"):
    """The FP64 reference on a workload: the numpy one, or the plain C++ program
    (impl="cxx") for the larger cases."""
    if impl == "cxx":
        from oracle import cxx as ref
    else:
        from oracle import sbs as ref
    o = ref.from_workload(wl, seed=seed, train_id=train_id)
    stops = list(t_stops or []) + [t_end if t_end is not None else wl.t_end]
    counts = []
    for t in stops:
        o.run_until(t)
        counts.append(o.counts())
    o.stop_counts = counts
    return o


def event_matrix(ev):
    return np.stack([ev["step"], ev["rxn"], ev["id_lo"], ev["id_hi"], ev["prod_id0"],
                     ev["n_prod"]], 1).astype(np.int64)


def step_matrix(st, n_types):
    return np.concatenate([np.stack([st["step"], st["n_live"], st["n_events"]], 1),
                           st["counts"][:, :n_types]], 1).astype(np.int64)


def assert_fp64_parity(g, o, L, pos_tol_rel=1e-12):
    """Identical event lists, per-step counts and tallies; positions within
    pos_tol_rel * L under the minimum image."""
    oev = o.events()
    gev = event_matrix(g["events"])
    assert gev.shape == oev.shape, (gev.shape, oev.shape)
    if gev.size:
        bad = np.nonzero(np.any(gev != oev, axis=1))[0]
        assert bad.size == 0, f"first differing event {bad[0]}: gpu {gev[bad[0]]} oracle {oev[bad[0]]}"
    ost = o.steps()
    gst = step_matrix(g["steps"], o.n_types)
    assert gst.shape == ost.shape, (gst.shape, ost.shape)
    assert np.array_equal(gst, ost)
    # per-step clock
    t_o = np.array([s[1] for s in o.step_log])
    dt_o = np.array([s[2] for s in o.step_log])
    for name, got, ref in (("t_start", g["steps"]["t_start_s"], t_o), ("dt", g["steps"]["dt_s"], dt_o)):
        bad = np.nonzero(got != ref)[0]
        assert bad.size == 0, (f"{name} differs at step {bad[0]} of {got.size}: "
                               f"gpu {got[bad[0]]!r} oracle {ref[bad[0]]!r}")
    tal = g["tally"]
    assert np.array_equal(tal["counts"], o.counts())
    assert np.array_equal(tal["events"], o.events_total)
    assert tal["species_steps"] == o.species_steps
    assert tal["t"] == o.t
    gi, gt, gx = g["state"]
    oi, ot, ox = o.state()
    assert np.array_equal(gi, oi) and np.array_equal(gt, ot)
    if gx.size:
        d = gx - ox
        d = d - L * np.round(d / L)
        assert np.abs(d).max() <= pos_tol_rel * L, np.abs(d).max()


def gpu_batch_run(wls, seeds, train_ids=None, precision=chem.CHEM_FP64, record=True,
                  launch_mode=chem.CHEM_LAUNCH_AUTO, steps_per_launch=0, t_end=None, stats=None):
    """Run several trains in one batched context; returns one result dict per train
    (and fills the dict ``stats`` with the context's counters when given)."""
    import torch
    train_ids = train_ids or list(range(len(wls)))
    cfgs, keep = [], []
    for wl, seed, tid in zip(wls, seeds, train_ids):
        s = wl.schedule
        n = wl.n_species
        cap = max(4096, 2 * n)
        cfg, k = chem.make_config(
            wl.L, wl.D, wl.reactions, seed=seed, train_id=tid, precision=precision,
            dt_min=s.dt_min, dt_max=s.dt_max, dt_growth=s.dt_growth,
            reset_on_release=s.reset_on_release, cutoff_c=s.cutoff_c, sbs_horizon=s.sbs_horizon,
            capacity_species=cap, capacity_pending=max(n, 1), capacity_candidates=max(4096, cap // 2),
            capacity_event_log=(4 * n + 1024) if record else 0,
            capacity_step_log=200000 if record else 0, steps_per_launch=steps_per_launch,
            launch_mode=launch_mode, stream=torch.cuda.current_stream().cuda_stream,
            allocator=chem.torch_allocator(0))
        cfgs.append(cfg)
        keep.append(k)
    ctx = chem.chem_batch_init(cfgs)
    outs = []
    try:
        for b, wl in enumerate(wls):
            for p in wl.pulses:
                chem.chem_batch_inject(ctx, b, p.types, p.xyz, p.t_arrival, p.energy_eV)
        ends = [t_end if t_end is not None else wl.t_end for wl in wls]
        chem.chem_batch_run_until(ctx, ends)
        ev = chem.chem_get_events(ctx) if record else None
        st = chem.chem_get_step_log(ctx) if record else None
        for b, wl in enumerate(wls):
            o = {"tally": chem.chem_batch_tally(ctx, b, wl.n_types, len(wl.reactions))}
            ids, types, xyz = chem.chem_batch_get_state(ctx, b)
            order = np.argsort(ids)
            o["state"] = (ids[order].astype(np.int64), types[order].astype(np.int64), xyz[order])
            if record:
                o["events"] = ev[ev["train"] == b]
                o["steps"] = st[st["train"] == b]
            outs.append(o)
        if stats is not None:
            stats.update(chem.chem_get_stats(ctx))
    finally:
        chem.chem_destroy(ctx)
    return outs
