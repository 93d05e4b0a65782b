"""Failure detection without a GPU fault: a bounded device wait that runs out comes back
as CHEM_ETIMEOUT, sticky on its context, and the GPU stays usable for the next context."""
import time

import numpy as np
import pytest

from harness import assert_fp64_parity, gpu_run, oracle_run
from paper_2509_03313_gb300 import chem, workloads as W

pytestmark = pytest.mark.gpu


def _ctx():
    import torch
    wl = W.uniform_2000(seed=3, L=400.0, n_steps=20)
    cfg, keep = chem.make_config(wl.L, wl.D, wl.reactions, seed=3, capacity_species=8192,
                                 stream=torch.cuda.current_stream().cuda_stream,
                                 allocator=chem.torch_allocator(0))
    return chem.chem_init(cfg), keep, wl


def test_bounded_wait_runs_out_with_a_status_and_the_gpu_stays_usable():
    ctx, keep, wl = _ctx()
    try:
        for p in wl.pulses:
            chem.chem_inject_pulse(ctx, p.types, p.xyz, p.t_arrival, p.energy_eV)
        t0 = time.perf_counter()
        with pytest.raises(chem.ChemError) as err:
            chem.chem_check_bounded_wait(ctx, 0.2)
        waited = time.perf_counter() - t0
        assert err.value.status == chem.CHEM_ETIMEOUT
        assert 0.15 < waited < 10.0
        with pytest.raises(chem.ChemError) as err:  # sticky: the context only reports it
            chem.chem_run_until(ctx, 1e-8)
        assert err.value.status == chem.CHEM_ETIMEOUT
    finally:
        chem.chem_destroy(ctx)
    # a new context on the same GPU runs and matches the reference
    g = gpu_run(wl, 3)
    o = oracle_run(wl, 3)
    assert_fp64_parity(g, o, wl.L)


def test_bounded_wait_limit_is_checked():
    ctx, keep, wl = _ctx()
    try:
        for bad in (0.0, -1.0, 11.0, float("nan")):
            with pytest.raises(chem.ChemError) as err:
                chem.chem_check_bounded_wait(ctx, bad)
            assert err.value.status == chem.CHEM_EINVAL
        chem.chem_run_until(ctx, 0.0)  # not sticky: the context is still fine
    finally:
        chem.chem_destroy(ctx)


def test_bad_inputs_are_refused_and_leave_the_context_usable():
    ctx, keep, wl = _ctx()
    try:
        p = wl.pulses[0]
        good_t = p.t_arrival.copy()
        for types, xyz, t in (
                (p.types, p.xyz, np.where(np.arange(p.n) == 5, np.nan, good_t)),      # NaN arrival
                (p.types, p.xyz, good_t - 1e-9),                                      # before the clock
                (p.types, np.where(np.arange(3 * p.n).reshape(-1, 3) == 7, wl.L, p.xyz), good_t),  # outside
                (np.where(np.arange(p.n) == 3, 7, p.types).astype(np.int32), p.xyz, good_t)):     # bad type
            with pytest.raises(chem.ChemError) as err:
                chem.chem_inject_pulse(ctx, types, xyz, t, p.energy_eV)
            assert err.value.status == chem.CHEM_EINVAL
        chem.chem_inject_pulse(ctx, p.types, p.xyz, p.t_arrival, p.energy_eV)  # still fine
        chem.chem_run_until(ctx, 2e-9)
        assert chem.chem_tally(ctx, 7, 9)["counts"][:7].sum() > 0
    finally:
        chem.chem_destroy(ctx)


def test_species_capacity_overflow_is_a_sticky_status():
    import torch
    wl = W.uniform_2000(seed=3, L=400.0, n_steps=20)
    cfg, keep = chem.make_config(wl.L, wl.D, wl.reactions, seed=3, capacity_species=1000,
                                 capacity_pending=4096, stream=torch.cuda.current_stream().cuda_stream,
                                 allocator=chem.torch_allocator(0))
    ctx = chem.chem_init(cfg)
    try:
        p = wl.pulses[0]
        chem.chem_inject_pulse(ctx, p.types, p.xyz, p.t_arrival, p.energy_eV)  # 2,000 > 1,000 slots
        with pytest.raises(chem.ChemError) as err:
            chem.chem_run_until(ctx, 1e-8)
        assert err.value.status == chem.CHEM_ECAPACITY
        with pytest.raises(chem.ChemError) as err:
            chem.chem_run_until(ctx, 2e-8)
        assert err.value.status == chem.CHEM_ECAPACITY
    finally:
        chem.chem_destroy(ctx)
