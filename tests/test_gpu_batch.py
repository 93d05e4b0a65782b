"""Batched trains (one hash for all trains, one persistent cooperative launch per graph
replay) against the FP64 reference per train, and FP32-local batches against
independent single-train runs."""
import numpy as np
import pytest

from harness import assert_fp64_parity, cuda_available, gpu_batch_run, gpu_run, oracle_run
from paper_2509_03313_gb300 import chem, workloads as W

pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not cuda_available(), reason="needs a CUDA GPU")]


def _mixed_trains():
    wls = [W.uniform_2000(seed=21, L=200.0, n_steps=120),
           W.uniform_2000(seed=22, L=300.0, n_steps=90)]
    pulse = W.track_pulse(8, 400.0, 250, seed=23, fwhm=10e-9)
    wls.append(W.Workload("tracks_b", 400.0, [pulse],
                          W.Schedule(dt_min=1e-12, dt_max=2e-9, dt_growth=W.LOG_GROWTH_20_PER_DECADE),
                          t_end=40e-9))
    return wls


def test_fp64_batch_equals_reference_per_train():
    wls = _mixed_trains()
    seeds, tids = [5, 6, 7], [0, 1, 2]
    outs = gpu_batch_run(wls, seeds, tids)
    for wl, s, tid, g in zip(wls, seeds, tids, outs):
        o = oracle_run(wl, s, train_id=tid)
        assert o.events_total.sum() > 50
        assert_fp64_parity(g, o, wl.L)


@pytest.mark.parametrize("mode", [chem.CHEM_LAUNCH_PHASES, chem.CHEM_LAUNCH_PERSISTENT])
def test_fp32_local_batch_equals_single_train_runs(mode):
    wls = _mixed_trains()
    seeds, tids = [8, 9, 10], [3, 4, 5]
    outs = gpu_batch_run(wls, seeds, tids, precision=chem.CHEM_FP32_LOCAL, launch_mode=mode)
    for wl, s, tid, g in zip(wls, seeds, tids, outs):
        single = gpu_run(wl, s, precision=chem.CHEM_FP32_LOCAL, train_id=tid)
        gi, gt, gx = g["state"]
        si, st, sx = single["state"]
        assert np.array_equal(gi, si) and np.array_equal(gt, st)
        assert np.array_equal(gx, sx)
        assert np.array_equal(g["tally"]["counts"], single["tally"]["counts"])
        assert np.array_equal(g["tally"]["events"], single["tally"]["events"])


def test_persistent_launch_single_train_matches_reference():
    wl = W.uniform_2000(seed=31, L=200.0, n_steps=150)
    g = gpu_run(wl, 31, launch_mode=chem.CHEM_LAUNCH_PERSISTENT)
    o = oracle_run(wl, 31)
    assert_fp64_parity(g, o, wl.L)


def test_trains_with_different_end_times():
    wls = _mixed_trains()
    ends = [30e-9, 60e-9, 20e-9]
    for b, wl in enumerate(wls):
        wl.t_end = ends[b]
    outs = gpu_batch_run(wls, [1, 2, 3], [0, 1, 2])
    for wl, g, s, b in zip(wls, outs, [1, 2, 3], range(3)):
        assert g["tally"]["t"] == ends[b]
        o = oracle_run(wl, s, train_id=b)
        assert_fp64_parity(g, o, wl.L)


def test_multi_pulse_with_free_diffusion_horizon():
    # Two pulses 2 us apart; after 200 ns without a release the train jumps by free
    # diffusion to the next arrival (and at the end), as in the reference.
    pulses = W.pulse_train(2, 2e-6, 20e-9, 6, 400.0, 200, seed=41)
    wl = W.Workload("two_pulses", 400.0, pulses,
                    W.Schedule(dt_min=1e-11, dt_max=5e-9, dt_growth=W.LOG_GROWTH_20_PER_DECADE,
                               sbs_horizon=200e-9),
                    t_end=5e-6)
    g = gpu_run(wl, 43)
    o = oracle_run(wl, 43)
    assert o.events_total.sum() > 50
    assert_fp64_parity(g, o, wl.L)
