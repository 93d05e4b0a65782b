"""The library's tallies (chem_tally) on the hand-computed cases that pin the reference's:
G-values as molecules per 100 eV of deposited energy (Sec. 1) and the species-step count
on schedules with known sums, in both precisions. Runs through the C ABI on the GPU."""
import numpy as np
import pytest

from harness import cuda_available
from paper_2509_03313_gb300 import chem, workloads as W

pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not cuda_available(), reason="needs a CUDA GPU")]


def _ctx(D, reactions, L, dt, growth=1.0, dt_max=None, precision=chem.CHEM_FP64):
    import torch
    cfg, keep = chem.make_config(L, D, reactions, seed=1, precision=precision, dt_min=dt,
                                 dt_max=dt_max or dt, dt_growth=growth, capacity_species=64, capacity_step_log=64,
                                 stream=torch.cuda.current_stream().cuda_stream)
    return chem.chem_init(cfg), keep


@pytest.mark.parametrize("precision", [chem.CHEM_FP64, chem.CHEM_FP32_LOCAL])
def test_g_values_and_species_steps_hand_computed(precision):
    ctx, keep = _ctx([1e9, 2e9], [], 100.0, 1e-9, precision=precision)
    try:
        chem.chem_inject_pulse(ctx, np.array([0, 0, 1], np.int32), np.zeros((3, 3)), np.zeros(3), 150.0)
        chem.chem_inject_pulse(ctx, np.array([1, 1], np.int32), np.full((2, 3), 10.0),
                               np.full(2, 2.5e-9), 50.0)
        chem.chem_run_until(ctx, 5e-9)
        tal = chem.chem_tally(ctx, 2, 0)
    finally:
        chem.chem_destroy(ctx)
    assert np.array_equal(tal["counts"], [2, 3])
    np.testing.assert_allclose(tal["G"], [1.0, 1.5], rtol=1e-15)
    assert tal["species_steps"] == 19 and tal["t"] == 5e-9


def test_species_steps_on_geometric_steps():
    ctx, keep = _ctx([1e9, 2e9], [], 100.0, 1e-9, growth=2.0, dt_max=8e-9)
    try:
        chem.chem_inject_pulse(ctx, np.array([0, 1, 1, 0], np.int32), np.zeros((4, 3)), np.zeros(4), 1.0)
        chem.chem_run_until(ctx, 20e-9)
        tal = chem.chem_tally(ctx, 2, 0)
        steps = chem.chem_get_step_log(ctx)
    finally:
        chem.chem_destroy(ctx)
    assert tal["species_steps"] == 20 and tal["t"] == 20e-9
    np.testing.assert_allclose(steps["dt_s"], [1e-9, 2e-9, 4e-9, 8e-9, 5e-9], rtol=1e-14)


def test_g_after_one_reaction():
    ctx, keep = _ctx(W.D_NM2_S, W.WATER_REACTIONS, 100.0, 1e-12)
    try:
        chem.chem_inject_pulse(ctx, np.array([W.E_AQ, W.OH], np.int32), np.zeros((2, 3)), np.zeros(2), 100.0)
        chem.chem_run_until(ctx, 1e-12)
        tal = chem.chem_tally(ctx, 7, 9)
    finally:
        chem.chem_destroy(ctx)
    assert tal["events"][1] == 1
    assert tal["G"][W.OHM] == 1.0 and tal["G"][W.E_AQ] == 0.0 and tal["G"][W.OH] == 0.0
