"""Both pair-search kernels (cell tiles: one warp per work item of up to 32 species of a
cell; one thread per home species) visit the same unordered pairs: FP64 runs with either
must reproduce the FP64 reference exactly, and FP32-local runs with either must give
identical results."""
import numpy as np
import pytest

from harness import assert_fp64_parity, cuda_available, gpu_run, oracle_run
from paper_2509_03313_gb300 import chem, workloads as W

pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not cuda_available(), reason="needs a CUDA GPU")]

PH, PE = chem.CHEM_LAUNCH_PHASES, chem.CHEM_LAUNCH_PERSISTENT
# (steps per launch, hash limit, species per item (0 = thread per species), launch form)
TUNINGS = {"tps": (8, 512, 0, PH), "tps_persistent": (4, 512, 0, PE), "items16": (8, 512, 16, PH),
           "items32": (8, 512, 32, PH), "items32_persistent": (4, 512, 32, PE), "items7": (8, 512, 7, PH),
           "tps_coarse": (8, 6, 0, PH), "items_coarse": (8, 6, 32, PH), "adaptive": (8, 512, -1, PH),
           "adaptive_persistent": (4, 512, -1, PE)}


def _tracks(seed):
    pulse = W.track_pulse(12, 600.0, 500, seed=seed)
    return W.Workload("tracks_s", 600.0, [pulse],
                      W.Schedule(dt_min=1e-12, dt_max=1e-7, dt_growth=W.LOG_GROWTH_20_PER_DECADE),
                      t_end=1e-7)


@pytest.mark.parametrize("name", sorted(TUNINGS))
def test_fp64_dense_mixture_equals_reference(name):
    wl = W.uniform_2000(seed=61, L=200.0, n_steps=150)
    g = gpu_run(wl, 61, tuning=TUNINGS[name])
    assert_fp64_parity(g, oracle_run(wl, 61), wl.L)


@pytest.mark.parametrize("name", ["tps", "tps_persistent", "items32", "items32_persistent", "adaptive",
                                  "adaptive_persistent"])
def test_fp64_tracks_equal_reference(name):
    wl = _tracks(62)
    g = gpu_run(wl, 62, tuning=TUNINGS[name])
    assert_fp64_parity(g, oracle_run(wl, 62), wl.L)
    st = g["stats"]
    if TUNINGS[name][2] < 0:  # chosen per step: both mappings ran (early steps: one thread per species)
        assert 0 < st["steps_cell_tiles"] < st["steps_advanced"], st
    else:
        assert st["steps_cell_tiles"] == (st["steps_advanced"] if TUNINGS[name][2] > 0 else 0), st


def test_fp32_local_kernels_give_identical_results():
    wl = _tracks(63)
    runs = [gpu_run(wl, 63, precision=chem.CHEM_FP32_LOCAL, tuning=t)
            for t in [(8, 512, 0, PH), (8, 512, 32, PH), (8, 512, 7, PH), (8, 512, 0, PE), (8, 512, 32, PE),
                      (8, 512, -1, PH), (4, 512, -1, PE)]]
    ref = runs[0]
    for g in runs[1:]:
        assert np.array_equal(g["tally"]["counts"], ref["tally"]["counts"])
        assert np.array_equal(g["tally"]["events"], ref["tally"]["events"])
        for k in ("step", "rxn", "id_lo", "id_hi", "prod_id0"):
            assert np.array_equal(g["events"][k], ref["events"][k])
        assert np.array_equal(g["state"][0], ref["state"][0])
        assert np.array_equal(g["state"][2], ref["state"][2])
