"""FP64 mode of the CUDA library against the FP64 reference: identical event lists,
per-step species counts and integer tallies, positions within 1e-12 L.
Runs through the C ABI on the GPU."""
import numpy as np
import pytest

from harness import assert_fp64_parity, cuda_available, gpu_run, oracle_run
from paper_2509_03313_gb300 import chem, workloads as W

pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not cuda_available(), reason="needs a CUDA GPU")]


@pytest.mark.parametrize("seed", [1, 2])
def test_dense_mixture_200nm(seed):
    wl = W.uniform_2000(seed=seed, L=200.0, n_steps=300)
    g = gpu_run(wl, seed)
    o = oracle_run(wl, seed)
    assert o.events_total.sum() > 300
    assert_fp64_parity(g, o, wl.L)


def test_uniform_2000_1um_1000_steps():
    wl = W.uniform_2000(seed=3, L=1000.0, n_steps=1000)
    g = gpu_run(wl, 3)
    o = oracle_run(wl, 3)
    assert_fp64_parity(g, o, wl.L)


def test_tracks_with_log_steps_and_staggered_arrivals():
    # 12 tracks arriving over a 20 ns square pulse, log-growing dt with resets.
    pulse = W.track_pulse(12, 400.0, 300, seed=5, fwhm=20e-9)
    wl = W.Workload("tracks_small", 400.0, [pulse],
                    W.Schedule(dt_min=1e-12, dt_max=2e-9, dt_growth=W.LOG_GROWTH_20_PER_DECADE),
                    t_end=60e-9)
    g = gpu_run(wl, 11)
    o = oracle_run(wl, 11)
    assert o.events_total.sum() > 100
    assert_fp64_parity(g, o, wl.L)


def test_tracks_whole_trajectory_at_benchmark_density():
    # The benchmark's track workload in a 1.6 um box at its track and species density
    # (20 tracks, 32,000 species), every step from 1 ps to 1 us (about 150 log-growing
    # steps, more than 10,000 events): checked against the C++ reference.
    wl = W.tracks_same_density(21, 1600.0)
    g = gpu_run(wl, 21)
    o = oracle_run(wl, 21, impl="cxx")
    assert o.events_total.sum() > 10_000
    assert_fp64_parity(g, o, wl.L)


def test_run_until_in_chunks_equals_oracle_chunks():
    wl = W.uniform_2000(seed=4, L=200.0, n_steps=100)
    stops = [13e-9, 50e-9, 50e-9, 77.5e-9]
    g = gpu_run(wl, 4, t_stops=stops)
    o = oracle_run(wl, 4, t_stops=stops)
    assert_fp64_parity(g, o, wl.L)


def test_many_tiles_free_diffusion_positions():
    # 60k inert species (no reactions): the sort spans many tiles; positions after 40
    # steps match the reference's to 1e-12 L.
    rng = np.random.default_rng(9)
    L = 3000.0
    n = 60000
    types = rng.integers(0, 7, n).astype(np.int32)
    xyz = rng.uniform(-L / 2, L / 2, (n, 3))
    pulse = W.Pulse(types, xyz, np.zeros(n), 1e4)
    wl = W.Workload("free", L, [pulse], W.Schedule(dt_min=1e-9, dt_max=1e-9), t_end=40e-9,
                    reactions=[])
    g = gpu_run(wl, 21)
    o = oracle_run(wl, 21)
    assert_fp64_parity(g, o, L)


def test_empty_and_single_species():
    wl = W.Workload("empty", 100.0, [], W.Schedule(dt_min=1e-9, dt_max=1e-9), t_end=5e-9)
    g = gpu_run(wl, 1)
    assert g["tally"]["t"] == 5e-9 and g["tally"]["species_steps"] == 0
    one = W.Pulse(np.array([0], np.int32), np.array([[49.999, -50.0, 0.0]]), np.zeros(1), 1.0)
    wl = W.Workload("one", 100.0, [one], W.Schedule(dt_min=1e-9, dt_max=1e-9), t_end=20e-9)
    g = gpu_run(wl, 2)
    o = oracle_run(wl, 2)
    assert_fp64_parity(g, o, wl.L)


@pytest.mark.parametrize("spl", [1, 3])
def test_steps_per_launch_does_not_change_results(spl):
    wl = W.uniform_2000(seed=6, L=200.0, n_steps=40)
    g = gpu_run(wl, 6, steps_per_launch=spl)
    o = oracle_run(wl, 6)
    assert_fp64_parity(g, o, wl.L)
