"""The two FP64 references against each other: the plain C++ program (``oracle.cxx``)
and the numpy one (``oracle.sbs``) written independently from the same passages (Sec.
2.1 workflow, Eq. 1, Eq. 2, Sec. 2.4 with Table 1). On every workload kind of the
benchmark (dense uniform mixture, log-growing steps on tracks, pulses spread over a
square pulse with releases that restart the step, the free-diffusion jump, Table S1
first products) they must give the same event list, the same per-step record and the
same tallies bit for bit, and positions that differ only by the last bits of the
host's exp/log/sin/cos."""
import numpy as np
import pytest

from oracle import cxx, sbs
from paper_2509_03313_gb300 import physchem, workloads as W


def _compare(wl, seed, t_stops=None, pos_atol=1e-9):
    a = sbs.from_workload(wl, seed=seed)
    b = cxx.from_workload(wl, seed=seed)
    for t in (t_stops or [wl.t_end]):
        na, nb = a.run_until(t), b.run_until(t)
        assert na == nb
        np.testing.assert_array_equal(a.counts(), b.counts())
    ea, eb = a.events(), b.events()
    assert ea.shape == eb.shape
    np.testing.assert_array_equal(ea, eb)
    np.testing.assert_array_equal(a.steps(), b.steps())
    la, lb = a.step_log, b.step_log
    assert len(la) == len(lb)
    # step start times and step lengths are the same arithmetic on both sides
    np.testing.assert_array_equal(np.array([s[1:3] for s in la]), np.array([s[1:3] for s in lb]))
    assert a.species_steps == b.species_steps and a.water == b.water and a.E_dep == b.E_dep
    np.testing.assert_array_equal(a.events_total, b.events_total)
    ia, ta, pa = a.state()
    ib, tb, pb = b.state()
    np.testing.assert_array_equal(ia, ib)
    np.testing.assert_array_equal(ta, tb)
    np.testing.assert_allclose(pa, pb, rtol=0, atol=pos_atol)
    assert a.t == b.t
    return ea


@pytest.mark.parametrize("seed", [3, 4])
def test_dense_uniform_mixture(seed):
    ev = _compare(W.uniform_2000(seed=seed, L=200.0, n_steps=300), seed, [100e-9, 300e-9])
    assert ev.shape[0] > 500


def test_tracks_log_growing_steps():
    wl = W.tracks_same_density(5, 600.0, t_end=2e-7)
    ev = _compare(wl, 5)
    assert ev.shape[0] > 200


def test_square_pulses_with_releases():
    wl = W.multi_pulse(6, n_pulses=3, period_s=30e-9, fwhm_s=8e-9, n_tracks=4, species_per_track=250,
                       L=400.0, dt_min=1e-11, dt_max=2e-9)
    ev = _compare(wl, 6, [10e-9, 45e-9, wl.t_end])
    assert ev.shape[0] > 50


def test_free_diffusion_jump():
    wl = W.uniform_2000(seed=8, L=300.0, n_steps=50)
    wl.schedule.sbs_horizon = 20e-9
    wl.pulses.append(W.uniform_mixture([50, 50, 0, 50, 0, 0, 0], wl.L, 9, t_arrival=200e-9))
    wl.t_end = 260e-9
    _compare(wl, 8, [120e-9, wl.t_end])


def test_table_s1_first_products():
    pulse, _ = physchem.physchem_pulse(3, 300.0, 400, seed=10)
    wl = W.Workload("physchem", 300.0, [pulse],
                    W.Schedule(dt_min=1e-12, dt_max=1e-8, dt_growth=W.LOG_GROWTH_20_PER_DECADE), t_end=1e-7)
    ev = _compare(wl, 10)
    assert ev.shape[0] > 50


def test_building_blocks_agree_elementwise():
    rng = np.random.default_rng(1)
    key = sbs.philox_key(2 ** 40 + 77, 5)
    assert cxx.philox_key(2 ** 40 + 77, 5) == key
    ids = rng.integers(0, 2 ** 31, 5000)
    np.testing.assert_allclose(cxx.gaussians(ids, 12, key), sbs.gaussians(ids, 12, key), rtol=1e-13, atol=1e-14)
    lo, hi = ids[:2500], ids[2500:]
    np.testing.assert_array_equal(cxx.acceptance_uniform(lo, hi, 3, key), sbs.acceptance_uniform(lo, hi, 3, key))
    x = rng.uniform(-40, 40, 5000)
    np.testing.assert_array_equal(cxx.wrap(x, 10.0), sbs.wrap(x, 10.0))
    dx = rng.uniform(-10, 10, 5000)
    np.testing.assert_array_equal(cxx.minimum_image(dx, 10.0), sbs.minimum_image(dx, 10.0))
    d0, d1 = rng.uniform(0.1, 5, 5000), rng.uniform(0.1, 5, 5000)
    np.testing.assert_allclose(cxx.touch_probability(d0, d1, 0.5, 1.3), sbs.touch_probability(d0, d1, 0.5, 1.3),
                               rtol=1e-13, atol=1e-300)
    for k, D in ((1.1e10, 14.6e9), (0.95e10, 4.4e9)):
        assert cxx.reaction_radius(k, D) == sbs.reaction_radius(k, D)


@pytest.mark.parametrize("ref", ["numpy", "cxx"])
def test_bad_inputs_raise(ref):
    mod = cxx if ref == "cxx" else sbs
    o = mod.SBSOracle(W.D_NM2_S, W.WATER_REACTIONS, 100.0, seed=1)
    with pytest.raises(ValueError):
        o.inject([7], [[0.0, 0.0, 0.0]], [0.0])           # no type 7
    with pytest.raises(ValueError):
        o.inject([0], [[50.0, 0.0, 0.0]], [0.0])          # x = L/2 is outside [-L/2, L/2)
    with pytest.raises(ValueError):
        o.inject([0], [[0.0, 0.0, 0.0]], [float("nan")])  # arrival not a number
    with pytest.raises(ValueError):
        o.inject([0], [[float("nan"), 0.0, 0.0]], [0.0])  # position not a number
    o.run_until(2e-9)
    with pytest.raises(ValueError):
        o.inject([0], [[0.0, 0.0, 0.0]], [1e-9])          # arrival in the past
    assert o.n_types == 7 and o.counts().sum() == 0
    with pytest.raises(ValueError):                       # two reactions for one type pair
        mod.SBSOracle([1e9, 1e9], [(0, 1, 1e10, (), 0), (1, 0, 2e10, (), 0)], 100.0, seed=1)
    with pytest.raises(ValueError):                       # R >= L/3
        mod.SBSOracle([1e9, 1e9], [(0, 1, 1e13, (), 0)], 30.0, seed=1)


def test_max_steps_stops_early():
    wl = W.uniform_2000(seed=2, L=200.0, n_steps=40)
    a = sbs.from_workload(wl, seed=2)
    b = cxx.from_workload(wl, seed=2)
    assert a.run_until(wl.t_end, max_steps=7) == b.run_until(wl.t_end, max_steps=7) == 7
    assert a.t == b.t and a.step == b.step == 7
    np.testing.assert_array_equal(a.events(), b.events())
