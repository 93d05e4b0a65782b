"""The synthetic inputs follow their stated recipes: species counts, box sizes, energies
(about 1 Gy per pulse where the recipe says so, 1 Gy = 1 J/kg of water at 1 kg/L),
arrival times inside the pulses, positions inside the box, and seeded reproducibility."""
import numpy as np
import pytest

from paper_2509_03313_gb300 import workloads as W

EV = 1.602176634e-19


def _dose_Gy(energy_eV, L_nm):
    return energy_eV * EV / (L_nm ** 3 * 1e-24)  # J per kg (1 L of water = 1 kg)


def _in_box(p, L):
    return np.all(p.xyz >= -0.5 * L) and np.all(p.xyz < 0.5 * L)


def test_large_build_up_recipe():
    wl = W.large_build_up(seed=1, n_pulses=3)
    assert wl.L == 10000.0 and len(wl.pulses) == 3 * 4
    per_pulse = sum(p.n for p in wl.pulses[:4])
    assert abs(per_pulse - 375_000) < 375_000 * 0.01
    dose = _dose_Gy(sum(p.energy_eV for p in wl.pulses[:4]), wl.L)
    assert 0.95 < dose < 1.05
    for k in range(3):
        t = np.concatenate([p.t_arrival for p in wl.pulses[4 * k:4 * k + 4]])
        assert t.min() == pytest.approx(k * 10e-6) and t.max() < k * 10e-6 + 1e-6
    assert all(_in_box(p, wl.L) for p in wl.pulses)
    assert wl.t_end == pytest.approx(30e-6)


def test_dose_series_recipe():
    wls, plans, meta = W.dose_series()
    assert [m["n_pulses"] for m in meta] == [1, 5, 10, 15, 20] * 2
    for wl, plan, m in zip(wls, plans, meta):
        per_pulse = wl.n_species / m["n_pulses"]
        assert abs(per_pulse - 1e5) < 2e3  # whole tracks of whole species
        dose = _dose_Gy(sum(p.energy_eV for p in wl.pulses), wl.L) / m["n_pulses"]
        assert 0.9 < dose < 1.1
        assert [k for k, _ in plan] == ["sbs", "ode"] * m["n_pulses"]
        assert plan[-1][1] == pytest.approx((m["n_pulses"] - 1) * m["period_s"] + 1e-6 + 10.0)
        assert m["period_s"] == pytest.approx(1.0 / m["avg_dose_rate"])  # 1 Gy per pulse


def test_hybrid_sweep_matches_the_dose_rate_sweep():
    wls, plans = W.hybrid_sweep(n_trains=8, scale=0.05)
    descs = W.dose_rate_sweep(n_trains=8, n_min=500, n_max=100_000)
    assert len(wls) == len(plans) == 8
    for wl, plan, d in zip(wls, plans, descs):
        assert wl.L == pytest.approx(d["L"])
        t = np.concatenate([p.t_arrival for p in wl.pulses])
        starts = np.arange(d["n_pulses"]) * d["period_s"]
        # every arrival inside a beam-on window, every window used
        k = np.floor(t / d["period_s"] + 1e-9).astype(int)
        assert np.all(t - starts[k] < 1e-6 + 1e-12) and set(k) == set(range(d["n_pulses"]))
        assert [kind for kind, _ in plan] == ["sbs", "ode"] * d["n_pulses"]


def test_volume_scaling_keeps_one_concentration():
    counts = [np.bincount(W.volume_scaling(L, seed=1).pulses[0].types, minlength=7)
              for L in (200.0, 500.0, 1000.0)]
    conc = [c / L ** 3 for c, L in zip(counts, (200.0, 500.0, 1000.0))]
    np.testing.assert_allclose(conc[1], conc[0], rtol=1e-3)
    np.testing.assert_allclose(conc[2], conc[0], rtol=1e-3)
    assert counts[0].tolist() == W.MIX_COUNTS.tolist()


def test_inputs_are_reproducible_from_their_seed():
    a = W.large_build_up(seed=4, n_pulses=1)
    b = W.large_build_up(seed=4, n_pulses=1)
    c = W.large_build_up(seed=5, n_pulses=1)
    np.testing.assert_array_equal(a.pulses[0].xyz, b.pulses[0].xyz)
    assert not np.array_equal(a.pulses[0].xyz, c.pulses[0].xyz)
