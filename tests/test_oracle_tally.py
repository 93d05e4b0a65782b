"""Pins of the references' tallies (numpy and C++, through the ``impl`` fixture): the
G-value and the species-step count.

G is the number of molecules per 100 eV of deposited energy (Sec. 1, radiation chemical
yield). The pins are hand-computed cases and the SI unit conversion to mol/J, so that a
dropped factor 100, an energy taken in keV, or an injection whose energy is not summed
fails here. The species-step count (the benchmark's unit) is pinned on a schedule whose
sum is known in closed form."""
import math

import numpy as np

from paper_2509_03313_gb300 import workloads as W

E_CHARGE = 1.602176634e-19   # J per eV (exact SI)
N_A = 6.02214076e23          # 1/mol (exact SI)


def _inert(impl, L=100.0, dt=1e-9, growth=1.0, dt_max=None):
    # two species types, no reactions
    return impl.SBSOracle([1e9, 2e9], [], L, seed=1, dt_min=dt, dt_max=dt_max or dt, dt_growth=growth,
                         record=False)


def test_g_values_hand_computed(impl):
    o = _inert(impl)
    assert np.array_equal(o.g_values(), [0.0, 0.0])  # no energy deposited yet
    o.inject([0, 0, 1], np.zeros((3, 3)), np.zeros(3), energy_eV=150.0)
    o.inject([1, 1], np.full((2, 3), 10.0), np.full(2, 2.5e-9), energy_eV=50.0)
    # 2 of type 0 and 3 of type 1 over 200 eV: 1.0 and 1.5 per 100 eV (pending species
    # are not counted until released)
    o.run_until(5e-9)
    assert o.E_dep == 200.0
    np.testing.assert_array_equal(o.counts(), [2, 3])
    np.testing.assert_allclose(o.g_values(), [1.0, 1.5], rtol=1e-15)


def test_g_value_in_si_units_matches_a_known_dose(impl):
    # 1 Gy in a (1 um)^3 water box (1e-15 kg) deposits 1e-15 J. Place n molecules with
    # exactly that energy: G [molecules/100 eV] converted to mol/J (x 1/(100 eV N_A))
    # times the dose must give n / N_A mol per kg of water.
    L = 1000.0
    energy_J = 1.0 * 1e-15
    energy_eV = energy_J / E_CHARGE
    n = 700
    o = _inert(impl, L=L)
    o.inject(np.zeros(n, np.int64), np.zeros((n, 3)), np.zeros(n), energy_eV=energy_eV)
    o.run_until(1e-9)
    G_mol_per_J = o.g_values()[0] / (100.0 * E_CHARGE * N_A)
    assert math.isclose(G_mol_per_J * 1.0 * 1e-15, n / N_A, rel_tol=1e-12)
    # the textbook factor: 1 molecule / 100 eV = 1.0364e-7 mol/J
    assert math.isclose(1.0 / (100.0 * E_CHARGE * N_A), 1.0364e-7, rel_tol=1e-4)


def test_species_steps_on_a_known_schedule(impl):
    # Fixed 1 ns steps to 5 ns: 3 species from t = 0 take 5 steps; 2 arriving at 2.5 ns
    # are released at the 3 ns boundary and take 2 steps: 3 * 5 + 2 * 2 = 19.
    o = _inert(impl)
    o.inject([0, 0, 1], np.zeros((3, 3)), np.zeros(3), energy_eV=1.0)
    o.inject([1, 1], np.zeros((2, 3)), np.full(2, 2.5e-9), energy_eV=1.0)
    o.run_until(5e-9)
    assert o.step == 5 and o.species_steps == 19
    # Geometric steps 1, 2, 4, 8 ns (capped at 8) to 20 ns: 1+2+4+8 = 15, then a 5 ns
    # step trimmed to land on 20 ns: 5 steps of 4 species = 20.
    o = _inert(impl, growth=2.0, dt_max=8e-9)
    o.inject([0, 1, 1, 0], np.zeros((4, 3)), np.zeros(4), energy_eV=1.0)
    o.run_until(20e-9)
    assert o.step == 5 and o.species_steps == 20
    assert o.t == 20e-9


def test_energy_and_counts_across_a_reaction(impl):
    # One e_aq + OH pair on top of each other reacts in the first step (R2 -> OH-):
    # the count of OH- is 1 over the 100 eV injected, so G(OH-) = 1 and G(e_aq) = 0.
    o = impl.SBSOracle(W.D_NM2_S, W.WATER_REACTIONS, 100.0, seed=2, dt_min=1e-12, dt_max=1e-12,
                      record=True)
    o.inject([W.E_AQ, W.OH], np.zeros((2, 3)), np.zeros(2), energy_eV=100.0)
    o.run_until(1e-12)
    assert o.events_total[1] == 1
    g = o.g_values()
    assert g[W.OHM] == 1.0 and g[W.E_AQ] == 0.0 and g[W.OH] == 0.0
