"""Pins of the reference homogeneous (beam-off) stage, Sec. 2.3 with the rate equations
Eq. 3 / Eq. 4: closed-form solutions of single reactions, the concentration form of the
same equations integrated by another scheme, exact conservation of charge and atoms
after rounding to whole events, unbiased rounding, uniform re-created positions, and the
hand-over to the step-by-step stage."""
import math

import numpy as np
import pytest
from scipy import stats

from oracle import homogeneous as H
from oracle import kinetics, sbs
from paper_2509_03313_gb300 import workloads as W


def _a_plus_b_events(a0, b0, kappa, T):
    # dn_a/dt = -kappa n_a n_b with n_a - n_b = a0 - b0 fixed: a logistic-type solution
    d = a0 - b0
    n_a = d / (1.0 - (b0 / a0) * math.exp(-kappa * d * T))
    return a0 - n_a


def _a_plus_a_events(a0, kappa, T):
    # dn/dt = -2 kappa n^2: 1/n = 1/a0 + 2 kappa t, two A per event
    return 0.5 * (a0 - a0 / (1.0 + 2.0 * kappa * a0 * T))


@pytest.mark.parametrize("T", [1e-7, 1e-5, 1e-3, 10.0])
def test_single_reactions_match_closed_forms(T):
    L = 500.0
    NV = sbs.N_AVOGADRO * L ** 3 * 1e-24
    k = 3.0e10
    # A + B -> C with 4000 A and 1500 B molecules
    e = H.extents([4000.0, 1500.0, 0.0], L, T, [(0, 1, k, (2,), 0)])
    assert e[0] == pytest.approx(_a_plus_b_events(4000.0, 1500.0, k / NV, T), rel=1e-9)
    # A + A -> B with the tabulated value being 2k: kappa = (k_tab / 2) / (N_A V)
    e = H.extents([3000.0, 0.0], L, T, [(0, 0, k, (1,), 0)])
    assert e[0] == pytest.approx(_a_plus_a_events(3000.0, 0.5 * k / NV, T), rel=1e-9)


def test_extents_agree_with_the_concentration_form_of_the_full_table():
    L = 1000.0
    n0 = W.MIX_COUNTS.astype(float) * 3.0
    nu = H.stoichiometry(7, W.WATER_REACTIONS)
    for T in (1e-6, 1e-4, 1e-2):
        e = H.extents(n0, L, T, W.WATER_REACTIONS)
        c = kinetics.integrate(kinetics.molar(n0, L), [0.0, T], W.D_NM2_S, W.WATER_REACTIONS,
                               method="LSODA", rtol=1e-12, atol=1e-24)[-1]
        n_ref = c / kinetics.molar(1.0, L)
        np.testing.assert_allclose(n0 + nu @ e, n_ref, rtol=1e-7, atol=1e-5)
        assert np.all(e >= -1e-9)


def _totals(n, water):
    return (int(n @ W.CHARGE), int(n @ W.N_H) + 2 * water, int(n @ W.N_O) + water)


@pytest.mark.parametrize("seed", range(6))
def test_whole_events_conserve_charge_and_atoms(seed):
    rng = np.random.default_rng(seed)
    n0 = rng.integers(0, 50, size=7)
    L = 60.0
    key = sbs.philox_key(seed, 0)
    e, E, n = H.stage(n0, L, 1e-3, W.WATER_REACTIONS, stage_index=seed, key=key)
    assert np.all(n >= 0)
    assert np.all(E <= np.ceil(np.maximum(e, 0.0)))  # rounding, then take-backs only lower
    w = H.water_change(E, W.WATER_REACTIONS)
    assert _totals(n, w) == _totals(n0, 0)
    nu = H.stoichiometry(7, W.WATER_REACTIONS)
    assert np.array_equal(n, n0 + nu @ E)


def test_rounding_is_unbiased_and_within_one_event():
    nu = H.stoichiometry(7, W.WATER_REACTIONS)
    n0 = np.array([10 ** 6] * 7)
    rng = np.random.default_rng(1)
    e = rng.uniform(0, 20, size=9)
    Es = np.array([H.integer_events(e, rng.uniform(size=9), n0, nu)[0] for _ in range(20000)])
    assert np.all(np.abs(Es - e) < 1.0)
    np.testing.assert_allclose(Es.mean(axis=0), e, atol=4 * 0.5 / math.sqrt(20000))


def test_negative_counts_are_taken_back_from_the_lowest_consuming_reaction():
    # X produced by reactions 0 and 1 (0.9 events each), consumed by reaction 2 (1.8):
    # rounding 0.9 down twice and 1.8 up leaves X at -1 before the take-back.
    # types: 0 P, 1 Q, 2 X, 3 Y; r0: P + P -> X, r1: Q + Q -> X, r2: X + Y -> 0
    rx = [(0, 0, 1.0, (2,), 0), (1, 1, 1.0, (2,), 0), (2, 3, 1.0, (), 0)]
    nu = H.stoichiometry(4, rx)
    n0 = np.array([10, 10, 0, 10])
    E, n = H.integer_events([0.9, 0.9, 1.8], [0.95, 0.95, 0.1], n0, nu)
    assert list(E) == [0, 0, 0] and list(n) == [10, 10, 0, 10]
    E, n = H.integer_events([0.9, 0.9, 1.8], [0.5, 0.95, 0.1], n0, nu)
    assert list(E) == [1, 0, 1] and list(n) == [8, 10, 0, 9]


def test_rounding_uniforms_follow_their_counter():
    key = sbs.philox_key(123, 4)
    u = H.rounding_uniforms(9, 5, key)
    w0, w1, _, _ = sbs.philox4x32_10((5, 7, 0, 4), key)
    assert u[7] == sbs.uniform_closed0(w0, w1)
    assert not np.array_equal(u, H.rounding_uniforms(9, 6, key))


def test_recreated_positions_are_uniform_in_the_box():
    L = 750.0
    key = sbs.philox_key(9, 2)
    ids = np.arange(1000, 41000)
    p = H.materialised_positions(ids, L, key)
    assert np.all(p >= -0.5 * L) and np.all(p < 0.5 * L)
    for a in range(3):
        assert stats.kstest((p[:, a] + 0.5 * L) / L, "uniform").pvalue > 1e-3
    assert abs(np.corrcoef(p[:, 0], p[:, 2])[0, 1]) < 0.03
    np.testing.assert_array_equal(p[5], H.materialised_positions([ids[5]], L, key)[0])


def test_stage_hands_over_to_the_step_by_step_stage():
    wl = W.uniform_2000(seed=2, L=300.0, n_steps=20)
    o = sbs.from_workload(wl, seed=2)
    o.run_until(2e-8)
    n_before, water_before = o.counts().copy(), o.water
    next_id = o.next_id
    ev_before = o.events_total.copy()
    e, E = o.run_homogeneous(1e-4)
    assert o.t == 1e-4 and o.ids.shape[0] == 0
    n_after = o.counts()
    assert _totals(n_after, o.water) == _totals(n_before, water_before)
    np.testing.assert_array_equal(o.events_total - ev_before, E)
    # the survivors come back as particles at the next release: ids from next_id in
    # ascending type order, at their counter-based uniform positions
    assert o._release() == n_after.sum()
    ids, types, pos = o.state()
    np.testing.assert_array_equal(ids, np.arange(next_id, next_id + n_after.sum()))
    np.testing.assert_array_equal(types, np.repeat(np.arange(7), n_after))
    np.testing.assert_array_equal(pos, H.materialised_positions(ids, o.L, o.key))
    assert o.t_last_release == 1e-4


def test_due_species_join_and_arrivals_inside_the_stage_are_refused():
    o = sbs.SBSOracle(W.D_NM2_S, W.WATER_REACTIONS, 200.0, seed=1)
    o.inject([W.OH, W.OH], [[0, 0, 0], [10, 0, 0]], [0.0, 0.0])
    e, E = o.run_homogeneous(1e-3)
    assert o.counts()[W.OH] + 2 * o.counts()[W.H2O2] == 2
    o.inject([W.E_AQ], [[0, 0, 0]], [5e-3])
    with pytest.raises(ValueError):
        o.run_homogeneous(1e-2)
    assert o.run_homogeneous(5e-3) is not None
