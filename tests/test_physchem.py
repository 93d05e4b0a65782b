"""The physico-chemical injector (Sec. 2.4, Table S1) on the CPU: the channel table
equals the paper's, sampled channels follow its probabilities within 3 sigma, and every
injected set conserves charge exactly and H and O atoms against the water molecules
consumed (and the O(3P) atoms, which are not chemical species here)."""
import math

import numpy as np

from conftest import read_golden
from paper_2509_03313_gb300 import physchem as P, workloads as W

NAMES = {"e_aq": W.E_AQ, "OH": W.OH, "H": W.H, "H3O": W.H3O, "OHm": W.OHM, "H2": W.H2, "H2O2": W.H2O2}


def _golden():
    rows = {}
    for branch, prob, prods in read_golden("table_s1_branching.txt"):
        parts = [] if prods == "-" else prods.split("+")
        o3p = parts.count("O3P")
        species = tuple(sorted(NAMES[x] for x in parts if x != "O3P"))
        rows.setdefault(branch, []).append((float(prob), species, o3p))
    return rows


def test_channel_table_is_table_s1():
    gold = _golden()
    assert set(gold) == set(P.TABLE_S1)
    for branch, chans in P.TABLE_S1.items():
        got = [(c.probability, tuple(sorted(c.products)), c.o3p) for c in chans]
        assert got == gold[branch], branch
        assert math.isclose(sum(c.probability for c in chans), 100.0, abs_tol=1e-9)


def test_sampled_channels_follow_table_s1_within_3_sigma():
    rng = np.random.default_rng(2024)
    n = 400_000
    for branch, chans in P.TABLE_S1.items():
        k = P.sample_channels(branch, n, rng)
        cnt = np.bincount(k, minlength=len(chans))
        for c, m in zip(chans, cnt):
            p = c.probability / 100.0
            sigma = math.sqrt(n * p * (1.0 - p))
            assert abs(m - n * p) <= 3.0 * sigma + 1e-9, (branch, c.name, m, n * p, sigma)


def test_channel_frequencies_through_whole_events():
    # the same check on the channel counts of a large synthetic event set: each branch
    # sees the events routed to it (ionisations without recombination, recombinations,
    # the electrons of solvation and attachment, the three excitations)
    kinds, fates, xyz = P.track_events(50, 2000.0, 4000, seed=3)
    fp = P.branch_events(kinds, fates, xyz, np.random.default_rng(9))
    for branch, cnt in fp.channel_counts.items():
        n = int(cnt.sum())
        assert n > 0, branch
        for c, m in zip(P.TABLE_S1[branch], cnt):
            p = c.probability / 100.0
            assert abs(m - n * p) <= 3.0 * math.sqrt(n * p * (1.0 - p)) + 1e-9, (branch, c.name)


def test_injected_sets_conserve_charge_and_atoms():
    for seed in range(5):
        kinds, fates, xyz = P.track_events(4, 500.0, 3000, seed=seed,
                                           kind_fractions=(0.5, 0.2, 0.2, 0.1),
                                           fate_fractions=(0.6, 0.2, 0.2))
        fp = P.branch_events(kinds, fates, xyz, np.random.default_rng(seed))
        c = np.bincount(fp.types, minlength=7)
        assert int(c @ W.CHARGE) == 0
        assert int(c @ W.N_H) == 2 * fp.water
        assert int(c @ W.N_O) + fp.o3p == fp.water
        # relaxation channels consume no water and add no species
        assert fp.types.shape[0] == sum(
            len(ch.products) * int(cnt[k]) for b, cnt in fp.channel_counts.items()
            for k, ch in enumerate(P.TABLE_S1[b]))


def test_every_ionisation_is_neutral_overall():
    # ionisations only, each electron fate alone: charge 0 for every set
    for f in range(3):
        n = 2000
        kinds = np.zeros(n, int)
        fates = np.full(n, f)
        fp = P.branch_events(kinds, fates, np.zeros((n, 3)), np.random.default_rng(f))
        c = np.bincount(fp.types, minlength=7)
        assert int(c @ W.CHARGE) == 0
        if f == 0:   # solvation: H+ + OH + e_aq per ionisation
            assert np.array_equal(c[[W.E_AQ, W.OH, W.H3O]], [n, n, n])
        if f == 1:   # attachment: H+ + OH, and OH + OH- + H2
            assert np.array_equal(c[[W.H3O, W.OH, W.OHM, W.H2]], [n, 2 * n, n, n])


def test_physchem_pulse_is_inside_the_box_and_deposits_the_tracks_energy():
    pulse, fp = P.physchem_pulse(6, 800.0, 1500, seed=4)
    assert pulse.n == fp.types.shape[0] > 0
    assert np.all(pulse.xyz >= -400.0) and np.all(pulse.xyz < 400.0)
    assert pulse.energy_eV == 6 * W.LET_EV_PER_NM * 800.0
