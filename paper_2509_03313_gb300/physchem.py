"""Physico-chemical stage: radiation events branched into the first chemical species
(Sec. 2.4 and the supplement's Table S1, Sec. 2.1 workflow).

The physical stage (proton transport, ionisation and excitation cross sections) is not
reproduced here: radiation events are synthetic, placed along straight tracks like the
species of ``workloads.track_pulse``. What this module takes from the paper is the
physico-chemical step of Sec. 2.4: every ionised or excited water molecule, and every
sub-excitation electron, ends in one of the dissociation channels of Table S1 with the
printed probability, and the channel's products are the species the step-by-step stage
receives (through ``chem_inject_pulse``). Host-side input preparation only: the products
are handed to the CUDA library (and to the FP64 reference) as plain arrays.

Readings where the paper is silent:

* event kinds: an ionisation leaves H2O+ (branch "ionization") and a sub-excitation
  electron whose fate is solvation (e_aq), dissociative attachment to a water molecule
  ("attachment": OH + OH- + H2, a second water molecule consumed) or recombination with
  the hole, which replaces the H2O+ branch by the "electron hole" channels; excitations
  are to the A1B1, B1A1 or Rydberg/diffusion-band states. The fractions of these kinds
  and fates come from the physical stage, which is not available: they are parameters;
* H+ is the library's H3O+ (same species, charge +1); O(3P) has no diffusion
  coefficient and no reaction in the paper and is not a chemical species here: its atoms
  are counted (``o3p``) so that oxygen stays exactly balanced;
* every channel's products are placed at the parent molecule plus an isotropic Gaussian
  offset (``rms_molecule_nm`` per axis); the electron's products (e_aq, or the
  attachment products) at the parent plus ``rms_electron_nm`` per axis (thermalisation);
* water consumed per event: the molecules whose atoms the products carry (two for the
  attachment channel and for H2 + 2 OH, none for relaxation back to H2O).
"""
from __future__ import annotations

import dataclasses
from typing import Dict, List, Sequence, Tuple

import numpy as np

from . import workloads as W

E_AQ, OH, H, H3O, OHM, H2, H2O2 = W.E_AQ, W.OH, W.H, W.H3O, W.OHM, W.H2, W.H2O2


@dataclasses.dataclass(frozen=True)
class Channel:
    """One row of Table S1: probability (percent, as printed), product species, water
    molecules whose atoms the products carry, O(3P) atoms produced."""
    name: str
    probability: float
    products: Tuple[int, ...]
    water: int
    o3p: int = 0


# Table S1 (branching ratios of the physico-chemical stage, after Geant4-DNA).
TABLE_S1: Dict[str, List[Channel]] = {
    "ionization": [Channel("H+ + OH", 100.0, (H3O, OH), 1)],
    "A1B1": [Channel("H + OH", 65.0, (H, OH), 1),
             Channel("H2O", 35.0, (), 0)],
    "B1A1": [Channel("H+ + OH + e_aq", 50.0, (H3O, OH, E_AQ), 1),
             Channel("H + OH", 25.35, (H, OH), 1),
             Channel("H2 + 2 OH", 3.25, (H2, OH, OH), 2),
             Channel("2 H + O(3P)", 3.9, (H, H), 1, 1),
             Channel("H2O", 17.5, (), 0)],
    "rydberg": [Channel("H+ + OH + e_aq", 50.0, (H3O, OH, E_AQ), 1),
                Channel("H2O", 50.0, (), 0)],
    "attachment": [Channel("OH + OH- + H2", 100.0, (OH, OHM, H2), 2)],
    "hole": [Channel("H + OH", 35.75, (H, OH), 1),
             Channel("H2 + 2 OH", 13.65, (H2, OH, OH), 2),
             Channel("2 H + O(3P)", 15.6, (H, H), 1, 1),
             Channel("H2O", 35.0, (), 0)],
    "solvation": [Channel("e_aq", 100.0, (E_AQ,), 0)],
}

# Event kinds of the synthetic physical stage and the electron fates of an ionisation.
EVENT_KINDS = ("ionization", "A1B1", "B1A1", "rydberg")
ELECTRON_FATES = ("solvation", "attachment", "hole")


def sample_channels(branch: str, n: int, rng: np.random.Generator) -> np.ndarray:
    """Indices into TABLE_S1[branch] for n independent events, drawn with the table's
    probabilities."""
    p = np.array([c.probability for c in TABLE_S1[branch]], dtype=np.float64)
    return rng.choice(p.size, size=n, p=p / p.sum())


@dataclasses.dataclass
class FirstProducts:
    """Species of a set of radiation events: types, positions (nm), and the exact
    bookkeeping of what they came from."""
    types: np.ndarray        # int32, species types
    xyz: np.ndarray          # float64, n x 3
    water: int               # water molecules consumed
    o3p: int                 # O(3P) atoms produced (not chemical species here)
    channel_counts: Dict[str, np.ndarray]  # per branch: events per channel


def branch_events(kinds: np.ndarray, fates: np.ndarray, xyz: np.ndarray, rng: np.random.Generator,
                  rms_molecule_nm: float = 1.0, rms_electron_nm: float = 6.0) -> FirstProducts:
    """First products of radiation events (Table S1). kinds[i] indexes EVENT_KINDS,
    fates[i] indexes ELECTRON_FATES (used for ionisations only), xyz[i] is the parent
    molecule's position."""
    kinds = np.asarray(kinds)
    fates = np.asarray(fates)
    xyz = np.asarray(xyz, dtype=np.float64).reshape(-1, 3)
    out_t: List[np.ndarray] = []
    out_x: List[np.ndarray] = []
    water = 0
    o3p = 0
    counts: Dict[str, np.ndarray] = {b: np.zeros(len(TABLE_S1[b]), np.int64) for b in TABLE_S1}

    def emit(branch: str, idx: np.ndarray, parent: np.ndarray, rms: float):
        nonlocal water, o3p
        if idx.size == 0:
            return
        ch = sample_channels(branch, idx.size, rng)
        counts[branch] += np.bincount(ch, minlength=len(TABLE_S1[branch]))
        for k, c in enumerate(TABLE_S1[branch]):
            sel = parent[ch == k]
            water += c.water * sel.shape[0]
            o3p += c.o3p * sel.shape[0]
            for prod in c.products:
                out_t.append(np.full(sel.shape[0], prod, np.int32))
                out_x.append(sel + rng.normal(0.0, rms, size=sel.shape))

    ion = kinds == EVENT_KINDS.index("ionization")
    # the ionised molecule: its own branch unless the electron recombines with the hole
    hole = ion & (fates == ELECTRON_FATES.index("hole"))
    emit("ionization", np.nonzero(ion & ~hole)[0], xyz[ion & ~hole], rms_molecule_nm)
    emit("hole", np.nonzero(hole)[0], xyz[hole], rms_molecule_nm)
    # the electron of the other ionisations, thermalised away from the parent
    for fate in ("solvation", "attachment"):
        sel = ion & (fates == ELECTRON_FATES.index(fate))
        emit(fate, np.nonzero(sel)[0], xyz[sel], rms_electron_nm)
    for kind in ("A1B1", "B1A1", "rydberg"):
        sel = kinds == EVENT_KINDS.index(kind)
        emit(kind, np.nonzero(sel)[0], xyz[sel], rms_molecule_nm)
    types = np.concatenate(out_t) if out_t else np.zeros(0, np.int32)
    pos = np.concatenate(out_x) if out_x else np.zeros((0, 3))
    return FirstProducts(types, pos, int(water), int(o3p), counts)


def track_events(n_tracks: int, L: float, events_per_track: int, seed: int,
                 kind_fractions: Sequence[float] = (0.6, 0.1, 0.2, 0.1),
                 fate_fractions: Sequence[float] = (0.8, 0.05, 0.15),
                 events_per_spur: float = 3.0, sigma_nm: float = 1.0, stream: int = 7):
    """Synthetic radiation events along straight tracks (as ``workloads.track_pulse``):
    spur centres uniform along each track, events at a random spur's centre plus an
    isotropic Gaussian offset, kinds and electron fates drawn with the given fractions
    (parameters standing in for the physical stage). Returns (kinds, fates, xyz)."""
    rng = W._rng(seed, stream)
    kf = np.asarray(kind_fractions, np.float64)
    ff = np.asarray(fate_fractions, np.float64)
    n_spurs = max(1, int(round(events_per_track / events_per_spur)))
    xs, ks, fs = [], [], []
    for _ in range(n_tracks):
        x0, y0 = rng.uniform(-0.5 * L, 0.5 * L, size=2)
        zc = rng.uniform(-0.5 * L, 0.5 * L, size=n_spurs)
        pick = rng.integers(0, n_spurs, size=events_per_track)
        p = np.empty((events_per_track, 3))
        p[:, 0], p[:, 1], p[:, 2] = x0, y0, zc[pick]
        xs.append(p + rng.normal(0.0, sigma_nm, size=p.shape))
        ks.append(rng.choice(kf.size, size=events_per_track, p=kf / kf.sum()))
        fs.append(rng.choice(ff.size, size=events_per_track, p=ff / ff.sum()))
    return np.concatenate(ks), np.concatenate(fs), np.concatenate(xs)


def physchem_pulse(n_tracks: int, L: float, events_per_track: int, seed: int, t0: float = 0.0,
                   let_eV_per_nm: float = W.LET_EV_PER_NM, **kw) -> Tuple[W.Pulse, FirstProducts]:
    """A pulse of synthetic tracks whose species are the Table S1 products of their
    radiation events, folded into the box (Eq. 1); all arrive at t0. Each track deposits
    let_eV_per_nm * L eV. Returns the pulse and the bookkeeping of its products."""
    rng = W._rng(seed, 11)
    ev_kw = {k: kw.pop(k) for k in ("kind_fractions", "fate_fractions", "events_per_spur", "sigma_nm")
             if k in kw}
    kinds, fates, xyz = track_events(n_tracks, L, events_per_track, seed, **ev_kw)
    fp = branch_events(kinds, fates, xyz, rng, **kw)
    pos = W._into_box(fp.xyz, L)
    pulse = W.Pulse(fp.types.astype(np.int32), pos, np.full(fp.types.shape[0], t0),
                    float(n_tracks * let_eV_per_nm * L))
    return pulse, fp
