"""Seeded synthetic inputs for the multi-pulse SBS chemistry (shared by the library's
callers, the tests and the benchmark).

This module holds data and random input generators only: the species list and the two
published tables the method consumes (Table 1 rate constants, Table S2 diffusion
coefficients), plus generators of initial positions, species types, arrival times and
deposited energies. It contains none of the method's arithmetic (no reaction radii, no
diffusion, no pair search): both the CUDA library and the FP64 reference receive the
arrays produced here and derive everything else themselves.

Random draws use numpy's counter-based ``Philox`` bit generator keyed by the seed, so a
(workload, seed) pair always yields the same arrays on any machine.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional, Sequence

import numpy as np

# Species order used throughout (Table S2). H3O+ is the paper's H+ (same species, +1).
SPECIES = ("e_aq", "OH", "H", "H3O+", "OH-", "H2", "H2O2")
E_AQ, OH, H, H3O, OHM, H2, H2O2 = range(7)

# Table S2: diffusion coefficients, in 1e9 nm^2/s, converted here to nm^2/s.
D_NM2_S = np.array([4.82, 2.2, 7.0, 9.3, 5.3, 4.8, 2.3], dtype=np.float64) * 1e9

# Charge and (H, O) atom content per species; used by conservation checks only.
CHARGE = np.array([-1, 0, 0, +1, -1, 0, 0], dtype=np.int64)
N_H = np.array([0, 1, 1, 1, 1, 2, 2], dtype=np.int64)
N_O = np.array([0, 1, 0, 0, 1, 0, 2], dtype=np.int64)


@dataclasses.dataclass(frozen=True)
class Reaction:
    """One row of Table 1: reactant types a, b; the tabulated rate constant in
    L mol^-1 s^-1 (for the self reactions R1, R6 and R8 the table prints "2k" and that
    printed value is what is stored); product types; water molecules created (+) or
    consumed (-) so that H and O atoms balance."""
    name: str
    a: int
    b: int
    k_tab: float
    products: tuple
    water_delta: int


# Table 1 (water radiolysis reactions, k in 1e10 L/mol/s).
WATER_REACTIONS: List[Reaction] = [
    Reaction("R1", E_AQ, E_AQ, 1.3e10, (H2, OHM, OHM), -2),
    Reaction("R2", E_AQ, OH, 3.0e10, (OHM,), 0),
    Reaction("R3", E_AQ, H, 2.6e10, (H2, OHM), -1),
    Reaction("R4", E_AQ, H3O, 2.3e10, (H,), 0),
    Reaction("R5", E_AQ, H2O2, 1.4e10, (OH, OHM), 0),
    Reaction("R6", OH, OH, 0.95e10, (H2O2,), 0),
    Reaction("R7", OH, H, 1.5e10, (), +1),
    Reaction("R8", H, H, 1.1e10, (H2,), 0),
    Reaction("R9", H3O, OHM, 11.0e10, (), +1),
]

# Species mix of the 2,000-species uniform workload: e 600, OH 600, H 120, H3O+ 600,
# OH- 80. Used as the type ratio of the synthetic tracks too.
MIX_COUNTS = np.array([600, 600, 120, 600, 80, 0, 0], dtype=np.int64)
LET_EV_PER_NM = 0.96  # 70 MeV protons, 0.96 keV/um (Sec. 2.5)


def _rng(seed: int, stream: int = 0) -> np.random.Generator:
    return np.random.Generator(np.random.Philox(key=[int(seed) & 0xFFFFFFFFFFFFFFFF, stream]))


@dataclasses.dataclass
class Pulse:
    """Species handed to one inject call: types (int32, n), absolute positions in the box
    [-L/2, L/2)^3 (float64, n x 3, nm), arrival times (float64, n, s) and the energy the
    pulse deposits (eV)."""
    types: np.ndarray
    xyz: np.ndarray
    t_arrival: np.ndarray
    energy_eV: float

    @property
    def n(self) -> int:
        return int(self.types.shape[0])


def _into_box(x: np.ndarray, L: float) -> np.ndarray:
    # Input preparation: fold generated coordinates into [-L/2, L/2).
    y = np.mod(x + 0.5 * L, L) - 0.5 * L
    y[y >= 0.5 * L] = -0.5 * L
    return y


def uniform_mixture(counts: Sequence[int], L: float, seed: int, t_arrival: float = 0.0,
                    energy_eV: float = 0.0) -> Pulse:
    """Homogeneous mixture: counts[type] species placed uniformly in the box."""
    rng = _rng(seed, 1)
    types = np.concatenate([np.full(int(c), t, dtype=np.int32) for t, c in enumerate(counts)])
    perm = rng.permutation(types.shape[0])
    types = types[perm]
    xyz = rng.uniform(-0.5 * L, 0.5 * L, size=(types.shape[0], 3))
    xyz = _into_box(xyz, L)
    return Pulse(types, xyz, np.full(types.shape[0], t_arrival), float(energy_eV))


def track_pulse(n_tracks: int, L: float, species_per_track: int, seed: int,
                sigma_nm: float = 2.0, species_per_spur: float = 5.0,
                mix: Sequence[float] = MIX_COUNTS, t0: float = 0.0, fwhm: float = 0.0,
                let_eV_per_nm: float = LET_EV_PER_NM, stream: int = 2) -> Pulse:
    """Synthetic proton tracks standing in for the physics stage (Sec. 2.1).

    Each track is a straight line along z at a uniform (x, y) that crosses the whole box.
    Spur centres are uniform along the track (a Poisson-like process, mean spacing
    L * species_per_spur / species_per_track); every species picks a spur at random and
    sits at its centre plus an isotropic Gaussian offset of sigma_nm. Types are drawn
    with probabilities proportional to ``mix``. The track arrives at t0 (fwhm == 0) or at
    a time uniform over the square pulse [t0, t0 + fwhm). Each track deposits
    let_eV_per_nm * L eV.
    """
    rng = _rng(seed, stream)
    p = np.asarray(mix, dtype=np.float64)
    p = p / p.sum()
    n_spurs = max(1, int(round(species_per_track / species_per_spur)))
    xyz_all, types_all, t_all = [], [], []
    for _ in range(n_tracks):
        x0, y0 = rng.uniform(-0.5 * L, 0.5 * L, size=2)
        t_arr = t0 + (fwhm * rng.uniform() if fwhm > 0.0 else 0.0)
        zc = rng.uniform(-0.5 * L, 0.5 * L, size=n_spurs)
        pick = rng.integers(0, n_spurs, size=species_per_track)
        xyz = np.empty((species_per_track, 3))
        xyz[:, 0] = x0
        xyz[:, 1] = y0
        xyz[:, 2] = zc[pick]
        xyz += rng.normal(0.0, sigma_nm, size=(species_per_track, 3))
        xyz_all.append(_into_box(xyz, L))
        types_all.append(rng.choice(len(p), size=species_per_track, p=p).astype(np.int32))
        t_all.append(np.full(species_per_track, t_arr))
    types = np.concatenate(types_all)
    xyz = np.concatenate(xyz_all)
    t_arrival = np.concatenate(t_all)
    return Pulse(types, xyz, t_arrival, float(n_tracks * let_eV_per_nm * L))


def pulse_train(n_pulses: int, period_s: float, fwhm_s: float, n_tracks: int, L: float,
                species_per_track: int, seed: int, **kw) -> List[Pulse]:
    """A train of square pulses starting at t = p * period_s (Sec. 2.1: the period is
    1/f, with the average dose rate Dp * f)."""
    return [track_pulse(n_tracks, L, species_per_track, seed, t0=p_i * period_s,
                        fwhm=fwhm_s, stream=1000 + p_i, **kw) for p_i in range(n_pulses)]


# ---------------------------------------------------------------------------------------
# Named workloads (sizes from the benchmark's configuration list).


@dataclasses.dataclass
class Schedule:
    """Time-step policy handed to both implementations: start at dt_min, multiply by
    dt_growth every step up to dt_max, restart at dt_min whenever species are released
    (if reset_on_release); cutoff_c sets the pair-search cutoff; sbs_horizon > 0 turns
    on the free-diffusion jump after that long without a release (0 = off)."""
    dt_min: float
    dt_max: float
    dt_growth: float = 1.0
    reset_on_release: bool = True
    cutoff_c: float = 3.0
    sbs_horizon: float = 0.0


@dataclasses.dataclass
class Workload:
    name: str
    L: float
    pulses: List[Pulse]
    schedule: Schedule
    t_end: float
    n_types: int = 7
    D: np.ndarray = dataclasses.field(default_factory=lambda: D_NM2_S.copy())
    reactions: List[Reaction] = dataclasses.field(default_factory=lambda: list(WATER_REACTIONS))

    @property
    def n_species(self) -> int:
        return sum(p.n for p in self.pulses)


LOG_GROWTH_20_PER_DECADE = 10.0 ** (1.0 / 20.0)


def uniform_2000(seed: int, L: float = 1000.0, n_steps: int = 1000) -> Workload:
    """Plain single pulse: 2,000 species (e 600, OH 600, H 120, H3O+ 600, OH- 80)
    uniform in a 1 um periodic cube, fixed dt = 1 ns, 1,000 steps to 1 us. The dense
    variant uses L = 200 nm."""
    pulse = uniform_mixture(MIX_COUNTS, L, seed, energy_eV=2000 * 100.0 / 6.0)
    return Workload(f"uniform2000_L{int(L)}", L, [pulse],
                    Schedule(dt_min=1e-9, dt_max=1e-9, dt_growth=1.0), t_end=n_steps * 1e-9)


def single_pulse_tracks(seed: int, n_species: int = 1_000_000, n_tracks: int = 200,
                        L: float = 5000.0, t_end: float = 1e-6, dt_min: float = 1e-12) -> Workload:
    """Single pulse of synthetic proton tracks: 5 um cube, 200 straight tracks of
    Gaussian spurs (sigma 2 nm), ~1e6 species, all arriving at t = 0, log-growing dt
    from 1 ps (20 steps per decade) to 1 us."""
    per_track = max(1, n_species // n_tracks)
    pulse = track_pulse(n_tracks, L, per_track, seed)
    return Workload(f"tracks{n_tracks}x{per_track}_L{int(L)}", L, [pulse],
                    Schedule(dt_min=dt_min, dt_max=1e-6, dt_growth=LOG_GROWTH_20_PER_DECADE),
                    t_end=t_end)


def tracks_same_density(seed: int, L: float, t_end: float = 1e-6) -> Workload:
    """The single-pulse track workload in a box of side L (nm) with the benchmark's track
    density per unit area (200 tracks per (5 um)^2) and species per nm of track (1e6
    species over 200 tracks of 5 um: one per nm), so the local structure, the species
    density and the time-step schedule are those of the 5 um workload: about 3.2e4
    species at L = 1.6 um, 2e7 at L = 13.6 um."""
    n_tracks = max(1, int(round(200.0 * (L / 5000.0) ** 2)))
    per_track = max(1, int(round(L)))
    return single_pulse_tracks(seed, n_species=n_tracks * per_track, n_tracks=n_tracks, L=L, t_end=t_end)


def multi_pulse(seed: int, n_pulses: int = 10, period_s: float = 1e-4, fwhm_s: float = 1e-6,
                n_tracks: int = 163, species_per_track: int = 1800, L: float = 5000.0,
                dt_min: float = 1e-11, dt_max: float = 1e-6) -> Workload:
    """Multi-pulse build-up: 10 square pulses of 1 us every 0.1 ms, species carried
    across the intervals (SBS throughout)."""
    pulses = pulse_train(n_pulses, period_s, fwhm_s, n_tracks, L, species_per_track, seed)
    return Workload(f"multipulse{n_pulses}_L{int(L)}", L, pulses,
                    Schedule(dt_min=dt_min, dt_max=dt_max, dt_growth=LOG_GROWTH_20_PER_DECADE),
                    t_end=(n_pulses - 1) * period_s + fwhm_s + 1e-6)


def hybrid_stages(n_pulses: int, period_s: float, fwhm_s: float, tail_s: float = 10.0,
                  sbs_after_s: float = 0.0) -> List[tuple]:
    """The alternation of Sec. 2.1: step-by-step chemistry while the beam is on (each
    pulse [T_k, T_k + fwhm_s), extended by sbs_after_s), the rate equations for the rest
    of the beam-off time up to the next pulse, and for tail_s after the last pulse.
    Returns the calls in order as (kind, t_end) with kind "sbs" or "ode"."""
    out = []
    for k in range(n_pulses):
        t_on = k * period_s + fwhm_s + sbs_after_s
        out.append(("sbs", t_on))
        t_next = (k + 1) * period_s if k + 1 < n_pulses else t_on + tail_s
        if t_next > t_on:
            out.append(("ode", t_next))
    return out


def dose_rate_sweep(n_trains: int = 64, seed: int = 0, n_min: int = 10_000,
                    n_max: int = 2_000_000, n_pulses: int = 10, fwhm_s: float = 1e-6,
                    sbs_horizon: float = 1e-3) -> List[dict]:
    """Batched sweep: n_trains independent pulse trains, average dose rate log-spaced over
    0.01-1e5 Gy/s at pulse dose rates 2e5 and 1e6 Gy/s (half the trains each), species
    counts log-spaced over [n_min, n_max]. Returns per-train descriptions (pulse period,
    box side, species per pulse); the pulses themselves come from ``pulse_train``."""
    half = n_trains // 2
    dav = np.logspace(-2, 5, max(half, 1))
    out = []
    counts = np.logspace(math.log10(n_min), math.log10(n_max), n_trains)
    for b in range(n_trains):
        dp_rate = 2e5 if b < half else 1e6
        dose_per_pulse = dp_rate * fwhm_s
        d_av = dav[b % max(half, 1)]
        period = dose_per_pulse / d_av
        n_total = int(counts[b])
        per_pulse = max(n_total // n_pulses, 50)
        # Box side scaled so that the species density stays that of a 5 um box holding
        # 3e5 species per pulse.
        L = 5000.0 * (per_pulse / 3e5) ** (1.0 / 3.0)
        out.append(dict(train=b, pulse_dose_rate=dp_rate, avg_dose_rate=float(d_av),
                        period_s=float(period), L=float(L), species_per_pulse=per_pulse,
                        n_pulses=n_pulses, fwhm_s=fwhm_s, sbs_horizon=sbs_horizon,
                        seed=seed * 1000 + b))
    return out


def hybrid_sweep(n_trains: int = 64, seed: int = 0, scale: float = 1.0, bunches: int = 4,
                 fwhm_s: float = 1e-6, n_min: int = 10_000, n_max: int = 2_000_000,
                 n_pulses: int = 10, tail_s: float = 10.0):
    """The dose-rate sweep of ``dose_rate_sweep`` with every pulse delivered (no window):
    each of the n_pulses square pulses (period Dp / Dav) arrives as ``bunches`` equally
    spaced bunches of tracks. Returns (workloads, plans): plans[b] is the (kind, t_end)
    alternation of ``hybrid_stages`` for train b, ending tail_s after its last pulse."""
    wls, plans = [], []
    for desc in dose_rate_sweep(n_trains, seed, int(n_min * scale), int(n_max * scale),
                                n_pulses=n_pulses, fwhm_s=fwhm_s):
        L = desc["L"]
        n_tracks = max(2, int(round(160 * (L / 5000.0) ** 2)))
        per_track = max(1, desc["species_per_pulse"] // n_tracks)
        pulses = []
        for k in range(n_pulses):
            t0 = k * desc["period_s"]
            for q in range(bunches):
                pulses.append(track_pulse(max(1, n_tracks // bunches), L, per_track, desc["seed"],
                                          t0=t0 + fwhm_s * q / bunches, stream=10_000 + 100 * k + q))
        wls.append(Workload(f"hybrid{desc['train']}", L, pulses,
                            Schedule(dt_min=1e-11, dt_max=1e-7, dt_growth=LOG_GROWTH_20_PER_DECADE),
                            t_end=(n_pulses - 1) * desc["period_s"] + fwhm_s + tail_s))
        plans.append(hybrid_stages(n_pulses, desc["period_s"], fwhm_s, tail_s))
    return wls, plans


def dose_series(avg_dose_rates=(1.0, 1e4), pulse_dose_rate: float = 1e6,
                n_pulses=(1, 5, 10, 15, 20), species_per_pulse: int = 100_000,
                fwhm_s: float = 1e-6, bunches: int = 4, tail_s: float = 10.0, seed: int = 0):
    """Separate irradiations of 1, 5, 10, 15 and 20 pulses at each average dose rate, each
    followed by tail_s of beam-off (Fig. Concentration-Dose: post-irradiation H2O2 after
    1-20 Gy). One train per (dose rate, pulse count); the box holds species_per_pulse
    per pulse at the density of the sweep, so each pulse deposits about
    pulse_dose_rate * fwhm_s of dose. Returns (workloads, plans, meta) with meta[b] =
    {"avg_dose_rate", "n_pulses", "period_s"}."""
    L = 5000.0 * (species_per_pulse / 3e5) ** (1.0 / 3.0)
    n_tracks = max(2, int(round(160 * (L / 5000.0) ** 2)))
    per_track = max(1, species_per_pulse // n_tracks)
    wls, plans, meta = [], [], []
    for i, dav in enumerate(avg_dose_rates):
        T = pulse_dose_rate * fwhm_s / dav
        for n in n_pulses:
            pulses = []
            for k in range(n):
                for q in range(bunches):
                    pulses.append(track_pulse(max(1, n_tracks // bunches), L, per_track, seed + 7 * i,
                                              t0=k * T + fwhm_s * q / bunches, stream=10_000 + 100 * k + q))
            wls.append(Workload(f"dose{i}_{n}", L, pulses,
                                Schedule(dt_min=1e-11, dt_max=1e-7, dt_growth=LOG_GROWTH_20_PER_DECADE),
                                t_end=(n - 1) * T + fwhm_s + tail_s))
            plans.append(hybrid_stages(n, T, fwhm_s, tail_s))
            meta.append({"avg_dose_rate": float(dav), "n_pulses": int(n), "period_s": float(T)})
    return wls, plans, meta


def volume_scaling(L: float, seed: int, counts_at_200nm: Sequence[int] = MIX_COUNTS,
                   t_end: float = 1e-3, dt_min: float = 1e-12, dt_max: float = 1.5e-8) -> Workload:
    """Volume-scaling study (Sec. 2.2 setup, Sec. 3.1 results: verification of the
    periodic boundaries): one
    homogeneous mixture concentration in cubes of side L (0.2, 0.5 and 1.0 um), i.e.
    counts_at_200nm scaled by (L / 200 nm)^3 (2,000 species at 0.2 um, 250,000 at 1 um),
    followed to t_end = 1 ms with log-growing dt from 1 ps up to dt_max. The default
    dt_max is just below the smallest box's cap (every cutoff <= L/3 allows 1.6e-8 s at
    0.2 um), so all boxes take the same steps and only their size differs."""
    counts = np.round(np.asarray(counts_at_200nm, dtype=np.float64) * (L / 200.0) ** 3).astype(np.int64)
    pulse = uniform_mixture(counts, L, seed, energy_eV=float(counts.sum()) * 100.0 / 6.0)
    return Workload(f"volume_L{int(L)}", L, [pulse],
                    Schedule(dt_min=dt_min, dt_max=dt_max, dt_growth=LOG_GROWTH_20_PER_DECADE), t_end=t_end)


def large_build_up(seed: int, n_pulses: int = 20, period_s: float = 10e-6, fwhm_s: float = 1e-6,
                   L: float = 10000.0, tracks_per_pulse: int = 648, species_per_pulse: int = 375_000,
                   bunches: int = 4, dt_min: float = 1e-11, dt_max: float = 1e-6) -> Workload:
    """Large build-up: a 10 um cube, 20 pulses of about 1 Gy each (pulse dose rate 1e6 Gy/s
    over 1 us, every 10 us: average 1e5 Gy/s, 20 Gy in all), about 7.5e6 species created.
    With the paper's LET a 10 um track deposits 9.6 keV, so about 650 tracks make 1 Gy in
    the 1e-12 kg cube; each pulse's tracks arrive in ``bunches`` equally spaced bunches
    over the pulse (not one by one: every arrival restarts the step at dt_min). Species
    are carried step by step across the intervals; ends 10 us after the last pulse."""
    per_bunch = max(1, tracks_per_pulse // bunches)
    per_track = max(1, species_per_pulse // (per_bunch * bunches))
    pulses = []
    for k in range(n_pulses):
        for q in range(bunches):
            pulses.append(track_pulse(per_bunch, L, per_track, seed, t0=k * period_s + fwhm_s * q / bunches,
                                      stream=20_000 + 100 * k + q))
    return Workload(f"large{n_pulses}_L{int(L)}", L, pulses,
                    Schedule(dt_min=dt_min, dt_max=dt_max, dt_growth=LOG_GROWTH_20_PER_DECADE),
                    t_end=n_pulses * period_s)


def batched_sweep(n_trains: int = 64, seed: int = 0, scale: float = 1.0, t_sim: float = 10e-6,
                  bunches: int = 4, fwhm_s: float = 1e-6, n_min: int = 10_000,
                  n_max: int = 2_000_000) -> List[Workload]:
    """Batched dose-rate sweep, one Workload per train: the trains of ``dose_rate_sweep``
    (species per train log-spaced over [n_min, n_max] * scale, spread over 10 pulses)
    simulated over the same window [0, t_sim). Each square pulse of width fwhm_s is
    delivered as ``bunches`` equally spaced bunches of tracks; pulses repeat with the
    train's period Dp / Dav, so high average dose rates put several pulses (and the
    species they leave behind) into the window."""
    out = []
    for desc in dose_rate_sweep(n_trains, seed, int(n_min * scale), int(n_max * scale),
                                fwhm_s=fwhm_s):
        b = desc["train"]
        L = desc["L"]
        per_pulse = desc["species_per_pulse"]
        n_tracks = max(2, int(round(160 * (L / 5000.0) ** 2)))
        per_track = max(1, per_pulse // n_tracks)
        pulses = []
        k = 0
        while k * desc["period_s"] < t_sim and k < desc["n_pulses"]:
            t0 = k * desc["period_s"]
            for q in range(bunches):
                tb = t0 + fwhm_s * q / bunches
                if tb >= t_sim:
                    break
                pulses.append(track_pulse(max(1, n_tracks // bunches), L, per_track, desc["seed"],
                                          t0=tb, stream=10_000 + 100 * k + q))
            k += 1
        out.append(Workload(f"sweep{b}", L, pulses,
                            Schedule(dt_min=1e-11, dt_max=1e-7, dt_growth=LOG_GROWTH_20_PER_DECADE,
                                     sbs_horizon=desc["sbs_horizon"]),
                            t_end=t_sim))
    return out
