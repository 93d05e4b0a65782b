"""Pulse trains that alternate the step-by-step stage and the rate equations (Sec. 2.1
workflow, Sec. 2.3 rate equations):
the step-by-step (SBS) chemistry runs while the beam is on, the rate equations of Table 1
(Eq. 3, Eq. 4) for the rest of the beam-off time up to the next pulse, and after the last
pulse for 10 s. Every step of both stages runs in the CUDA library; this module only
sequences the calls for the trains of a batched context and reads their tallies.

The post-irradiation analysis of Sec. 3.3 (the H2O2 yield as the slope of its
post-irradiation concentration against dose, Fig. Concentration-Dose and Fig.
G-yield_Dav, and the average dose rate above which radicals build up from pulse to pulse)
works on those tallies on the host.
"""
from __future__ import annotations

import time
from typing import List, Sequence

import numpy as np

from . import chem

N_AVOGADRO = 6.02214076e23
MOL_PER_J_PER_MOLECULE_PER_100EV = 1.0 / (N_AVOGADRO * 100.0 * 1.602176634e-19)


def run_plans(ctx, plans: Sequence[Sequence[tuple]], n_types: int = 7, n_rxn: int = 9):
    """Advance every train b of the batched context through plans[b], a list of
    (kind, t_end) calls with kind "sbs" (chem_batch_run_until) or "ode"
    (chem_batch_run_homogeneous). Call i of all plans runs together: trains whose call i
    is of the other kind, or whose plan has ended, are given an end time of 0 (no-op).

    Returns a dict: ``counts`` [calls, trains, n_types] and ``events`` [calls, trains,
    n_rxn] after every call, ``extents`` [calls, trains, n_rxn] (the real extents of an
    "ode" call, else 0), ``t`` [calls, trains], ``kinds`` [calls][trains] (None past the
    end), wall seconds per kind (``seconds``), and the species-steps of the run."""
    B = len(plans)
    n_calls = max(len(p) for p in plans) if plans else 0
    counts = np.zeros((n_calls, B, n_types), np.int64)
    events = np.zeros((n_calls, B, n_rxn), np.int64)
    extents = np.zeros((n_calls, B, n_rxn))
    tt = np.zeros((n_calls, B))
    kinds: List[List] = []
    seconds = {"sbs": 0.0, "ode": 0.0}
    ss0 = sum(chem.chem_batch_tally(ctx, b, n_types, n_rxn)["species_steps"] for b in range(B))
    for i in range(n_calls):
        row = [p[i][0] if i < len(p) else None for p in plans]
        kinds.append(row)
        for kind in ("sbs", "ode"):
            if kind not in row:
                continue
            ends = np.array([p[i][1] if row[b] == kind else 0.0 for b, p in enumerate(plans)])
            t0 = time.perf_counter()
            if kind == "sbs":
                chem.chem_batch_run_until(ctx, ends)
            else:
                chem.chem_batch_run_homogeneous(ctx, ends)
            seconds[kind] += time.perf_counter() - t0
        for b in range(B):
            tal = chem.chem_batch_tally(ctx, b, n_types, n_rxn)
            counts[i, b] = tal["counts"][:n_types]
            events[i, b] = tal["events"][:n_rxn]
            tt[i, b] = tal["t"]
            if row[b] == "ode":
                extents[i, b] = chem.chem_batch_homogeneous_report(ctx, b)[0][:n_rxn]
    ss1 = sum(chem.chem_batch_tally(ctx, b, n_types, n_rxn)["species_steps"] for b in range(B))
    return {"counts": counts, "events": events, "extents": extents, "t": tt, "kinds": kinds,
            "seconds": seconds, "species_steps": ss1 - ss0}


def stoichiometry(n_types: int, reactions):
    """nu[x, r]: change of species x per event of reaction r (reactants -1 each, products
    +1 each)."""
    nu = np.zeros((n_types, len(reactions)), np.int64)
    for r, rx in enumerate(reactions):
        nu[rx.a, r] -= 1
        nu[rx.b, r] -= 1
        for p in rx.products:
            nu[p, r] += 1
    return nu


def concentration(count, L_nm: float):
    """Molecules in a cube of side L (nm) -> mol/L (1 L = 1e24 nm^3)."""
    return np.asarray(count, dtype=np.float64) / (N_AVOGADRO * L_nm ** 3 * 1e-24)


def dose_slope_yield(dose_Gy, conc_mol_per_L):
    """Yield as the least-squares slope of post-irradiation concentration against dose,
    the way Sec. 3.3 derives the H2O2 yield from Fig. Concentration-Dose. With water at
    1 kg/L the slope in (mol/L)/Gy is mol/J; returned in mol/J and in molecules/100 eV."""
    d = np.asarray(dose_Gy, dtype=np.float64)
    c = np.asarray(conc_mol_per_L, dtype=np.float64)
    dm, cm = d.mean(), c.mean()
    slope = float(((d - dm) * (c - cm)).sum() / ((d - dm) ** 2).sum())
    return slope, slope / MOL_PER_J_PER_MOLECULE_PER_100EV


def buildup_fraction(run, radicals: Sequence[int] = (0, 1, 2), nu=None):
    """Per train, the radicals (e_aq, OH, H by default) left when the next pulse starts,
    as a fraction of those present when the previous beam-on stage ended, for the last
    inter-pulse interval of its plan. Near 0: steady state reached between pulses;
    large: the radicals build up (Sec. 3.3). With the stoichiometry ``nu`` the numbers left
    are the rate equations' real ones (before the rounding to whole events, whose +-1
    noise would dominate in small boxes), else the whole counts."""
    kinds, counts = run["kinds"], run["counts"]
    B = counts.shape[1]
    out = np.full(B, np.nan)
    for b in range(B):
        seq = [i for i in range(len(kinds)) if kinds[i][b] is not None]
        # the last "ode" that is followed by an "sbs" (an interval between two pulses)
        for j in range(len(seq) - 2, 0, -1):
            i_ode, i_sbs = seq[j], seq[j + 1]
            if kinds[i_ode][b] == "ode" and kinds[i_sbs][b] == "sbs" and kinds[seq[j - 1]][b] == "sbs":
                before = counts[seq[j - 1], b, list(radicals)].sum()
                if nu is not None:
                    real = counts[seq[j - 1], b] + np.asarray(nu) @ run["extents"][i_ode, b]
                    after = max(0.0, float(real[list(radicals)].sum()))
                else:
                    after = counts[i_ode, b, list(radicals)].sum()
                out[b] = after / before if before > 0 else 0.0
                break
    return out


def threshold_dose_rate(avg_dose_rates, fractions, level: float = 0.01):
    """Lowest average dose rate whose build-up fraction exceeds ``level`` (the SDR/UHDR
    threshold of Sec. 3.3, read as: radicals no longer fall below ``level`` of their
    end-of-pulse number before the next pulse), or None."""
    dav = np.asarray(avg_dose_rates, dtype=np.float64)
    f = np.asarray(fractions, dtype=np.float64)
    over = np.nonzero(f > level)[0]
    if over.size == 0:
        return None
    return float(dav[over].min())
