"""Well-mixed stochastic reference for the volume-scaling study (Sec. 2.2 setup and
Sec. 3.1 results of the verification of the periodic boundary conditions): the paper compares the SBS in boxes of 0.2, 0.5 and
1.0 um with Kinetiscope, which runs Gillespie's stochastic simulation algorithm. This is
an independent implementation of that algorithm (the direct method of Gillespie, J.
Phys. Chem. 81, 2340, 1977) for the reaction table of Table 1.

TEST INFRASTRUCTURE ONLY (see ``oracle/sbs.py``).

Propensities in the box volume V (N_A V molecules per mol/L): a reaction A + B of rate
constant k fires at k / (N_A V) * n_A n_B per second; a self reaction A + A whose table
value k_tab is 2k fires at (k_tab / 2) / (N_A V) * n_A (n_A - 1) per second, the
number of distinct pairs n_A (n_A - 1) / 2 times the pair rate k_tab / (N_A V). For large
numbers both tend to the rate equations Eq. 3 / Eq. 4. The waiting time to the next event
is exponential with the total propensity; the event is drawn in proportion to its
propensity.
"""
from __future__ import annotations

import math

import numpy as np

from .sbs import N_AVOGADRO


def _unpack(rx):
    if hasattr(rx, "a"):
        return rx.a, rx.b, rx.k_tab, tuple(rx.products), getattr(rx, "water_delta", 0)
    if len(rx) == 4:
        return rx[0], rx[1], rx[2], tuple(rx[3]), 0
    return rx[0], rx[1], rx[2], tuple(rx[3]), rx[4]


def ssa(n0, L_nm: float, reactions, t_points, seed: int, max_events: int = 50_000_000):
    """Counts at the (ascending) times t_points, water change and event counts, from one
    run of the direct method started at t = 0 with counts n0."""
    rng = np.random.default_rng(seed)
    n = np.asarray(n0, dtype=np.int64).copy()
    NV = N_AVOGADRO * L_nm ** 3 * 1e-24
    rx = [_unpack(r) for r in reactions]
    c = np.array([(0.5 * k if a == b else k) / NV for a, b, k, _, _ in rx])
    nu = np.zeros((n.shape[0], len(rx)), dtype=np.int64)
    for r, (a, b, _, prods, _) in enumerate(rx):
        nu[a, r] -= 1
        nu[b, r] -= 1
        for p in prods:
            nu[p, r] += 1
    water_r = np.array([w for *_, w in rx], dtype=np.int64)
    A = np.array([a for a, *_ in rx])
    B = np.array([b for _, b, *_ in rx])
    self_r = A == B
    t = 0.0
    out = np.zeros((len(t_points), n.shape[0]), dtype=np.int64)
    events = np.zeros(len(rx), dtype=np.int64)
    k = 0
    for _ in range(max_events):
        prop = np.where(self_r, c * n[A] * (n[A] - 1), c * n[A] * n[B])
        a0 = float(prop.sum())
        if a0 <= 0.0:
            break
        tau = -math.log(1.0 - rng.random()) / a0
        while k < len(t_points) and t_points[k] < t + tau:
            out[k] = n
            k += 1
        if k == len(t_points):
            break
        t += tau
        r = int(np.searchsorted(np.cumsum(prop), rng.random() * a0, side="right"))
        r = min(r, len(rx) - 1)
        n += nu[:, r]
        events[r] += 1
    while k < len(t_points):
        out[k] = n
        k += 1
    return out, int(events @ water_r), events
