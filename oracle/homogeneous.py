"""Homogeneous stage of a pulse train (Sec. 2.1 workflow, Sec. 2.3 rate equations
Eq. 3 / Eq. 4) in plain FP64 numpy/scipy.

TEST INFRASTRUCTURE ONLY (see ``oracle/sbs.py``).

During the beam-off time the paper stops following particles and integrates the
empirical rate equations of the well-mixed system until the next pulse (and for 10 s
after the last one). The paper gives the equations (every reaction of Table 1
contributes its rate k [A][B], a self reaction A + A its k [A]^2 with the tabulated
value being 2k, Eq. 3 and Eq. 4) but not how particles are turned into concentrations
and back. The readings used here, identically in the library:

* the stage starts from the train's species counts n0 (live species plus pending ones
  already due) in the box volume V = L^3; every particle is removed;
* the rate equations are integrated for the reaction extents e_r, counted in events
  (molecules) rather than mol/L: n(e) = n0 + nu e, rate_r = kappa_r n_a n_b with
  kappa_r = k_r / (N_A V), and for a self reaction rate_r = (k_tab / 2) / (N_A V) n_a^2
  (two A removed per event), which is Eq. 3 multiplied through by N_A V;
* the real extents are rounded to whole events without bias, E_r = floor(e_r) + [u_r <
  frac(e_r)], with u_r from Philox4x32-10 at counter (stage, r, 0, 4) of the train's
  key; where a species would go negative, events of the lowest-index reaction that
  consumes it are taken back one at a time (lowest negative species first) until no
  count is negative;
* the counts n0 + nu E, the event tallies and the water balance are updated with the
  integer events, so charge and atoms stay exactly conserved;
* the survivors are re-created as particles at uniform positions when the train takes
  its next SBS step: in ascending type order, ids from the train's next id, position
  -L/2 + L u wrapped by Eq. 1 with u from counter (id, 0, 0, 3) words (0,1) -> x,
  (2,3) -> y and counter (id, 1, 0, 3) words (0,1) -> z.
"""
from __future__ import annotations

import math

import numpy as np
from scipy.integrate import solve_ivp

from .sbs import N_AVOGADRO, philox4x32_10, uniform_closed0, wrap

TAG_MATERIALISE = 3
TAG_ROUNDING = 4


def _unpack(rx):
    if hasattr(rx, "a"):
        return rx.a, rx.b, rx.k_tab, tuple(rx.products), getattr(rx, "water_delta", 0)
    if isinstance(rx, dict):
        return rx["a"], rx["b"], rx["k_tab"], tuple(rx["products"]), rx.get("water_delta", 0)
    if len(rx) == 4:
        return rx[0], rx[1], rx[2], tuple(rx[3]), 0
    return rx[0], rx[1], rx[2], tuple(rx[3]), rx[4]


def stoichiometry(n_types: int, reactions):
    """nu[x, r]: change of species x per event of reaction r (Table 1)."""
    nu = np.zeros((n_types, len(reactions)), dtype=np.int64)
    for r, rx in enumerate(reactions):
        a, b, _, products, _ = _unpack(rx)
        nu[a, r] -= 1
        nu[b, r] -= 1
        for p in products:
            nu[p, r] += 1
    return nu


def event_rate_constants(reactions, L_nm: float):
    """kappa_r in events per second per molecule pair in the box of side L (nm):
    k / (N_A V) for A + B, (k_tab / 2) / (N_A V) for A + A (1 L = 1e24 nm^3)."""
    NV = N_AVOGADRO * L_nm ** 3 * 1e-24
    out = []
    for rx in reactions:
        a, b, k_tab, _, _ = _unpack(rx)
        out.append((0.5 * k_tab if a == b else k_tab) / NV)
    return np.asarray(out, dtype=np.float64)


def event_rates(n, reactions, kappa):
    """Events per second of every reaction at molecule numbers n (Eq. 3, Eq. 4)."""
    out = np.zeros(len(reactions))
    for r, rx in enumerate(reactions):
        a, b, _, _, _ = _unpack(rx)
        out[r] = kappa[r] * n[a] * n[b]
    return out


def extents(n0, L_nm: float, T: float, reactions, method: str = "Radau", rtol: float = 1e-12,
            atol: float = 1e-9):
    """Reaction extents e_r (events, real) after integrating the rate equations for T
    seconds from molecule numbers n0 (scipy's stiff integrator as the library primitive)."""
    n0 = np.asarray(n0, dtype=np.float64)
    nu = stoichiometry(n0.shape[0], reactions).astype(np.float64)
    kappa = event_rate_constants(reactions, L_nm)
    n_rxn = len(reactions)
    if n_rxn == 0 or T <= 0.0:
        return np.zeros(n_rxn)

    def f(_t, e):
        return event_rates(n0 + nu @ e, reactions, kappa)

    def jac(_t, e):
        n = n0 + nu @ e
        dr_dn = np.zeros((n_rxn, n0.shape[0]))
        for r, rx in enumerate(reactions):
            a, b, _, _, _ = _unpack(rx)
            dr_dn[r, a] += kappa[r] * n[b]
            dr_dn[r, b] += kappa[r] * n[a]
        return dr_dn @ nu

    sol = solve_ivp(f, (0.0, float(T)), np.zeros(n_rxn), method=method, rtol=rtol, atol=atol,
                    jac=jac if method in ("Radau", "BDF", "LSODA") else None)
    if not sol.success:
        raise RuntimeError(sol.message)
    return sol.y[:, -1].copy()


def rounding_uniforms(n_rxn: int, stage: int, key):
    """u_r in [0, 1) for the unbiased rounding of stage ``stage``: counter (stage, r, 0, 4)."""
    r = np.arange(n_rxn, dtype=np.uint64)
    st = np.full_like(r, np.uint64(stage & 0xFFFFFFFF))
    z = np.zeros_like(r)
    w0, w1, _, _ = philox4x32_10((st, r, z, z + np.uint64(TAG_ROUNDING)), key)
    return uniform_closed0(w0, w1)


def integer_events(e, u, n0, nu):
    """Whole events from the real extents: unbiased rounding, then events of the
    lowest-index consuming reaction taken back while any count is negative (lowest
    negative species first). Returns (E, n)."""
    e = np.maximum(np.asarray(e, dtype=np.float64), 0.0)
    fl = np.floor(e)
    E = (fl + (np.asarray(u) < e - fl)).astype(np.int64)
    n0 = np.asarray(n0, dtype=np.int64)
    n = n0 + nu @ E
    while np.any(n < 0):
        x = int(np.nonzero(n < 0)[0][0])
        r = int(np.nonzero((nu[x] < 0) & (E > 0))[0][0])
        E[r] -= 1
        n = n0 + nu @ E
    return E, n


def materialised_positions(ids, L: float, key):
    """Uniform positions of re-created particles: counter (id, 0, 0, 3) words (0,1) -> x,
    (2,3) -> y; counter (id, 1, 0, 3) words (0,1) -> z; x = -L/2 + L u, Eq. 1 wrap."""
    ids = np.asarray(ids, dtype=np.uint64)
    z = np.zeros_like(ids)
    tag = z + np.uint64(TAG_MATERIALISE)
    a0, a1, a2, a3 = philox4x32_10((ids, z, z, tag), key)
    b0, b1, _, _ = philox4x32_10((ids, z + np.uint64(1), z, tag), key)
    u = np.stack([uniform_closed0(a0, a1), uniform_closed0(a2, a3), uniform_closed0(b0, b1)],
                 axis=-1)
    return wrap(-0.5 * L + L * u, L)


def stage(n0, L_nm: float, T: float, reactions, stage_index: int, key):
    """One homogeneous stage: (e, E, n) = real extents, integer events, counts after."""
    n0 = np.asarray(n0, dtype=np.int64)
    nu = stoichiometry(n0.shape[0], reactions)
    e = extents(n0.astype(np.float64), L_nm, T, reactions)
    u = rounding_uniforms(len(reactions), stage_index, key)
    E, n = integer_events(e, u, n0, nu)
    return e, E, n


def water_change(E, reactions):
    return int(sum(int(E[r]) * int(_unpack(rx)[4]) for r, rx in enumerate(reactions)))
