"""Homogeneous rate equations (Eq. 3, Eq. 4) — a fixed point for the SBS reference.

TEST INFRASTRUCTURE ONLY (see ``oracle/sbs.py``).

For a reaction A + B with tabulated rate k_tab the event rate per litre is
k_tab [A][B] (Eq. rateequation). For a self reaction A + A the table prints 2k and the
event rate is k [A]^2 = (k_tab / 2) [A]^2, each event removing two A, so that
-d[A]/dt = k_tab [A]^2 (Eq. 3 with its "-2 R1" term and Eq. 4, Eq. rateequation2).
With ``transient=True`` every k is multiplied by the Smoluchowski factor
1 + R / sqrt(pi D_AB t) of Eq. kdiff1, which is what a particle simulation started
from a uniform, unreacted mixture reproduces at early times.
"""
from __future__ import annotations

import math

import numpy as np
from scipy.integrate import solve_ivp

from .sbs import N_AVOGADRO, reaction_radius


def _unpack(rx):
    if hasattr(rx, "a"):
        return rx.a, rx.b, rx.k_tab, tuple(rx.products)
    if isinstance(rx, dict):
        return rx["a"], rx["b"], rx["k_tab"], tuple(rx["products"])
    return rx[0], rx[1], rx[2], tuple(rx[3])


def rates(conc, t, D, reactions, transient=False):
    """d[X]/dt in mol/L/s for concentrations ``conc`` (mol/L) at time t (s)."""
    dcdt = np.zeros_like(conc)
    for rx in reactions:
        a, b, k_tab, products = _unpack(rx)
        k = k_tab
        if transient and t > 0.0:
            D_AB = D[a] + D[b]
            R = reaction_radius(k_tab, D_AB)
            k = k_tab * (1.0 + R / math.sqrt(math.pi * D_AB * t))
        if a == b:
            nu = 0.5 * k * conc[a] * conc[a]
        else:
            nu = k * conc[a] * conc[b]
        dcdt[a] -= nu
        dcdt[b] -= nu
        for p in products:
            dcdt[p] += nu
    return dcdt


def integrate(conc0, t_eval, D, reactions, transient=False, method="LSODA", rtol=1e-10,
              atol=1e-22):
    """Concentrations (mol/L) at the times ``t_eval`` (s, ascending, >= 0)."""
    conc0 = np.asarray(conc0, dtype=np.float64)
    t_eval = np.asarray(t_eval, dtype=np.float64)
    t0 = 0.0
    if transient:
        # The transient factor diverges like t^-1/2 at t = 0 (integrable); start just after.
        t0 = min(1e-18, 1e-6 * t_eval[t_eval > 0].min()) if np.any(t_eval > 0) else 0.0
    sol = solve_ivp(lambda t, y: rates(y, t, D, reactions, transient), (t0, float(t_eval[-1])),
                    conc0, t_eval=np.maximum(t_eval, t0), method=method, rtol=rtol, atol=atol)
    if not sol.success:
        raise RuntimeError(sol.message)
    return sol.y.T


def molar(count, L_nm: float):
    """Species count in a cube of side L (nm) -> concentration in mol/L (1 L = 1e24 nm^3)."""
    return np.asarray(count, dtype=np.float64) / (N_AVOGADRO * L_nm ** 3 * 1e-24)
