"""FP64 reference ("oracle") of the step-by-step (SBS) chemical stage with periodic
boundaries and pulse injection.

TEST INFRASTRUCTURE ONLY. Nothing in the library imports this module; only the tests,
``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` may use it. It shares
no code with the CUDA path: it receives the same input arrays and computes the method
from the paper's definitions in plain numpy, slowly and in an order a reader can check
against the paper:

* Sec. 2.1 (workflow): species of each radiation event enter the SBS at their sampled
  times and are carried from pulse to pulse.
* Eq. 1 (periodic boundary condition 1): a species leaving [-L/2, L/2) re-enters on the
  opposite side.
* Eq. 2 (periodic boundary condition 2, minimum image): pair separations are taken to
  the nearest image, which is unique because 2R < L.
* Table 1 + Table S2 + Eq. kdiff1/kdiff2 (supplement): every reaction is diffusion
  controlled and its radius follows from k = 4 pi R D_AB N_A, where for the self
  reactions R1, R6 and R8 the tabulated value is already 2k.
* Sec. 2.2 (Fig. PBClattice), Sec. 2.4 and the supplement: two reactants react when
  they come within R.

Where the paper is silent the following readings are used, identically in the library:

* time step: dt starts at dt_min, grows by dt_growth per step up to dt_max, restarts at
  dt_min after a release, is capped so that every cutoff stays <= L/3, and the last
  step of a ``run_until`` is trimmed to land exactly on its end time;
* arrival times are rounded up to the next step boundary; released species get ids in
  (arrival time, caller order) order and diffuse in the step that releases them;
* Brownian displacement: Philox4x32-10 (Salmon et al., SC'11), key = (seed low word,
  seed high word XOR train id), counter = (id, step, 0, tag) for tag 0 and 1, 53-bit
  uniforms, Box-Muller;
* pair search cutoff R_cut = R + c * sqrt(2 D_AB dt); encounters during the step are
  caught by the probability that the pair's relative Brownian path, conditioned on its
  start (d0) and end (d1) separations, touched the reaction sphere:
  p = (exp(-a) - exp(-b)) / (1 - exp(-b)), a = (d0 - R)(d1 - R) / (D_AB dt),
  b = d0 d1 / (D_AB dt) (p = 1 when d0 or d1 <= R), accepted against a uniform drawn
  from counter (id_lo, step, id_hi, 2). This is the ratio of the absorbing-sphere and
  free Green's functions of the angle-averaged relative motion (the image solution
  behind Eq. kdiff1 and Eq. PDF0), so the expected number of reactions per step is that
  of a fully absorbing sphere of radius R, i.e. rate 4 pi R D_AB (1 + R / sqrt(pi D_AB t)),
  at any dt. For R >> sqrt(D_AB dt) it tends to the planar bridge exp(-a);
* one reaction per species per step, closest pair first, lower ids breaking ties;
* products at the diffusion-weighted encounter point, ids assigned in ascending id_lo
  order and table order; products diffuse from the next step;
* optional free-diffusion jump (no reactions) once sbs_horizon has passed since the
  last release, up to the next arrival or the end time;
* the beam-off (homogeneous) stage of Sec. 2.3 with its own readings in
  ``oracle/homogeneous.py``; its survivors are re-created ahead of the pending species
  at the next release.
"""
from __future__ import annotations

import math
from typing import List, Optional, Sequence

import numpy as np
from scipy.spatial import cKDTree

N_AVOGADRO = 6.02214076e23  # 1/mol (exact SI value)
TWO_PI = 2.0 * math.pi
TWO_POW_M53 = math.ldexp(1.0, -53)
END_SLACK = 1.0 + 1e-6

# Philox4x32-10 constants (Salmon et al., SC'11, Sec. 5).
_M0 = np.uint64(0xD2511F53)
_M1 = np.uint64(0xCD9E8D57)
_W0 = np.uint64(0x9E3779B9)
_W1 = np.uint64(0xBB67AE85)
_MASK = np.uint64(0xFFFFFFFF)
_S32 = np.uint64(32)
_S11 = np.uint64(11)


def philox4x32_10(ctr, key):
    """Philox4x32 with 10 rounds. ``ctr`` is 4 arrays (or scalars) of 32-bit words,
    ``key`` 2 words. Each round multiplies words 0 and 2 by the two constants, XORs the
    high halves with words 1, 3 and the key, and the key is bumped by the Weyl
    constants between rounds. Returns 4 uint64 arrays holding 32-bit words."""
    c0, c1, c2, c3 = (np.asarray(c, dtype=np.uint64) & _MASK for c in ctr)
    k0, k1 = (np.asarray(k, dtype=np.uint64) & _MASK for k in key)
    for rnd in range(10):
        if rnd > 0:
            k0 = (k0 + _W0) & _MASK
            k1 = (k1 + _W1) & _MASK
        p0 = _M0 * c0
        p1 = _M1 * c2
        hi0, lo0 = p0 >> _S32, p0 & _MASK
        hi1, lo1 = p1 >> _S32, p1 & _MASK
        c0, c1, c2, c3 = hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0
    return c0, c1, c2, c3


def u53(w_hi, w_lo):
    """53-bit integer from two 32-bit words: the top 53 bits of (w_hi:w_lo)."""
    return ((np.asarray(w_hi, np.uint64) << _S32) | np.asarray(w_lo, np.uint64)) >> _S11


def uniform_open0(w_hi, w_lo):
    """Uniform in (0, 1]: (m + 1) * 2^-53."""
    return (u53(w_hi, w_lo).astype(np.float64) + 1.0) * TWO_POW_M53


def uniform_closed0(w_hi, w_lo):
    """Uniform in [0, 1): m * 2^-53."""
    return u53(w_hi, w_lo).astype(np.float64) * TWO_POW_M53


def philox_key(seed: int, train_id: int):
    seed = int(seed) & 0xFFFFFFFFFFFFFFFF
    return (seed & 0xFFFFFFFF, ((seed >> 32) ^ int(train_id)) & 0xFFFFFFFF)


def gaussians(ids, step: int, key):
    """Three standard normals per species for Brownian step ``step`` (Box-Muller on two
    Philox blocks, tag 0 -> (g0, g1), tag 1 -> g2; the fourth normal is unused)."""
    ids = np.asarray(ids, dtype=np.uint64)
    z = np.zeros_like(ids)
    st = np.full_like(ids, np.uint64(step & 0xFFFFFFFF))
    a0, a1, a2, a3 = philox4x32_10((ids, st, z, z), key)
    b0, b1, b2, b3 = philox4x32_10((ids, st, z, z + np.uint64(1)), key)
    u1 = uniform_open0(a0, a1)
    u2 = uniform_closed0(a2, a3)
    u3 = uniform_open0(b0, b1)
    u4 = uniform_closed0(b2, b3)
    r = np.sqrt(-2.0 * np.log(u1))
    th = TWO_PI * u2
    r2 = np.sqrt(-2.0 * np.log(u3))
    th2 = TWO_PI * u4
    return np.stack([r * np.cos(th), r * np.sin(th), r2 * np.cos(th2)], axis=-1)


def acceptance_uniform(id_lo, id_hi, step: int, key):
    """Uniform in [0, 1) for the pair (id_lo, id_hi) at step ``step``."""
    id_lo = np.asarray(id_lo, dtype=np.uint64)
    id_hi = np.asarray(id_hi, dtype=np.uint64)
    st = np.full_like(id_lo, np.uint64(step & 0xFFFFFFFF))
    c0, c1, _, _ = philox4x32_10((id_lo, st, id_hi, np.full_like(id_lo, np.uint64(2))), key)
    return uniform_closed0(c0, c1)


def touch_probability(d0, d1, R, DABdt):
    """Probability that the relative Brownian path of a pair, started at separation d0
    and ended at d1 after a step with D_AB dt = DABdt, touched the sphere of radius R,
    given only those two separations: 1 - G_abs / G_free with the angle-averaged Green's
    functions of free diffusion and of diffusion outside a fully absorbing sphere (image
    solutions in r times density), i.e. (exp(-a) - exp(-b)) / (1 - exp(-b)) with
    a = (d0 - R)(d1 - R) / DABdt, b = d0 d1 / DABdt; 1 when either end is inside. Written
    as exp(-a) expm1(-c) / expm1(-b), c = b - a = R (d0 + d1 - R) / DABdt."""
    d0 = np.asarray(d0, dtype=np.float64)
    d1 = np.asarray(d1, dtype=np.float64)
    R = np.asarray(R, dtype=np.float64)
    with np.errstate(over="ignore", under="ignore", divide="ignore", invalid="ignore"):
        a = ((d0 - R) * (d1 - R)) / DABdt
        b = (d0 * d1) / DABdt
        c = (R * ((d0 + d1) - R)) / DABdt
        p = np.exp(-a) * (np.expm1(-c) / np.expm1(-b))
    return np.where((d1 <= R) | (d0 <= R), 1.0, p)


def wrap(x, L: float):
    """Eq. 1 (periodic boundary condition 1), applied as many times as needed: shift x
    by whole box lengths into [-L/2, L/2)."""
    x = np.asarray(x, dtype=np.float64)
    k = np.floor((x + 0.5 * L) / L)
    x = x - k * L
    x = np.where(x >= 0.5 * L, x - L, x)
    x = np.where(x < -0.5 * L, x + L, x)
    return x


def minimum_image(dx, L: float):
    """Eq. 2 (periodic boundary condition 2) for a separation of two in-box points."""
    dx = np.asarray(dx, dtype=np.float64)
    dx = np.where(dx >= 0.5 * L, dx - L, dx)
    dx = np.where(dx < -0.5 * L, dx + L, dx)
    return dx


def reaction_radius(k_tab: float, D_AB: float) -> float:
    """Eq. kdiff1 at steady state, k = 4 pi R D_AB N_A, solved for R (nm) with k in
    L/mol/s and D_AB in nm^2/s. For self reactions k_tab is the printed 2k (Eq. kdiff2).
    1 L = 1e24 nm^3."""
    k_nm3_per_s = k_tab * 1e24 / N_AVOGADRO
    return k_nm3_per_s / (4.0 * math.pi * D_AB)


def sq_norm(v):
    return (v[..., 0] * v[..., 0] + v[..., 1] * v[..., 1]) + v[..., 2] * v[..., 2]


class SBSOracle:
    """One pulse train advanced step by step in FP64.

    Parameters mirror the library's configuration: ``D`` (nm^2/s per type), reactions
    as (a, b, k_tab, products, water_delta), box side ``L`` (nm), ``seed``/``train_id``
    (Philox key), the time-step policy and the pair cutoff factor ``cutoff_c``.
    """

    def __init__(self, D: Sequence[float], reactions, L: float, seed: int, train_id: int = 0,
                 dt_min: float = 1e-9, dt_max: float = 1e-9, dt_growth: float = 1.0,
                 reset_on_release: bool = True, cutoff_c: float = 3.0,
                 sbs_horizon: float = 0.0, record: bool = True):
        self.D = np.asarray(D, dtype=np.float64)
        self.n_types = self.D.shape[0]
        self.L = float(L)
        self.key = philox_key(seed, train_id)
        self.dt_min, self.dt_max, self.dt_growth = float(dt_min), float(dt_max), float(dt_growth)
        self.reset_on_release = bool(reset_on_release)
        self.c = float(cutoff_c)
        self.horizon = float(sbs_horizon)
        self.record = record
        # Reaction table (Table 1): type pair -> reaction index, radius, D_AB, products.
        self.rx = []
        self.pair_rxn = -np.ones((self.n_types, self.n_types), dtype=np.int64)
        for r, rx in enumerate(reactions):
            a, b, k_tab, products, water = _unpack_reaction(rx)
            D_AB = self.D[a] + self.D[b]
            R = reaction_radius(k_tab, D_AB)
            if self.pair_rxn[a, b] >= 0:
                raise ValueError("two reactions for one type pair")
            self.pair_rxn[a, b] = self.pair_rxn[b, a] = r
            self.rx.append(dict(a=a, b=b, D_AB=D_AB, R=R, products=tuple(products), water=water,
                                k_tab=float(k_tab)))
        self.n_rxn = len(self.rx)
        self.R = np.array([x["R"] for x in self.rx], dtype=np.float64)
        self.D_AB = np.array([x["D_AB"] for x in self.rx], dtype=np.float64)
        # Largest dt for which every cutoff R + c sqrt(2 D_AB dt) stays <= L/3, which
        # keeps the minimum image (Eq. 2, 2R < L) unambiguous.
        self.dt_L = math.inf
        for x in self.rx:
            room = self.L / 3.0 - x["R"]
            if room <= 0.0:
                raise ValueError("reaction radius too large for the box")
            if self.c > 0.0:
                self.dt_L = min(self.dt_L, (room / self.c) ** 2 / (2.0 * x["D_AB"]))
        # Live species.
        self.ids = np.zeros(0, dtype=np.int64)
        self.types = np.zeros(0, dtype=np.int64)
        self.pos = np.zeros((0, 3), dtype=np.float64)
        # Pending (not yet released) species, kept in (arrival, caller order) order.
        self.p_types = np.zeros(0, dtype=np.int64)
        self.p_pos = np.zeros((0, 3), dtype=np.float64)
        self.p_t = np.zeros(0, dtype=np.float64)
        # Survivors of the last homogeneous stage, re-created as particles at the next
        # release (types in ascending order), and the number of stages taken.
        self.mat_types = np.zeros(0, dtype=np.int64)
        self.hx_stage = 0
        self.t = 0.0
        self.step = 0
        self.dt_cur = self.dt_min
        self.t_last_release = 0.0
        self.next_id = 0
        self.E_dep = 0.0
        self.water = 0
        self.species_steps = 0
        self.events_total = np.zeros(self.n_rxn, dtype=np.int64)
        self.event_log: List[tuple] = []      # (step, rxn, id_lo, id_hi, prod_id0, n_prod)
        self.step_log: List[tuple] = []       # (step, t_start, dt, n_live, counts...)

    # -- inputs ------------------------------------------------------------------
    def inject(self, types, xyz, t_arrival, energy_eV: float = 0.0):
        types = np.asarray(types, dtype=np.int64)
        xyz = np.asarray(xyz, dtype=np.float64).reshape(-1, 3)
        t_arrival = np.asarray(t_arrival, dtype=np.float64)
        if np.any(~(t_arrival >= self.t)):
            raise ValueError("arrival before the current time or not a number")
        if np.any((types < 0) | (types >= self.n_types)):
            raise ValueError("bad species type")
        if np.any(~((xyz >= -0.5 * self.L) & (xyz < 0.5 * self.L))):
            raise ValueError("position outside the box or not a number")
        self.E_dep += float(energy_eV)
        all_t = np.concatenate([self.p_t, t_arrival])
        order = np.argsort(all_t, kind="stable")
        self.p_t = all_t[order]
        self.p_types = np.concatenate([self.p_types, types])[order]
        self.p_pos = np.concatenate([self.p_pos, xyz])[order]

    # -- one SBS step --------------------------------------------------------------
    def _release(self):
        n = int(np.searchsorted(self.p_t, self.t, side="right"))
        m = self.mat_types.shape[0]
        if n + m == 0:
            return 0
        if m:
            # survivors of a homogeneous stage first, at uniform positions
            from .homogeneous import materialised_positions
            mat_ids = np.arange(self.next_id, self.next_id + m, dtype=np.int64)
            self.next_id += m
            self.ids = np.concatenate([self.ids, mat_ids])
            self.types = np.concatenate([self.types, self.mat_types])
            self.pos = np.concatenate([self.pos, materialised_positions(mat_ids, self.L, self.key)])
            self.mat_types = np.zeros(0, dtype=np.int64)
        new_ids = np.arange(self.next_id, self.next_id + n, dtype=np.int64)
        self.next_id += n
        self.ids = np.concatenate([self.ids, new_ids])
        self.types = np.concatenate([self.types, self.p_types[:n]])
        self.pos = np.concatenate([self.pos, self.p_pos[:n]])
        self.p_t, self.p_types, self.p_pos = self.p_t[n:], self.p_types[n:], self.p_pos[n:]
        self.t_last_release = self.t
        if self.reset_on_release:
            self.dt_cur = self.dt_min
        return n + m

    def _choose_dt(self, t_end: float):
        next_arrival = self.p_t[0] if self.p_t.shape[0] else math.inf
        free = (self.horizon > 0.0 and (self.t - self.t_last_release) >= self.horizon
                and next_arrival > self.t)
        if free:
            t_next = min(t_end, next_arrival)
            return t_next - self.t, t_next, True
        dt = min(self.dt_cur, self.dt_L)
        # Land exactly on t_end when it is less than a step (plus a 1e-6 relative slack
        # so that accumulated rounding never leaves a sliver step).
        if t_end - self.t <= dt * END_SLACK:
            return t_end - self.t, t_end, False
        return dt, self.t + dt, False

    def candidates(self, delta, dt):
        """Accepted reactive pairs of this step (Sec. 2.4 criterion with the bridge
        reading). Returns arrays (lo, hi, rxn, d1sq, r1) with lo/hi indices into the live
        arrays ordered so that ids[lo] < ids[hi]."""
        N = self.ids.shape[0]
        empty = (np.zeros(0, np.int64),) * 3 + (np.zeros(0), np.zeros((0, 3)))
        if N < 2 or self.n_rxn == 0:
            return empty
        R_cut = self.R + self.c * np.sqrt(2.0 * self.D_AB * dt)
        r_query = float(R_cut.max()) * (1.0 + 1e-9) + 1e-9
        pairs = all_pairs_within(self.pos, self.L, r_query)
        if pairs.shape[0] == 0:
            return empty
        i, j = pairs[:, 0], pairs[:, 1]
        rxn = self.pair_rxn[self.types[i], self.types[j]]
        keep = rxn >= 0
        i, j, rxn = i[keep], j[keep], rxn[keep]
        swap = self.ids[i] > self.ids[j]
        lo = np.where(swap, j, i)
        hi = np.where(swap, i, j)
        r1 = minimum_image(self.pos[hi] - self.pos[lo], self.L)
        d1sq = sq_norm(r1)
        rc = R_cut[rxn]
        keep = d1sq < rc * rc
        lo, hi, rxn, d1sq, r1 = lo[keep], hi[keep], rxn[keep], d1sq[keep], r1[keep]
        R = self.R[rxn]
        d1 = np.sqrt(d1sq)
        r0 = r1 - (delta[hi] - delta[lo])
        d0 = np.sqrt(sq_norm(r0))
        p = touch_probability(d0, d1, R, self.D_AB[rxn] * dt)
        u = acceptance_uniform(self.ids[lo], self.ids[hi], self.step, self.key)
        keep = u < p
        return lo[keep], hi[keep], rxn[keep], d1sq[keep], r1[keep]

    def step_once(self, t_end: float):
        self._release()
        dt, t_next, free = self._choose_dt(t_end)
        n_live = self.ids.shape[0]
        self.species_steps += n_live
        t_start = self.t
        # Brownian displacement (Sec. 2.1 SBS) and Eq. 1.
        if n_live:
            g = gaussians(self.ids, self.step, self.key)
            s = np.sqrt(2.0 * self.D[self.types] * dt)
            delta = s[:, None] * g
            self.pos = wrap(self.pos + delta, self.L)
        else:
            delta = np.zeros((0, 3))
        n_events = 0
        if not free and n_live >= 2:
            lo, hi, rxn, d1sq, r1 = self.candidates(delta, dt)
            committed = greedy_matching(self.ids[lo], self.ids[hi], d1sq)
            taken = np.zeros(n_live, dtype=bool)
            taken[lo[committed]] = True
            taken[hi[committed]] = True
            committed = sorted(committed, key=lambda c: self.ids[lo[c]])
            new_ids, new_types, new_pos = [], [], []
            for c in committed:
                a, b, r = lo[c], hi[c], int(rxn[c])
                rx = self.rx[r]
                ta, tb = self.types[a], self.types[b]
                w = self.D[ta] / (self.D[ta] + self.D[tb])
                P = wrap(self.pos[a] + w * r1[c], self.L)
                first = self.next_id
                for pt in rx["products"]:
                    new_ids.append(self.next_id)
                    new_types.append(pt)
                    new_pos.append(P)
                    self.next_id += 1
                self.water += rx["water"]
                self.events_total[r] += 1
                if self.record:
                    self.event_log.append((self.step, r, int(self.ids[a]), int(self.ids[b]),
                                           first, len(rx["products"])))
            n_events = len(committed)
            if n_events:
                keep = ~taken
                self.ids = np.concatenate([self.ids[keep], np.asarray(new_ids, np.int64)])
                self.types = np.concatenate([self.types[keep], np.asarray(new_types, np.int64)])
                pos_new = np.asarray(new_pos, np.float64).reshape(-1, 3)
                self.pos = np.concatenate([self.pos[keep], pos_new])
        if self.record:
            self.step_log.append((self.step, t_start, dt, n_live, n_events) +
                                 tuple(int(c) for c in self.counts()))
        self.t = t_next
        self.step += 1
        self.dt_cur = min(self.dt_cur * self.dt_growth, self.dt_max)

    def run_until(self, t_end: float, max_steps: Optional[int] = None):
        n = 0
        while self.t < t_end and (max_steps is None or n < max_steps):
            self.step_once(t_end)
            n += 1
        return n

    # -- homogeneous stage (Sec. 2.3) ------------------------------------------------
    def run_homogeneous(self, t_end: float):
        """Beam-off stage: the species (and pending ones already due) become molecule
        numbers, the rate equations of Table 1 (Eq. 3, Eq. 4) run for t_end - t, and the
        survivors wait to be re-created uniformly at the next step (see
        ``oracle/homogeneous.py`` for the readings). Returns (e, E): real extents and
        integer events of the stage."""
        from .homogeneous import stage, water_change
        if not (t_end > self.t):
            return None
        n_due = int(np.searchsorted(self.p_t, self.t, side="right"))
        if n_due < self.p_t.shape[0] and self.p_t[n_due] < t_end:
            raise ValueError("species arrive during the homogeneous stage")
        n0 = self.counts() + np.bincount(self.p_types[:n_due], minlength=self.n_types)
        self.p_t, self.p_types, self.p_pos = (self.p_t[n_due:], self.p_types[n_due:],
                                              self.p_pos[n_due:])
        reactions = [(x["a"], x["b"], x["k_tab"], x["products"], x["water"]) for x in self.rx]
        e, E, n = stage(n0, self.L, t_end - self.t, reactions, self.hx_stage, self.key)
        self.hx_stage += 1
        self.events_total += E
        self.water += water_change(E, reactions)
        self.ids = np.zeros(0, dtype=np.int64)
        self.types = np.zeros(0, dtype=np.int64)
        self.pos = np.zeros((0, 3), dtype=np.float64)
        self.mat_types = np.repeat(np.arange(self.n_types, dtype=np.int64), n)
        self.t = float(t_end)
        return e, E

    # -- outputs -------------------------------------------------------------------
    def counts(self):
        return (np.bincount(self.types, minlength=self.n_types) +
                np.bincount(self.mat_types, minlength=self.n_types)).astype(np.int64)

    def g_values(self):
        """G = molecules per 100 eV deposited."""
        if self.E_dep <= 0.0:
            return np.zeros(self.n_types)
        return self.counts().astype(np.float64) * 100.0 / self.E_dep

    def state(self):
        """Live species sorted by id: (ids, types, positions)."""
        o = np.argsort(self.ids)
        return self.ids[o], self.types[o], self.pos[o]

    def events(self):
        return np.asarray(self.event_log, dtype=np.int64).reshape(-1, 6)

    def steps(self):
        return np.asarray([s[:1] + s[3:] for s in self.step_log], dtype=np.int64).reshape(
            -1, 3 + self.n_types)


def greedy_matching(id_lo, id_hi, d1sq):
    """One reaction per species: walk the accepted pairs by increasing (d1^2, id_lo,
    id_hi) and keep a pair when neither species is already taken. Returns the indices
    of the kept pairs."""
    order = np.lexsort((np.asarray(id_hi), np.asarray(id_lo), np.asarray(d1sq)))
    taken = set()
    kept = []
    for c in order:
        a, b = int(id_lo[c]), int(id_hi[c])
        if a not in taken and b not in taken:
            taken.add(a)
            taken.add(b)
            kept.append(int(c))
    return np.asarray(kept, dtype=np.int64)


def all_pairs_within(pos, L: float, r: float):
    """All unordered index pairs whose periodic distance is <= r (a periodic k-d tree
    from scipy as the pair-finding library primitive)."""
    q = np.asarray(pos, dtype=np.float64) + 0.5 * L
    q = np.where(q >= L, q - L, q)
    q = np.where(q < 0.0, 0.0, q)
    tree = cKDTree(q, boxsize=L)
    return tree.query_pairs(r, output_type="ndarray").astype(np.int64).reshape(-1, 2)


def all_pairs_within_bruteforce(pos, L: float, r: float):
    """Same set as ``all_pairs_within`` by checking every pair (small inputs only)."""
    pos = np.asarray(pos, dtype=np.float64)
    n = pos.shape[0]
    out = []
    for i in range(n):
        d = minimum_image(pos[i + 1:] - pos[i], L)
        js = np.nonzero(sq_norm(d) <= r * r)[0]
        out.extend((i, i + 1 + j) for j in js)
    return np.asarray(out, dtype=np.int64).reshape(-1, 2)


def _unpack_reaction(rx):
    if hasattr(rx, "a"):
        return rx.a, rx.b, rx.k_tab, rx.products, rx.water_delta
    if isinstance(rx, dict):
        return rx["a"], rx["b"], rx["k_tab"], rx["products"], rx.get("water_delta", 0)
    a, b, k_tab, products, water = rx
    return a, b, k_tab, products, water


def from_workload(wl, seed: int, train_id: int = 0, record: bool = True) -> SBSOracle:
    """Build an oracle for a ``workloads.Workload`` and inject all its pulses."""
    s = wl.schedule
    o = SBSOracle(wl.D, wl.reactions, wl.L, seed, train_id, s.dt_min, s.dt_max, s.dt_growth,
                  s.reset_on_release, s.cutoff_c, s.sbs_horizon, record)
    for p in wl.pulses:
        o.inject(p.types, p.xyz, p.t_arrival, p.energy_eV)
    return o
