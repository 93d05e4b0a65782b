"""The plain FP64 C++ reference of the SBS stage (``oracle/csrc/sbs_oracle.cpp``) behind
the same Python interface as ``oracle.sbs``.

TEST INFRASTRUCTURE ONLY: imported by the tests and the CPU-baseline legs of
``bench.py``; never by the library. The C++ program computes what ``oracle/sbs.py``
computes, from the same passages of the paper (Sec. 2.1 workflow, Eq. 1, Eq. 2, Sec. 2.4
with Table 1 and Eq. kdiff1/kdiff2) and the same readings, single-threaded in FP64 with
no fused multiply-add. The two references share no code: this module only moves arrays
across the C boundary. ``build()`` compiles the program in-tree with the host compiler
(it is the checker, so building it is not using it); ``load()`` builds it when missing.

What the C++ program does not hold: the beam-off stage of Sec. 2.3
(``run_homogeneous``), which stays in ``oracle/homogeneous.py``.
"""
from __future__ import annotations

import ctypes as C
import os
import shutil
import subprocess
import threading
from typing import Optional, Sequence

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SOURCE = os.path.join(HERE, "csrc", "sbs_oracle.cpp")
OUT_DIR = os.path.join(HERE, "_build")
LIBRARY = os.path.join(OUT_DIR, "libsbs_oracle.so")
FLAGS = ["-O2", "-std=c++17", "-ffp-contract=off", "-fno-fast-math", "-shared", "-fPIC"]

_lib = None
_lock = threading.Lock()


def compiler() -> str:
    for c in (os.environ.get("CXX", ""), shutil.which("g++") or "", shutil.which("c++") or ""):
        if c and os.path.exists(c):
            return c
    raise RuntimeError("no C++ compiler found for the reference program")


def build(force: bool = False) -> str:
    """Compile the reference program into oracle/_build (skipped when up to date)."""
    if not force and os.path.exists(LIBRARY) and os.path.getmtime(LIBRARY) >= os.path.getmtime(SOURCE):
        return LIBRARY
    os.makedirs(OUT_DIR, exist_ok=True)
    tmp = f"{LIBRARY}.{os.getpid()}.tmp"
    r = subprocess.run([compiler(), *FLAGS, SOURCE, "-o", tmp], capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"building the reference program failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, LIBRARY)
    return LIBRARY


class _Reaction(C.Structure):
    _fields_ = [("a", C.c_int32), ("b", C.c_int32), ("k_tab", C.c_double), ("n_prod", C.c_int32),
                ("prod", C.c_int32 * 3), ("water_delta", C.c_int32)]


_P = C.c_void_p
_I64, _I32, _U32, _F64 = C.c_int64, C.c_int32, C.c_uint32, C.c_double
_SIGS = {
    "oracle_new": (_P, [_I32, _P, _I32, _P, _F64, C.c_uint64, _U32, _F64, _F64, _F64, _I32, _F64, _F64, _I32]),
    "oracle_free": (None, [_P]),
    "oracle_inject": (_I32, [_P, _I64, _P, _P, _P, _F64]),
    "oracle_step_once": (None, [_P, _F64]),
    "oracle_run_until": (_I64, [_P, _F64, _I64]),
    "oracle_time": (_F64, [_P]),
    "oracle_energy": (_F64, [_P]),
    "oracle_step_index": (_I64, [_P]),
    "oracle_species_steps": (_I64, [_P]),
    "oracle_water": (_I64, [_P]),
    "oracle_n_live": (_I64, [_P]),
    "oracle_n_pending": (_I64, [_P]),
    "oracle_n_events": (_I64, [_P]),
    "oracle_n_steps": (_I64, [_P]),
    "oracle_counts": (None, [_P, _P]),
    "oracle_events_total": (None, [_P, _P]),
    "oracle_events": (None, [_P, _P]),
    "oracle_steps": (None, [_P, _P, _P]),
    "oracle_pending_types": (None, [_P, _P]),
    "oracle_state": (None, [_P, _P, _P, _P]),
    "oracle_philox": (None, [_P, _P, _P]),
    "oracle_uniforms": (None, [_I64, _P, _P, _P, _P]),
    "oracle_gaussians": (None, [_I64, _P, _I64, _U32, _U32, _P]),
    "oracle_acceptance_uniform": (None, [_I64, _P, _P, _I64, _U32, _U32, _P]),
    "oracle_wrap": (None, [_I64, _P, _F64, _P]),
    "oracle_min_image": (None, [_I64, _P, _F64, _P]),
    "oracle_touch_probability": (None, [_I64, _P, _P, _P, _F64, _P]),
    "oracle_reaction_radius": (_F64, [_F64, _F64]),
    "oracle_pairs_within": (_I64, [_I64, _P, _F64, _F64, _P, _I64]),
    "oracle_greedy_matching": (_I64, [_I64, _P, _P, _P, _P]),
}


def load():
    """The compiled reference program (built on first use)."""
    global _lib
    with _lock:
        if _lib is None:
            lib = C.CDLL(build())
            for name, (res, args) in _SIGS.items():
                f = getattr(lib, name)
                f.restype = res
                f.argtypes = args
            _lib = lib
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(C.c_void_p)


def _arr(x, dtype):
    return np.ascontiguousarray(np.asarray(x, dtype=dtype))


# ------------------------------------------------------------ building blocks (elementwise)
def philox_key(seed: int, train_id: int):
    """Key words (seed low word, seed high word XOR train id)."""
    seed = int(seed) & 0xFFFFFFFFFFFFFFFF
    return (seed & 0xFFFFFFFF, ((seed >> 32) ^ int(train_id)) & 0xFFFFFFFF)


def philox4x32_10(ctr, key):
    """Philox4x32-10 of one counter block (4 words) under a key (2 words)."""
    c = _arr([int(v) & 0xFFFFFFFF for v in ctr], np.uint32)
    k = _arr([int(v) & 0xFFFFFFFF for v in key], np.uint32)
    out = np.zeros(4, np.uint32)
    load().oracle_philox(_ptr(c), _ptr(k), _ptr(out))
    return tuple(np.uint64(v) for v in out)


def _uniforms(w_hi, w_lo):
    hi, lo = np.broadcast_arrays(np.asarray(w_hi, np.uint64), np.asarray(w_lo, np.uint64))
    shape = hi.shape
    hi = _arr(hi.ravel(), np.uint32)
    lo = _arr(lo.ravel(), np.uint32)
    a, b = np.zeros(hi.size), np.zeros(hi.size)
    load().oracle_uniforms(hi.size, _ptr(hi), _ptr(lo), _ptr(a), _ptr(b))
    return a.reshape(shape), b.reshape(shape)


def uniform_open0(w_hi, w_lo):
    a = _uniforms(w_hi, w_lo)[0]
    return a if a.ndim else float(a)


def uniform_closed0(w_hi, w_lo):
    b = _uniforms(w_hi, w_lo)[1]
    return b if b.ndim else float(b)


def gaussians(ids, step: int, key):
    ids = _arr(ids, np.int64).ravel()
    out = np.zeros((ids.size, 3))
    load().oracle_gaussians(ids.size, _ptr(ids), int(step), int(key[0]), int(key[1]), _ptr(out))
    return out


def acceptance_uniform(id_lo, id_hi, step: int, key):
    lo = _arr(id_lo, np.int64).ravel()
    hi = _arr(id_hi, np.int64).ravel()
    out = np.zeros(lo.size)
    load().oracle_acceptance_uniform(lo.size, _ptr(lo), _ptr(hi), int(step), int(key[0]), int(key[1]), _ptr(out))
    return out


def _elementwise(name, x, L):
    x = np.asarray(x, np.float64)
    flat = _arr(x.ravel(), np.float64)
    out = np.zeros(flat.size)
    getattr(load(), name)(flat.size, _ptr(flat), float(L), _ptr(out))
    return out.reshape(x.shape)


def wrap(x, L: float):
    return _elementwise("oracle_wrap", x, L)


def minimum_image(dx, L: float):
    return _elementwise("oracle_min_image", dx, L)


def touch_probability(d0, d1, R, DABdt):
    d0, d1, R = np.broadcast_arrays(np.asarray(d0, np.float64), np.asarray(d1, np.float64),
                                    np.asarray(R, np.float64))
    shape = d0.shape
    a, b, r = (_arr(v.ravel(), np.float64) for v in (d0, d1, R))
    out = np.zeros(a.size)
    load().oracle_touch_probability(a.size, _ptr(a), _ptr(b), _ptr(r), float(DABdt), _ptr(out))
    return out.reshape(shape)


def reaction_radius(k_tab: float, D_AB: float) -> float:
    return float(load().oracle_reaction_radius(float(k_tab), float(D_AB)))


def all_pairs_within(pos, L: float, r: float):
    """All unordered index pairs whose periodic distance is <= r (the program's cell list)."""
    pos = _arr(pos, np.float64).reshape(-1, 3)
    cap = 1024
    while True:
        out = np.zeros((cap, 2), np.int64)
        m = load().oracle_pairs_within(pos.shape[0], _ptr(pos), float(L), float(r), _ptr(out), cap)
        if m <= cap:
            return out[:m]
        cap = int(m)


def greedy_matching(id_lo, id_hi, d1sq):
    lo = _arr(id_lo, np.int64).ravel()
    hi = _arr(id_hi, np.int64).ravel()
    d = _arr(d1sq, np.float64).ravel()
    kept = np.zeros(lo.size, np.int64)
    m = load().oracle_greedy_matching(lo.size, _ptr(lo), _ptr(hi), _ptr(d), _ptr(kept))
    return kept[:m]


# ------------------------------------------------------------ one pulse train
def _unpack_reaction(rx):
    if hasattr(rx, "a"):
        return rx.a, rx.b, rx.k_tab, rx.products, rx.water_delta
    if isinstance(rx, dict):
        return rx["a"], rx["b"], rx["k_tab"], rx["products"], rx.get("water_delta", 0)
    return tuple(rx)


class SBSOracle:
    """One pulse train advanced step by step by the C++ program; same constructor and
    methods as ``oracle.sbs.SBSOracle`` (without the beam-off stage)."""

    def __init__(self, D: Sequence[float], reactions, L: float, seed: int, train_id: int = 0,
                 dt_min: float = 1e-9, dt_max: float = 1e-9, dt_growth: float = 1.0,
                 reset_on_release: bool = True, cutoff_c: float = 3.0,
                 sbs_horizon: float = 0.0, record: bool = True):
        self._lib = load()
        self.D = np.asarray(D, dtype=np.float64)
        self.n_types = self.D.shape[0]
        self.L = float(L)
        self.key = philox_key(seed, train_id)
        self.record = bool(record)
        rows = [_unpack_reaction(rx) for rx in reactions]
        tab = (_Reaction * max(1, len(rows)))()
        for i, (a, b, k_tab, products, water) in enumerate(rows):
            products = tuple(int(p) for p in products)
            if len(products) > 3:
                raise ValueError("more than 3 products")
            tab[i].a, tab[i].b, tab[i].k_tab = int(a), int(b), float(k_tab)
            tab[i].n_prod = len(products)
            for q in range(3):
                tab[i].prod[q] = products[q] if q < len(products) else -1
            tab[i].water_delta = int(water)
        self._D = _arr(self.D, np.float64)
        self._h = self._lib.oracle_new(self.n_types, _ptr(self._D), len(rows), C.cast(tab, C.c_void_p), self.L,
                                       int(seed) & 0xFFFFFFFFFFFFFFFF, int(train_id) & 0xFFFFFFFF,
                                       float(dt_min), float(dt_max), float(dt_growth), int(bool(reset_on_release)),
                                       float(cutoff_c), float(sbs_horizon), int(self.record))
        if not self._h:
            raise ValueError("bad reaction table or a reaction radius too large for the box")
        self.n_rxn = len(rows)
        self.D_AB = np.array([self.D[r[0]] + self.D[r[1]] for r in rows], dtype=np.float64)
        self.R = np.array([reaction_radius(r[2], d) for r, d in zip(rows, self.D_AB)], dtype=np.float64)

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            self._lib.oracle_free(h)
            self._h = None

    # -- inputs
    def inject(self, types, xyz, t_arrival, energy_eV: float = 0.0):
        types = _arr(types, np.int32).ravel()
        xyz = _arr(xyz, np.float64).reshape(-1, 3)
        t_arrival = _arr(t_arrival, np.float64).ravel()
        if not (types.size == xyz.shape[0] == t_arrival.size):
            raise ValueError("types, positions and arrival times differ in length")
        if self._lib.oracle_inject(self._h, types.size, _ptr(types), _ptr(xyz), _ptr(t_arrival),
                                   float(energy_eV)) != 0:
            raise ValueError("arrival before the current time, bad species type or position outside the box")

    # -- stepping
    def step_once(self, t_end: float):
        self._lib.oracle_step_once(self._h, float(t_end))

    def run_until(self, t_end: float, max_steps: Optional[int] = None):
        return int(self._lib.oracle_run_until(self._h, float(t_end), -1 if max_steps is None else int(max_steps)))

    def run_homogeneous(self, t_end: float):
        raise NotImplementedError("the beam-off stage is in oracle.sbs / oracle.homogeneous")

    # -- outputs
    @property
    def t(self) -> float:
        return float(self._lib.oracle_time(self._h))

    @property
    def step(self) -> int:
        return int(self._lib.oracle_step_index(self._h))

    @property
    def E_dep(self) -> float:
        return float(self._lib.oracle_energy(self._h))

    @property
    def species_steps(self) -> int:
        return int(self._lib.oracle_species_steps(self._h))

    @property
    def water(self) -> int:
        return int(self._lib.oracle_water(self._h))

    @property
    def events_total(self) -> np.ndarray:
        out = np.zeros(self.n_rxn, np.int64)
        if self.n_rxn:
            self._lib.oracle_events_total(self._h, _ptr(out))
        return out

    @property
    def p_types(self) -> np.ndarray:
        out = np.zeros(int(self._lib.oracle_n_pending(self._h)), np.int32)
        self._lib.oracle_pending_types(self._h, _ptr(out))
        return out.astype(np.int64)

    def counts(self):
        out = np.zeros(self.n_types, np.int64)
        self._lib.oracle_counts(self._h, _ptr(out))
        return out

    def g_values(self):
        """G = molecules per 100 eV deposited."""
        E = self.E_dep
        if E <= 0.0:
            return np.zeros(self.n_types)
        return self.counts().astype(np.float64) * 100.0 / E

    def state(self):
        """Live species sorted by id: (ids, types, positions)."""
        n = int(self._lib.oracle_n_live(self._h))
        ids = np.zeros(n, np.int64)
        types = np.zeros(n, np.int32)
        pos = np.zeros((n, 3))
        self._lib.oracle_state(self._h, _ptr(ids), _ptr(types), _ptr(pos))
        return ids, types.astype(np.int64), pos

    def events(self):
        n = int(self._lib.oracle_n_events(self._h))
        out = np.zeros((n, 6), np.int64)
        if n:
            self._lib.oracle_events(self._h, _ptr(out))
        return out

    def _step_arrays(self):
        n = int(self._lib.oracle_n_steps(self._h))
        ints = np.zeros((n, 3 + self.n_types), np.int64)
        times = np.zeros((n, 2))
        if n:
            self._lib.oracle_steps(self._h, _ptr(ints), _ptr(times))
        return ints, times

    def steps(self):
        """(step, n_live, n_events, counts per type) per step."""
        return self._step_arrays()[0]

    @property
    def step_log(self):
        """(step, t_start, dt, n_live, n_events, counts...) per step."""
        ints, times = self._step_arrays()
        return [(int(r[0]), float(t[0]), float(t[1]), *(int(v) for v in r[1:])) for r, t in zip(ints, times)]


def from_workload(wl, seed: int, train_id: int = 0, record: bool = True) -> SBSOracle:
    """Build a C++ reference train for a ``workloads.Workload`` and inject all its pulses."""
    s = wl.schedule
    o = SBSOracle(wl.D, wl.reactions, wl.L, seed, train_id, s.dt_min, s.dt_max, s.dt_growth,
                  s.reset_on_release, s.cutoff_c, s.sbs_horizon, record)
    for p in wl.pulses:
        o.inject(p.types, p.xyz, p.t_arrival, p.energy_eV)
    return o
