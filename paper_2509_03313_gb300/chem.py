"""Thin Python binding of the C ABI in include/chem.h (argument marshalling only).

Every function here has the name of the C entry point it calls; arrays are numpy arrays
on the host. The CUDA library must be present: importing this module raises if
libchem.so cannot be loaded, and there is no CPU fallback. PyTorch, when used, only
provides device memory (``torch_allocator``) and the CUDA stream.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional, Sequence

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libchem.so")

CHEM_OK, CHEM_EINVAL, CHEM_ENOMEM, CHEM_ECAPACITY, CHEM_ECUDA, CHEM_ETIMEOUT, CHEM_ESTATE = range(7)
CHEM_FP64, CHEM_FP32_LOCAL = 0, 1
CHEM_LAUNCH_AUTO, CHEM_LAUNCH_PHASES, CHEM_LAUNCH_PERSISTENT = 0, 1, 2
STATUS_NAMES = {0: "CHEM_OK", 1: "CHEM_EINVAL", 2: "CHEM_ENOMEM", 3: "CHEM_ECAPACITY",
                4: "CHEM_ECUDA", 5: "CHEM_ETIMEOUT", 6: "CHEM_ESTATE"}

ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p)
FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p)


class chem_reaction(ctypes.Structure):
    _fields_ = [("a", ctypes.c_int32), ("b", ctypes.c_int32), ("k_tab", ctypes.c_double),
                ("n_prod", ctypes.c_int32), ("prod", ctypes.c_int32 * 3),
                ("water_delta", ctypes.c_int32)]


class chem_config(ctypes.Structure):
    _fields_ = [
        ("n_types", ctypes.c_int32), ("D_nm2_s", ctypes.POINTER(ctypes.c_double)),
        ("n_rxn", ctypes.c_int32), ("rxn", ctypes.POINTER(chem_reaction)),
        ("L_nm", ctypes.c_double), ("seed", ctypes.c_uint64), ("train_id", ctypes.c_uint32),
        ("precision", ctypes.c_int32),
        ("dt_min_s", ctypes.c_double), ("dt_max_s", ctypes.c_double), ("dt_growth", ctypes.c_double),
        ("dt_reset_on_release", ctypes.c_int32), ("cutoff_c", ctypes.c_double),
        ("sbs_horizon_s", ctypes.c_double),
        ("capacity_species", ctypes.c_int64), ("capacity_pending", ctypes.c_int64),
        ("capacity_candidates", ctypes.c_int64), ("capacity_event_log", ctypes.c_int64),
        ("capacity_step_log", ctypes.c_int64),
        ("cells_per_axis_max", ctypes.c_int32), ("steps_per_launch", ctypes.c_int32),
        ("launch_mode", ctypes.c_int32),
        ("cuda_stream", ctypes.c_void_p),
        ("dev_alloc", ALLOC_FN), ("dev_free", FREE_FN), ("alloc_user", ctypes.c_void_p),
    ]


class chem_event(ctypes.Structure):
    _fields_ = [("step", ctypes.c_uint32), ("rxn", ctypes.c_int32), ("id_lo", ctypes.c_uint32),
                ("id_hi", ctypes.c_uint32), ("prod_id0", ctypes.c_uint32), ("n_prod", ctypes.c_int32),
                ("train", ctypes.c_uint32), ("reserved", ctypes.c_uint32)]


class chem_step_record(ctypes.Structure):
    _fields_ = [("step", ctypes.c_uint32), ("train", ctypes.c_uint32), ("t_start_s", ctypes.c_double),
                ("dt_s", ctypes.c_double), ("n_live", ctypes.c_int64), ("n_events", ctypes.c_int64),
                ("counts", ctypes.c_int64 * 8)]


class chem_stats(ctypes.Structure):
    _fields_ = [("graph_replays", ctypes.c_int64), ("kernel_launches", ctypes.c_int64),
                ("steps_launched", ctypes.c_int64), ("bytes_h2d", ctypes.c_int64),
                ("bytes_d2h", ctypes.c_int64), ("phase_ms", ctypes.c_double * 8),
                ("phase_launches", ctypes.c_int64 * 8), ("react_rounds_global", ctypes.c_int64),
                ("react_order_global", ctypes.c_int64), ("react_order_radix", ctypes.c_int64),
                ("max_conflict_pairs", ctypes.c_int64), ("max_step_events", ctypes.c_int64),
                ("pairs_tested", ctypes.c_int64), ("pairs_in_cutoff", ctypes.c_int64),
                ("pairs_accepted", ctypes.c_int64), ("steps_advanced", ctypes.c_int64),
                ("steps_cell_tiles", ctypes.c_int64)]


PHASES = ("begin", "release", "diffuse", "sort", "gather", "search", "react", "persistent")

EVENT_DTYPE = np.dtype([("step", np.uint32), ("rxn", np.int32), ("id_lo", np.uint32),
                        ("id_hi", np.uint32), ("prod_id0", np.uint32), ("n_prod", np.int32),
                        ("train", np.uint32), ("reserved", np.uint32)])
STEP_DTYPE = np.dtype([("step", np.uint32), ("train", np.uint32), ("t_start_s", np.float64),
                       ("dt_s", np.float64), ("n_live", np.int64), ("n_events", np.int64),
                       ("counts", np.int64, (8,))])

# Every entry point of include/chem.h.
EXPORTS = ["chem_init", "chem_inject_pulse", "chem_run_until", "chem_tally", "chem_get_state",
           "chem_get_events", "chem_get_step_log", "chem_reset", "chem_last_error", "chem_destroy",
           "chem_batch_init", "chem_batch_inject", "chem_batch_run_until", "chem_batch_tally",
           "chem_batch_get_state", "chem_batch_reset", "chem_batch_size", "chem_autotune", "chem_set_tuning",
           "chem_version", "chem_get_stats", "chem_set_profiling", "chem_step_noalloc",
           "chem_run_homogeneous", "chem_batch_run_homogeneous", "chem_batch_homogeneous_report",
           "chem_check_bounded_wait", "chem_check_acceptance"]


class ChemError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


def load(path: str = LIB_PATH) -> ctypes.CDLL:
    if not os.path.exists(path):
        raise ImportError(f"CUDA library not built: {path} (run __graft_entry__.build())")
    lib = ctypes.CDLL(path)
    P = ctypes.POINTER
    vp, i32, i64, dbl = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_double
    sig = {
        "chem_init": (i32, [P(chem_config), P(vp)]),
        "chem_inject_pulse": (i32, [vp, i64, vp, vp, vp, dbl]),
        "chem_run_until": (i32, [vp, dbl]),
        "chem_tally": (i32, [vp, vp, vp, vp, vp, vp]),
        "chem_get_state": (i32, [vp, i64, vp, vp, vp, vp]),
        "chem_get_events": (i32, [vp, i64, vp, vp]),
        "chem_get_step_log": (i32, [vp, i64, vp, vp]),
        "chem_reset": (i32, [vp, ctypes.c_uint64]),
        "chem_last_error": (ctypes.c_char_p, [vp]),
        "chem_destroy": (None, [vp]),
        "chem_batch_init": (i32, [P(chem_config), i32, P(vp)]),
        "chem_batch_inject": (i32, [vp, i32, i64, vp, vp, vp, dbl]),
        "chem_batch_run_until": (i32, [vp, vp]),
        "chem_batch_tally": (i32, [vp, i32, vp, vp, vp, vp, vp]),
        "chem_batch_get_state": (i32, [vp, i32, i64, vp, vp, vp, vp]),
        "chem_batch_reset": (i32, [vp, vp]),
        "chem_batch_size": (i32, [vp]),
        "chem_autotune": (i32, [vp, dbl, vp]),
        "chem_set_tuning": (i32, [vp, vp]),
        "chem_version": (ctypes.c_char_p, []),
        "chem_get_stats": (i32, [vp, P(chem_stats)]),
        "chem_set_profiling": (i32, [vp, i32]),
        "chem_step_noalloc": (i32, [P(chem_config), ctypes.c_uint32, dbl, dbl, ctypes.c_uint32, i32,
                                    vp, vp, vp, vp, vp, vp, vp, vp, vp, vp]),
        "chem_run_homogeneous": (i32, [vp, dbl]),
        "chem_batch_run_homogeneous": (i32, [vp, vp]),
        "chem_batch_homogeneous_report": (i32, [vp, i32, vp, vp, vp]),
        "chem_check_bounded_wait": (i32, [vp, dbl]),
        "chem_check_acceptance": (i32, [vp, i32, ctypes.c_uint32, dbl, i64, vp, vp, vp, vp, vp, vp]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    return lib


_LIB: Optional[ctypes.CDLL] = None


def lib() -> ctypes.CDLL:
    global _LIB
    if _LIB is None:
        _LIB = load()
    return _LIB


def _ptr(a: Optional[np.ndarray]):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _check(ctx, status: int):
    if status != CHEM_OK:
        msg = lib().chem_last_error(ctx).decode() if ctx else ""
        raise ChemError(status, msg)


class torch_allocator:
    """Device memory from PyTorch's caching allocator, for chem_config.dev_alloc/free."""

    def __init__(self, device: int = 0, stream=None):
        import torch
        self.torch = torch
        self.device = device
        self.stream = stream
        self.alloc = ALLOC_FN(self._alloc)
        self.free = FREE_FN(self._free)

    def _alloc(self, nbytes, user):
        try:
            return self.torch.cuda.caching_allocator_alloc(int(nbytes), self.device, self.stream)
        except Exception:  # noqa: BLE001 - reported to C as NULL
            return None

    def _free(self, ptr, nbytes, user):
        self.torch.cuda.caching_allocator_delete(ptr)


def make_config(L_nm: float, D: Sequence[float], reactions, seed: int = 0, train_id: int = 0,
                precision: int = CHEM_FP64, dt_min: float = 1e-9, dt_max: float = 1e-9,
                dt_growth: float = 1.0, reset_on_release: bool = True, cutoff_c: float = 3.0,
                sbs_horizon: float = 0.0, capacity_species: int = 1 << 16,
                capacity_pending: Optional[int] = None, capacity_candidates: Optional[int] = None,
                capacity_event_log: int = 0, capacity_step_log: int = 0,
                cells_per_axis_max: int = 0, steps_per_launch: int = 0,
                launch_mode: int = CHEM_LAUNCH_AUTO, stream=None,
                allocator: Optional[torch_allocator] = None):
    """Build a chem_config. Returns (config, keepalive); keep both alive while in use.
    ``reactions`` holds objects with a, b, k_tab, products, water_delta (or tuples)."""
    D = np.ascontiguousarray(D, dtype=np.float64)
    rx = (chem_reaction * max(1, len(reactions)))()
    for i, r in enumerate(reactions):
        if hasattr(r, "a"):
            a, b, k, prods, w = r.a, r.b, r.k_tab, tuple(r.products), r.water_delta
        else:
            a, b, k, prods, w = r[0], r[1], r[2], tuple(r[3]), r[4]
        rx[i].a, rx[i].b, rx[i].k_tab, rx[i].n_prod, rx[i].water_delta = a, b, k, len(prods), w
        for q, p in enumerate(prods):
            rx[i].prod[q] = p
    cfg = chem_config()
    cfg.n_types = D.shape[0]
    cfg.D_nm2_s = D.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    cfg.n_rxn = len(reactions)
    cfg.rxn = ctypes.cast(rx, ctypes.POINTER(chem_reaction))
    cfg.L_nm = L_nm
    cfg.seed = seed & 0xFFFFFFFFFFFFFFFF
    cfg.train_id = train_id
    cfg.precision = precision
    cfg.dt_min_s, cfg.dt_max_s, cfg.dt_growth = dt_min, dt_max, dt_growth
    cfg.dt_reset_on_release = 1 if reset_on_release else 0
    cfg.cutoff_c = cutoff_c
    cfg.sbs_horizon_s = sbs_horizon
    cfg.capacity_species = capacity_species
    cfg.capacity_pending = capacity_pending if capacity_pending is not None else capacity_species
    cfg.capacity_candidates = (capacity_candidates if capacity_candidates is not None
                               else max(1024, capacity_species // 4))
    cfg.capacity_event_log = capacity_event_log
    cfg.capacity_step_log = capacity_step_log
    cfg.cells_per_axis_max = cells_per_axis_max
    cfg.steps_per_launch = steps_per_launch
    cfg.launch_mode = launch_mode
    if stream is not None:
        cfg.cuda_stream = ctypes.c_void_p(int(stream))
    if allocator is not None:
        cfg.dev_alloc = allocator.alloc
        cfg.dev_free = allocator.free
    return cfg, (D, rx, allocator)


def chem_init(cfg: chem_config):
    ctx = ctypes.c_void_p()
    st = lib().chem_init(ctypes.byref(cfg), ctypes.byref(ctx))
    if st != CHEM_OK:
        msg = lib().chem_last_error(ctx).decode() if ctx else ""
        if ctx:
            lib().chem_destroy(ctx)
        raise ChemError(st, msg)
    return ctx


def chem_batch_init(cfgs: Sequence[chem_config]):
    arr = (chem_config * len(cfgs))(*cfgs)
    ctx = ctypes.c_void_p()
    st = lib().chem_batch_init(arr, len(cfgs), ctypes.byref(ctx))
    if st != CHEM_OK:
        msg = lib().chem_last_error(ctx).decode() if ctx else ""
        if ctx:
            lib().chem_destroy(ctx)
        raise ChemError(st, msg)
    return ctx


def _inject_arrays(types, xyz, t_arrival):
    types = np.ascontiguousarray(types, dtype=np.int32)
    xyz = np.ascontiguousarray(xyz, dtype=np.float64).reshape(-1, 3)
    t_arrival = np.ascontiguousarray(t_arrival, dtype=np.float64)
    if not (types.shape[0] == xyz.shape[0] == t_arrival.shape[0]):
        raise ValueError("inconsistent array lengths")
    return types, xyz, t_arrival


def chem_inject_pulse(ctx, types, xyz, t_arrival, energy_eV: float = 0.0):
    types, xyz, t_arrival = _inject_arrays(types, xyz, t_arrival)
    _check(ctx, lib().chem_inject_pulse(ctx, types.shape[0], _ptr(types), _ptr(xyz), _ptr(t_arrival),
                                        float(energy_eV)))


def chem_batch_inject(ctx, train: int, types, xyz, t_arrival, energy_eV: float = 0.0):
    types, xyz, t_arrival = _inject_arrays(types, xyz, t_arrival)
    _check(ctx, lib().chem_batch_inject(ctx, train, types.shape[0], _ptr(types), _ptr(xyz),
                                        _ptr(t_arrival), float(energy_eV)))


def chem_run_until(ctx, t_end: float):
    _check(ctx, lib().chem_run_until(ctx, float(t_end)))


def chem_batch_run_until(ctx, t_end):
    t = np.ascontiguousarray(t_end, dtype=np.float64)
    _check(ctx, lib().chem_batch_run_until(ctx, _ptr(t)))


def chem_run_homogeneous(ctx, t_end: float):
    """Homogeneous (beam-off) stage of every train up to t_end (rate equations, Sec. 2.3)."""
    _check(ctx, lib().chem_run_homogeneous(ctx, float(t_end)))


def chem_batch_run_homogeneous(ctx, t_end):
    t = np.ascontiguousarray(t_end, dtype=np.float64)
    _check(ctx, lib().chem_batch_run_homogeneous(ctx, _ptr(t)))


def chem_batch_homogeneous_report(ctx, train: int = 0, n_rxn: int = 16):
    """(real extents, whole events, integrator steps) of the train's last homogeneous stage."""
    e = np.zeros(n_rxn, np.float64)
    E = np.zeros(n_rxn, np.int64)
    st = np.zeros(1, np.int64)
    _check(ctx, lib().chem_batch_homogeneous_report(ctx, int(train), _ptr(e), _ptr(E), _ptr(st)))
    return e, E, int(st[0])


def chem_check_bounded_wait(ctx, limit_s: float):
    """Diagnostic: a device wait on a word nothing writes, bounded by limit_s; raises
    ChemError(CHEM_ETIMEOUT) (sticky on ctx)."""
    _check(ctx, lib().chem_check_bounded_wait(ctx, float(limit_s)))


def chem_check_acceptance(ctx, precision: int, step: int, dt_s: float, d0sq, d1sq, rxn, id_lo, id_hi):
    """The search's acceptance test on given squared separations: returns (tiered, exact)
    boolean arrays (the tiered FP32/FP64 decision and u < p in FP64)."""
    d0 = np.ascontiguousarray(d0sq, np.float64)
    d1 = np.ascontiguousarray(d1sq, np.float64)
    r = np.ascontiguousarray(rxn, np.int32)
    lo = np.ascontiguousarray(id_lo, np.uint32)
    hi = np.ascontiguousarray(id_hi, np.uint32)
    out = np.zeros(d0.shape[0], np.uint8)
    _check(ctx, lib().chem_check_acceptance(ctx, int(precision), int(step), float(dt_s), d0.shape[0], _ptr(d0),
                                            _ptr(d1), _ptr(r), _ptr(lo), _ptr(hi), _ptr(out)))
    return (out & 1) != 0, (out & 2) != 0


def chem_batch_size(ctx) -> int:
    return int(lib().chem_batch_size(ctx))


def _tally(ctx, train: Optional[int], n_types: int = 8, n_rxn: int = 16):
    counts = np.zeros(n_types, np.int64)
    G = np.zeros(n_types, np.float64)
    events = np.zeros(n_rxn, np.int64)
    t = np.zeros(1, np.float64)
    ss = np.zeros(1, np.int64)
    if train is None:
        st = lib().chem_tally(ctx, _ptr(counts), _ptr(G), _ptr(events), _ptr(t), _ptr(ss))
    else:
        st = lib().chem_batch_tally(ctx, train, _ptr(counts), _ptr(G), _ptr(events), _ptr(t), _ptr(ss))
    _check(ctx, st)
    return dict(counts=counts, G=G, events=events, t=float(t[0]), species_steps=int(ss[0]))


def chem_tally(ctx, n_types: int = 8, n_rxn: int = 16):
    """counts[n_types], G per 100 eV, events[n_rxn], clock t, species_steps."""
    return _tally(ctx, None, n_types, n_rxn)


def chem_batch_tally(ctx, train: int, n_types: int = 8, n_rxn: int = 16):
    return _tally(ctx, train, n_types, n_rxn)


def _state(ctx, train: Optional[int]):
    n = np.zeros(1, np.int64)
    call = (lambda cap, a, b, c: lib().chem_get_state(ctx, cap, a, b, c, _ptr(n))) if train is None else \
        (lambda cap, a, b, c: lib().chem_batch_get_state(ctx, train, cap, a, b, c, _ptr(n)))
    st = call(0, None, None, None)
    if st not in (CHEM_OK, CHEM_EINVAL):
        _check(ctx, st)
    cap = int(n[0])
    types = np.zeros(cap, np.int32)
    ids = np.zeros(cap, np.uint32)
    xyz = np.zeros((cap, 3), np.float64)
    _check(ctx, call(cap, _ptr(types), _ptr(ids), _ptr(xyz)))
    return ids, types, xyz


def chem_get_state(ctx):
    """(ids, types, xyz) of the live species of train 0, in device order."""
    return _state(ctx, None)


def chem_batch_get_state(ctx, train: int):
    return _state(ctx, train)


def chem_get_events(ctx) -> np.ndarray:
    n = np.zeros(1, np.int64)
    _check(ctx, lib().chem_get_events(ctx, 0, None, _ptr(n)))
    out = np.zeros(int(n[0]), EVENT_DTYPE)
    _check(ctx, lib().chem_get_events(ctx, out.shape[0], _ptr(out), _ptr(n)))
    return out


def chem_get_step_log(ctx) -> np.ndarray:
    n = np.zeros(1, np.int64)
    _check(ctx, lib().chem_get_step_log(ctx, 0, None, _ptr(n)))
    out = np.zeros(int(n[0]), STEP_DTYPE)
    _check(ctx, lib().chem_get_step_log(ctx, out.shape[0], _ptr(out), _ptr(n)))
    return out


def chem_reset(ctx, seed: int):
    _check(ctx, lib().chem_reset(ctx, seed & 0xFFFFFFFFFFFFFFFF))


def chem_batch_reset(ctx, seeds):
    s = np.ascontiguousarray(seeds, dtype=np.uint64)
    _check(ctx, lib().chem_batch_reset(ctx, _ptr(s)))


def chem_autotune(ctx, budget_ms: float = 2000.0):
    """Returns (steps_per_launch, cells_per_axis_limit, species_per_item, launch_mode)."""
    chosen = np.zeros(4, np.int32)
    _check(ctx, lib().chem_autotune(ctx, float(budget_ms), _ptr(chosen)))
    return int(chosen[0]), int(chosen[1]), int(chosen[2]), int(chosen[3])


def chem_set_tuning(ctx, steps_per_launch: int, cells_per_axis_limit: int, species_per_item: int,
                    launch_mode: int):
    """Apply the parameters chem_autotune would choose (same order as its result)."""
    t = np.array([steps_per_launch, cells_per_axis_limit, species_per_item, launch_mode], np.int32)
    _check(ctx, lib().chem_set_tuning(ctx, _ptr(t)))


def chem_last_error(ctx) -> str:
    return lib().chem_last_error(ctx).decode()


def chem_destroy(ctx):
    if ctx:
        lib().chem_destroy(ctx)


def chem_get_stats(ctx) -> dict:
    st = chem_stats()
    _check(ctx, lib().chem_get_stats(ctx, ctypes.byref(st)))
    return dict(graph_replays=st.graph_replays, kernel_launches=st.kernel_launches,
                steps_launched=st.steps_launched, bytes_h2d=st.bytes_h2d, bytes_d2h=st.bytes_d2h,
                phase_ms={PHASES[i]: st.phase_ms[i] for i in range(8)},
                phase_launches={PHASES[i]: st.phase_launches[i] for i in range(8)},
                react_rounds_global=st.react_rounds_global, react_order_global=st.react_order_global,
                react_order_radix=st.react_order_radix, max_conflict_pairs=st.max_conflict_pairs,
                max_step_events=st.max_step_events, pairs_tested=st.pairs_tested,
                pairs_in_cutoff=st.pairs_in_cutoff, pairs_accepted=st.pairs_accepted,
                steps_advanced=st.steps_advanced, steps_cell_tiles=st.steps_cell_tiles)


def chem_set_profiling(ctx, on: bool):
    _check(ctx, lib().chem_set_profiling(ctx, 1 if on else 0))


CHEM_NOALLOC_MAX_SPECIES = 16384


def chem_step_noalloc(cfg: chem_config, step: int, t_s: float, dt_s: float, next_id: int, n: int,
                      id_ptr: int, type_ptr: int, xyz_ptr: int, id_out: int, type_out: int,
                      xyz_out: int, n_out: int, next_id_out: int, events_out: int,
                      n_events_out: int) -> int:
    """One FP64 step on caller-owned DEVICE buffers (integer device addresses); returns
    the chem_status."""
    vp = ctypes.c_void_p
    return int(lib().chem_step_noalloc(ctypes.byref(cfg), step, t_s, dt_s, next_id, n, vp(id_ptr),
                                       vp(type_ptr), vp(xyz_ptr), vp(id_out), vp(type_out), vp(xyz_out),
                                       vp(n_out), vp(next_id_out), vp(events_out), vp(n_events_out)))


def chem_version() -> str:
    return lib().chem_version().decode()
