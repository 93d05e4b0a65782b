"""A track pulse built by the physico-chemical injector (Sec. 2.4, Table S1) through the
library on the GPU: FP64 mode equals the FP64 reference event for event, and in both
precisions charge is conserved exactly and H and O atoms balance against the water the
injector consumed and the reactions' water changes. Runs through the C ABI."""
import numpy as np
import pytest

from harness import assert_fp64_parity, cuda_available, gpu_run, oracle_run
from paper_2509_03313_gb300 import chem, physchem as P, workloads as W

pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not cuda_available(), reason="needs a CUDA GPU")]


def _workload(seed, n_tracks=8, L=600.0, events=600, t_end=2e-7):
    pulse, fp = P.physchem_pulse(n_tracks, L, events, seed=seed)
    wl = W.Workload("physchem", L, [pulse],
                    W.Schedule(dt_min=1e-12, dt_max=1e-7, dt_growth=W.LOG_GROWTH_20_PER_DECADE),
                    t_end=t_end)
    return wl, fp


def _balance(wl, fp, tally):
    c = tally["counts"][:7]
    ev = tally["events"][:len(wl.reactions)]
    water = int((ev * np.array([r.water_delta for r in wl.reactions])).sum()) - fp.water
    assert int(c @ W.CHARGE) == 0
    assert int(c @ W.N_H) + 2 * water == 0
    assert int(c @ W.N_O) + water + fp.o3p == 0


def test_physchem_pulse_fp64_equals_reference():
    wl, fp = _workload(31)
    g = gpu_run(wl, 31)
    o = oracle_run(wl, 31)
    assert o.events_total.sum() > 100
    assert_fp64_parity(g, o, wl.L)
    _balance(wl, fp, g["tally"])


def test_physchem_pulse_fp32_local_conserves():
    wl, fp = _workload(32, n_tracks=20, L=1000.0, events=2000, t_end=1e-6)
    g = gpu_run(wl, 32, precision=chem.CHEM_FP32_LOCAL, record=False)
    _balance(wl, fp, g["tally"])
    assert g["tally"]["events"].sum() > 1000
