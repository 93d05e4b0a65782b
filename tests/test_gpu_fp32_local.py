"""FP32-local mode against the FP64 reference.

Positions are FP32 offsets from their hash cell's origin and the normals are FP32, so
trajectories differ from the FP64 reference's; what must agree is the chemistry: the
G-values of H2O2, OH and e_aq, compared over 32 seeds with the tolerance
|mean_fp32 - mean_fp64| <= max(1 % of mean_fp64, 3 sigma), sigma the standard error of
the difference of the two 32-seed means. Exact integer identities (charge, counts vs
events) and free-diffusion MSD are checked per run."""
import math

import numpy as np
import pytest

from harness import cuda_available, gpu_run, oracle_run
from paper_2509_03313_gb300 import chem, workloads as W

pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not cuda_available(), reason="needs a CUDA GPU")]

SPECIES_G = {"H2O2": W.H2O2, "OH": W.OH, "e_aq": W.E_AQ}


def _stoich(reactions, n_types):
    m = np.zeros((len(reactions), n_types), dtype=np.int64)
    for r, rx in enumerate(reactions):
        m[r, rx.a] -= 1
        m[r, rx.b] -= 1
        for p in rx.products:
            m[r, p] += 1
    return m


def _compare_G(g32, g64, what):
    g32, g64 = np.asarray(g32), np.asarray(g64)
    diff = abs(g32.mean() - g64.mean())
    sigma = math.sqrt(g32.var(ddof=1) / g32.size + g64.var(ddof=1) / g64.size)
    tol = max(0.01 * abs(g64.mean()), 3.0 * sigma)
    assert diff <= tol, f"{what}: fp32 {g32.mean():.5g} fp64 {g64.mean():.5g} diff {diff:.3g} tol {tol:.3g}"


def test_counts_follow_events_and_charge_is_conserved():
    wl = W.uniform_2000(seed=5, L=200.0, n_steps=300)
    g = gpu_run(wl, 5, precision=chem.CHEM_FP32_LOCAL)
    tal = g["tally"]
    c0 = np.bincount(wl.pulses[0].types, minlength=7)
    expect = c0 + tal["events"] @ _stoich(wl.reactions, 7)
    assert np.array_equal(tal["counts"], expect)
    assert int((tal["counts"] * W.CHARGE).sum()) == int((c0 * W.CHARGE).sum())
    ids, types, xyz = g["state"]
    assert np.array_equal(np.bincount(types, minlength=7), tal["counts"])
    assert np.unique(ids).size == ids.size
    assert np.all(xyz >= -wl.L / 2) and np.all(xyz < wl.L / 2)
    # per-step records are consistent
    st = g["steps"]
    assert np.all(st["n_live"][1:] == st["counts"][:-1, :7].sum(1))


def test_free_diffusion_msd_with_regridding():
    # Inert species, log-growing dt: the hash grid coarsens many times; the displacement
    # of every species must still have variance 2 D t per axis.
    rng = np.random.default_rng(3)
    L, n = 5000.0, 40000
    types = rng.integers(0, 7, n).astype(np.int32)
    xyz = rng.uniform(-L / 2, L / 2, (n, 3))
    t_end = 2e-7
    # An absent 8th type reacting only with itself sets the cutoffs (and so the hash).
    wl = W.Workload("free32", L, [W.Pulse(types, xyz, np.zeros(n), 1.0)],
                    W.Schedule(dt_min=1e-12, dt_max=1e-7, dt_growth=W.LOG_GROWTH_20_PER_DECADE),
                    t_end=t_end, n_types=8, D=np.r_[W.D_NM2_S, 9.3e9],
                    reactions=[W.Reaction("X", 7, 7, 11e10, (), 0)])
    g = gpu_run(wl, 9, precision=chem.CHEM_FP32_LOCAL, record=False)
    ids, gt, gx = g["state"]
    assert ids.size == n and np.array_equal(ids, np.arange(n))
    d = gx - xyz[ids]
    d -= L * np.round(d / L)
    for ty in range(7):
        m = gt == ty
        var = d[m].var(axis=0) / (2 * W.D_NM2_S[ty] * t_end)
        assert np.all(np.abs(var - 1.0) < 6 * math.sqrt(2.0 / m.sum())), (ty, var)


@pytest.mark.parametrize("wl_name", ["dense_uniform", "tracks"])
def test_g_values_match_fp64_reference_over_seeds(wl_name):
    seeds = list(range(32))
    g32 = {k: [] for k in SPECIES_G}
    g64 = {k: [] for k in SPECIES_G}
    for s in seeds:
        if wl_name == "dense_uniform":
            wl = W.uniform_2000(seed=100 + s, L=200.0, n_steps=200)
        else:
            pulse = W.track_pulse(20, 600.0, 400, seed=200 + s)
            wl = W.Workload("tracks32", 600.0, [pulse],
                            W.Schedule(dt_min=1e-12, dt_max=1e-6, dt_growth=W.LOG_GROWTH_20_PER_DECADE),
                            t_end=1e-7)
        g = gpu_run(wl, 1000 + s, precision=chem.CHEM_FP32_LOCAL, record=False)
        o = oracle_run(wl, 1000 + s)
        og = o.g_values()
        for k, t in SPECIES_G.items():
            g32[k].append(g["tally"]["G"][t])
            g64[k].append(og[t])
    for k in SPECIES_G:
        _compare_G(g32[k], g64[k], f"{wl_name} G({k})")
