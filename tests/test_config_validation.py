"""Configuration checks of chem_init / chem_batch_init: every bad field is refused with
CHEM_EINVAL before any device work, so these run without a GPU (only the library is
loaded). Covers the bad tables and inputs the boundary promises to reject."""
import math

import pytest

from paper_2509_03313_gb300 import chem, workloads as W


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2509_03313_gb300 import build
    build.build()


def _cfg(**kw):
    base = dict(L_nm=1000.0, D=W.D_NM2_S, reactions=W.WATER_REACTIONS, seed=1, dt_min=1e-9, dt_max=1e-9,
                capacity_species=4096)
    base.update(kw)
    return chem.make_config(**base)


def _refused(cfg_keep):
    cfg, keep = cfg_keep
    with pytest.raises(chem.ChemError) as err:
        chem.chem_init(cfg)
    assert err.value.status == chem.CHEM_EINVAL


@pytest.mark.parametrize("L", [0.0, -5.0, math.inf, math.nan])
def test_bad_box(L):
    _refused(_cfg(L_nm=L))


def test_box_too_small_for_a_reaction_radius():
    # R9 (H3O+ + OH-) has R ~ 1 nm: cutoffs must stay below L/3 (minimum image, Eq. 2)
    _refused(_cfg(L_nm=2.5))


@pytest.mark.parametrize("kw", [dict(dt_min=0.0), dict(dt_min=1e-9, dt_max=1e-10), dict(dt_growth=0.9),
                                dict(cutoff_c=-1.0), dict(sbs_horizon=-1.0), dict(capacity_species=0),
                                dict(precision=7)])
def test_bad_schedule_capacity_or_precision(kw):
    _refused(_cfg(**kw))


def test_bad_diffusion_coefficients_and_type_count():
    D = W.D_NM2_S.copy()
    D[2] = 0.0
    _refused(_cfg(D=D))
    _refused(_cfg(D=list(W.D_NM2_S) + [1e9, 1e9]))  # 9 types > 8


def test_bad_reaction_tables():
    rx = list(W.WATER_REACTIONS)
    _refused(_cfg(reactions=rx + [(0, 1, 1e10, (3,), 0)]))        # second reaction for (e, OH)
    _refused(_cfg(reactions=rx[:8] + [(3, 9, 1e10, (), 0)]))      # reactant type out of range
    _refused(_cfg(reactions=rx[:8] + [(3, 4, 1e10, (12,), 0)]))   # product type out of range
    _refused(_cfg(reactions=rx[:8] + [(3, 4, 0.0, (), 1)]))       # k must be positive
    cfg, keep = _cfg()
    cfg.rxn[0].n_prod = 4                                          # at most 3 products
    _refused((cfg, keep))


def test_batched_trains_must_share_the_chemistry():
    a, ka = _cfg()
    b, kb = _cfg(D=W.D_NM2_S * 1.01)
    with pytest.raises(chem.ChemError) as err:
        chem.chem_batch_init([a, b])
    assert err.value.status == chem.CHEM_EINVAL
    c, kc = _cfg(precision=chem.CHEM_FP32_LOCAL)
    with pytest.raises(chem.ChemError) as err:
        chem.chem_batch_init([a, c])
    assert err.value.status == chem.CHEM_EINVAL
