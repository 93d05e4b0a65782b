"""The C-ABI library builds, loads and exports every entry point of include/chem.h
(no compute calls: these run without a GPU)."""
import ctypes
import os
import re

import pytest

from conftest import ROOT


def _declared():
    src = open(os.path.join(ROOT, "include", "chem.h")).read()
    return sorted(set(re.findall(r"\b(chem_[a-z_0-9]+)\s*\(", src)) - {"chem_alloc_fn", "chem_free_fn"})


@pytest.fixture(scope="module")
def lib():
    from paper_2509_03313_gb300 import build
    build.build()
    from paper_2509_03313_gb300 import chem
    return chem.load()


def test_every_declared_entry_point_is_exported(lib):
    names = _declared()
    assert len(names) >= 19
    for n in names:
        assert hasattr(lib, n), n


def test_binding_covers_every_entry_point():
    from paper_2509_03313_gb300 import chem
    assert sorted(chem.EXPORTS) == _declared()


def test_version_string(lib):
    assert b"sm_103a" in lib.chem_version()


def test_struct_sizes_match_header(lib):
    from paper_2509_03313_gb300 import chem
    assert ctypes.sizeof(chem.chem_event) == 32
    assert ctypes.sizeof(chem.chem_step_record) == 4 * 2 + 8 * 2 + 8 * 2 + 8 * 8
    assert chem.EVENT_DTYPE.itemsize == ctypes.sizeof(chem.chem_event)
    assert chem.STEP_DTYPE.itemsize == ctypes.sizeof(chem.chem_step_record)


def test_invalid_configs_are_rejected_before_touching_a_gpu(lib):
    from paper_2509_03313_gb300 import chem, workloads as W
    bad = [dict(L_nm=-1.0), dict(dt_min=0.0), dict(dt_growth=0.5), dict(capacity_species=0),
           dict(L_nm=1.0)]  # L/3 below the largest radius
    for kw in bad:
        args = dict(L_nm=100.0, D=W.D_NM2_S, reactions=W.WATER_REACTIONS)
        L = kw.pop("L_nm", 100.0)
        cfg, keep = chem.make_config(L, W.D_NM2_S, W.WATER_REACTIONS, **kw)
        with pytest.raises(chem.ChemError) as e:
            chem.chem_init(cfg)
        assert e.value.status == chem.CHEM_EINVAL, kw


def test_binding_fails_loudly_without_the_library(tmp_path):
    from paper_2509_03313_gb300 import chem
    with pytest.raises(ImportError):
        chem.load(str(tmp_path / "libchem.so"))
