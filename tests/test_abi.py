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


def test_library_and_references_stay_apart():
    """The library never loads a reference, and the C++ reference includes nothing of the
    CUDA path (each side computes the method on its own)."""
    import subprocess
    import sys
    code = ("import sys; import paper_2509_03313_gb300 as p; "
            "from paper_2509_03313_gb300 import chem, workloads, physchem, hybrid, build; "
            "bad = [m for m in sys.modules if m == 'oracle' or m.startswith('oracle.')]; "
            "print(bad); sys.exit(1 if bad else 0)")
    r = subprocess.run([sys.executable, "-c", code], cwd=ROOT, capture_output=True, text=True)
    assert r.returncode == 0, r.stdout + r.stderr
    pkg = os.path.join(ROOT, "paper_2509_03313_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h", ".cpp")):
                text = open(os.path.join(dirpath, f), errors="replace").read()
                assert not re.search(r"^\s*(from|import)\s+oracle\b", text, re.M), f
                assert "sbs_oracle" not in text, f
    src = open(os.path.join(ROOT, "oracle", "csrc", "sbs_oracle.cpp")).read()
    includes = re.findall(r'#include\s*[<"]([^>"]+)[>"]', src)
    assert includes and all("/" not in i and not i.endswith((".h", ".cuh")) for i in includes), includes
