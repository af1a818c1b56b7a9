"""C-ABI checks that need no GPU: the library builds and loads, exports exactly
the functions include/*.h declares, and rejects bad configurations before it
touches CUDA.  Plus a static check that the product never reaches the oracle."""
import glob
import os
import re
import subprocess

import numpy as np
import pytest

import paper_2007_06048_gb300 as M

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for hdr in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = re.sub(r"/\*.*?\*/", "", open(hdr).read(), flags=re.S)
        names.update(re.findall(r"\b(mmod_\w+)\s*\(", text))
    return names


def exported_symbols():
    out = subprocess.run(["nm", "-D", "--defined-only", M.build()], capture_output=True, text=True,
                         check=True).stdout
    return {line.split()[-1] for line in out.splitlines() if line.split()[-1].startswith("mmod_")}


def test_header_and_library_agree():
    decl = declared_functions()
    assert decl == set(M.EXPORTED)
    assert exported_symbols() == decl


def header_constants():
    """Every NAME = value of the header's enums (comments stripped)."""
    consts = {}
    for hdr in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = re.sub(r"/\*.*?\*/", "", open(hdr).read(), flags=re.S)
        for body in re.findall(r"enum\s*\{(.*?)\}", text, flags=re.S):
            for name, value in re.findall(r"\b(MMOD_\w+)\s*=\s*(-?\d+)", body):
                consts[name] = int(value)
    return consts


def test_binding_constants_match_the_header():
    """The binding's option, mode and status numbers are the header's."""
    consts = header_constants()
    pairs = {name[len("MMOD_"):]: value for name, value in consts.items()}
    checked = 0
    for py_name, value in pairs.items():
        if hasattr(M, py_name):
            assert getattr(M, py_name) == value, py_name
            checked += 1
    assert checked >= 20
    for status, text in M.STATUS.items():
        assert consts["MMOD_" + text] == status
    for needed in ("OPT_PDL", "OPT_ZLEN", "OPT_CPML_PLANES", "OPT_TEST_STALL", "BATCH_PERSISTENT", "KERNEL_TMA"):
        assert hasattr(M, needed), needed


def test_every_symbol_loads():
    lib = M.load()
    for name in M.EXPORTED:
        assert getattr(lib, name) is not None


def test_only_api_symbols_are_exported():
    out = subprocess.run(["nm", "-D", "--defined-only", M.build()], capture_output=True, text=True,
                         check=True).stdout
    public = [l.split()[-1] for l in out.splitlines() if l.split()[1] in "TDB"]
    assert all(s.startswith("mmod_") or s.startswith("_") for s in public), public


def test_version_and_cfl():
    assert "sm_103a" in M.mmod_version()
    assert M.mmod_cfl_dt(0.4, 10.0, 4500.0) == pytest.approx(0.4 * 10 / 4500)
    assert M.mmod_cfl_dt(-1.0, 10.0, 4500.0) < 0


GOOD = dict(nx=20, ny=21, nz=22, h=(10.0, 10.0, 10.0), dt=1e-3, nt=10, nbl=3,
            src_ijk=[[5, 5, 5]], rec_ijk=[[1, 2, 3], [4, 5, 6]])


@pytest.mark.parametrize("change,status,needle", [
    (dict(nx=0), -1, "grid sizes"),
    (dict(h=(10.0, -1.0, 10.0)), -1, "spacings"),
    (dict(dt=0.0), -1, "dt"),
    (dict(nt=-1), -1, "nt"),
    (dict(nbl=11), -1, "damping width"),
    (dict(src_ijk=[[20, 0, 0]]), -1, "source 0 outside"),
    (dict(rec_ijk=[[0, 0, 0], [0, -1, 0]]), -1, "receiver 1 outside"),
    (dict(order=6), -7, "order 8"),
])
def test_create_rejects_bad_configs(change, status, needle):
    kw = dict(GOOD)
    kw.update(change)
    with pytest.raises(M.MmodError) as ei:
        M.mmod_create(kw.pop("nx"), kw.pop("ny"), kw.pop("nz"), kw.pop("h"), kw.pop("dt"), kw.pop("nt"), **kw)
    assert ei.value.status == status
    assert needle in str(ei.value)


def test_product_never_reaches_the_oracle():
    pkg = os.path.join(ROOT, "paper_2007_06048_gb300")
    for path in glob.glob(os.path.join(pkg, "**", "*"), recursive=True):
        if os.path.isfile(path) and path.endswith((".py", ".cu", ".h", ".cuh", ".cpp")):
            text = open(path).read()
            for needle in ("import oracle", "from oracle", "liboracle", "orc_"):
                assert needle not in text, (path, needle)
