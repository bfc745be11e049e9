"""The C-ABI library builds for sm_103a, loads without a GPU, and exports
exactly the entry points declared in include/roks.h (no compute calls)."""
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    txt = open(os.path.join(ROOT, "include", "roks.h")).read()
    return sorted(set(re.findall(r"ROKS_API\s+[\w\s\*]*?\b(roks_\w+)\s*\(", txt)))


def test_header_declares_boundary():
    names = declared_symbols()
    for must in ("roks_setup", "roks_density", "roks_potential", "roks_apply_h", "roks_orthonormalize",
                 "roks_pcg_step", "roks_destroy"):
        assert must in names


def test_library_loads_and_exports_every_symbol():
    import __graft_entry__ as g
    g.build()
    from paper_2605_28637_gb300 import roks
    lib = roks.load()
    for name in declared_symbols():
        assert hasattr(lib, name), name
    out = subprocess.run(["nm", "-D", "--defined-only", roks.LIB_PATH], capture_output=True, text=True)
    if out.returncode == 0:
        exported = sorted(set(re.findall(r" T (roks_\w+)", out.stdout)))
        assert exported == declared_symbols()
    assert sorted(roks.EXPORTS) == declared_symbols()


def test_binding_fails_loudly_without_library(tmp_path):
    from paper_2605_28637_gb300 import roks
    saved = roks._lib
    roks._lib = None
    try:
        with pytest.raises(FileNotFoundError):
            roks.load(str(tmp_path / "missing.so"))
    finally:
        roks._lib = saved


def test_oracle_not_reachable_from_product():
    """The package and the CUDA sources never mention the oracle."""
    pkg = os.path.join(ROOT, "paper_2605_28637_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                txt = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in txt and "from oracle" not in txt, f
