"""CPU-only checks of the C-ABI library: it builds, loads, exports every entry
point include/mpm.h declares, and the binding refuses to run without it."""
import ctypes
import os
import re

import pytest

from paper_1905_00671_gb300 import build as B

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    text = open(os.path.join(ROOT, "include", "mpm.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(mpm_\w+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    path = B.build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("mpm_create", "mpm_step", "mpm_read", "mpm_destroy", "mpm_get_stats",
                     "mpm_last_error", "mpm_default_options"):
        assert required in names


def test_every_declared_symbol_is_exported(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_default_options_without_gpu(lib):
    from paper_1905_00671_gb300 import mpm

    o = mpm.default_options()
    assert o.shape == mpm.MPM_SHAPE_GIMP and o.newton_rtol == 1e-8 and o.krylov_restart == 120
    assert o.precond_lag == 2
    assert o.precond == mpm.MPM_PRECOND_SCHUR_MG


def test_binding_fails_loudly_without_library(monkeypatch, tmp_path):
    from paper_1905_00671_gb300 import mpm

    monkeypatch.setattr(B, "SO", str(tmp_path / "missing.so"))
    monkeypatch.setattr(mpm, "_lib", None)
    with pytest.raises(RuntimeError, match="not built"):
        mpm.load()


def test_product_path_never_imports_the_oracle():
    pkg = os.path.join(ROOT, "paper_1905_00671_gb300")
    for dirpath, _, files in os.walk(pkg):
        if "_build" in dirpath:
            continue
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                src = open(os.path.join(dirpath, f)).read()
                assert "oracle" not in re.sub(r"#.*|//.*", "", src).lower() or f == "inputs.py", f
