"""The C-ABI library loads and exports every entry point include/sv.h
declares (no compute call: this runs without a GPU)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "sv.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(sv_[a-z_0-9]+)\s*\(", src)))


def test_header_declares_entry_points():
    names = declared_functions()
    for must in ["sv_create", "sv_apply_circuit", "sv_expect", "sv_grad", "sv_get_state", "sv_plan_qsu",
                 "sv_plan_evc", "sv_batch_run", "sv_destroy", "sv_last_error", "sv_vqe_step"]:
        assert must in names


def test_library_exports_every_declared_symbol():
    sv = pytest.importorskip("paper_2410_04252_gb300.sv")
    lib = ctypes.CDLL(sv.LIB_PATH)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing
    # the binding configures exactly the declared set
    assert set(sv.EXPORTS) == set(declared_functions())


def test_version_and_error_string():
    sv = pytest.importorskip("paper_2410_04252_gb300.sv")
    assert "sm_103a" in sv.version()
    assert isinstance(sv._lib.sv_last_error(), bytes)
