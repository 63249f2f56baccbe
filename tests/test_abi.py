"""The C-ABI library builds for sm_103a, loads, and exports every entry point
that include/petvr.h declares (CPU only: no compute call is made)."""
import ctypes
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "petvr.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return set(re.findall(r"^\s*(?:pet_status|void|uint64_t|const char \*)\s*\*?\s*(pet_\w+)\s*\(", src, re.M))


def test_header_declares_the_boundary():
    names = _declared()
    for must in ("pet_plan_create", "pet_forward", "pet_back", "pet_osem_epoch", "pet_svrem_epoch",
                 "pet_saga_epoch", "pet_svrg_epoch", "pet_objective", "pet_problem_create",
                 "pet_state_create"):
        assert must in names


def test_library_exports_every_declared_symbol():
    from paper_2106_03172_gb300 import build
    path = build.build()
    lib = ctypes.CDLL(path)
    missing = [n for n in sorted(_declared()) if not hasattr(lib, n)]
    assert not missing, missing
    from paper_2106_03172_gb300 import petvr
    assert set(petvr._SIGS) == _declared()


def test_binding_refuses_to_run_without_library(tmp_path, monkeypatch):
    """No fallback: a missing shared object is an error, not a CPU path."""
    import importlib
    import pytest
    from paper_2106_03172_gb300 import petvr
    monkeypatch.setattr(petvr, "LIB_PATH", str(tmp_path / "missing.so"))
    monkeypatch.setattr(petvr, "_lib", None)
    with pytest.raises(RuntimeError, match="missing"):
        petvr.lib()
