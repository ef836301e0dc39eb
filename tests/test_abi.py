"""The C-ABI library builds for sm_103a, loads without a GPU and exports every
function that include/tantrg.h declares (no compute calls here)."""
import ctypes
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"\b(tt_\w+)\s*\(", src))
    return names


def test_library_exports_every_declared_symbol():
    from paper_2212_11973_gb300 import build
    lib_path = build.build()
    lib = ctypes.CDLL(lib_path)
    names = _declared()
    assert len(names) >= 15
    missing = [n for n in sorted(names) if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_declares_the_same_functions():
    from paper_2212_11973_gb300 import tantrg
    assert set(tantrg.SIGNATURES) <= _declared()
    assert _declared() - set(tantrg.SIGNATURES) <= {"tt_batch_create", "tt_batch_step", "tt_batch_measure",
                                                    "tt_batch_destroy"}


def test_missing_library_fails_loudly(tmp_path):
    from paper_2212_11973_gb300 import tantrg
    import pytest
    with pytest.raises(RuntimeError, match="no fallback"):
        tantrg._lib, saved = None, tantrg._lib
        try:
            tantrg.load_library(str(tmp_path / "absent.so"))
        finally:
            tantrg._lib = saved
