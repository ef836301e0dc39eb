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


def test_binding_structs_match_the_header_layout(tmp_path):
    """Every struct the binding marshals has the header's size and field
    offsets (a C program compiled against include/tantrg.h prints them)."""
    import shutil
    import subprocess
    import pytest
    from paper_2212_11973_gb300 import tantrg
    cc = shutil.which("gcc") or shutil.which("cc")
    if not cc:
        pytest.skip("no C compiler")
    structs = {n: getattr(tantrg, n) for n in ("tt_alloc_cb", "tt_model", "tt_run_opts", "tt_obs", "tt_stats")}
    lines = ['#include <stddef.h>', '#include <stdio.h>', '#include "tantrg.h"', "int main(void) {"]
    for name, cls in structs.items():
        lines.append(f'  printf("{name} sizeof %zu\\n", sizeof({name}));')
        for f, _ in cls._fields_:
            lines.append(f'  printf("{name} {f} %zu\\n", offsetof({name}, {f}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run([cc, "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split("\n")
    got = {}
    for l in out:
        if l.strip():
            s, f, v = l.split()
            got[(s, f)] = int(v)
    for name, cls in structs.items():
        assert got[(name, "sizeof")] == ctypes.sizeof(cls), name
        for f, _ in cls._fields_:
            assert got[(name, f)] == getattr(cls, f).offset, (name, f)
