"""The C-ABI library builds and exports every symbol declared in include/fv3.h
(no compute call: this runs without a GPU)."""
import ctypes
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared():
    txt = open(os.path.join(ROOT, "include", "fv3.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(fv3_[a-z_0-9]+)\s*\(", txt)))


def test_library_exports_header_symbols():
    from paper_2205_04148_gb300 import build, fv3
    lib = build.build()
    L = ctypes.CDLL(lib)
    names = declared()
    assert "fv3_acoustic_substep" in names and "fv3_run_dyn" in names
    for nm in names:
        assert hasattr(L, nm), nm
    assert set(fv3.SYMBOLS) <= set(names)


def test_null_arguments_rejected_without_gpu():
    from paper_2205_04148_gb300 import build, fv3
    build.build()
    L = fv3.load()
    assert L.fv3_init_grid(None, None, None) == -1
    assert L.fv3_acoustic_substep(None, None, None, None) == -1
    assert L.fv3_last_error(None) == b"no context"
