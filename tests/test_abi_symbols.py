"""The C-ABI library builds for sm_103a, loads, and exports every function
include/trime.h declares (no compute calls: no GPU needed)."""
import ctypes
import os
import re

HERE = os.path.dirname(os.path.abspath(__file__))
HDR = os.path.join(os.path.dirname(HERE), "include", "trime.h")


def declared_functions():
    src = open(HDR).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:const\s+)?\w+\s*\*?\s*((?:mesh|mlp)_\w+)\s*\(", src, flags=re.M)))


def test_library_exports_header_symbols():
    import paper_2309_13824_gb300 as g

    g.build()
    lib = ctypes.CDLL(str(g.LIB_PATH))
    names = declared_functions()
    assert len(names) >= 10
    for n in names:
        assert hasattr(lib, n), n
    assert sorted(g.EXPORTS) == names


def test_missing_library_fails_loudly(tmp_path, monkeypatch):
    import paper_2309_13824_gb300 as g

    monkeypatch.setattr(g, "LIB_PATH", tmp_path / "nope.so")
    monkeypatch.setattr(g, "_lib", None)
    try:
        g.lib()
    except RuntimeError as e:
        assert "missing" in str(e)
    else:
        raise AssertionError("no error without the library")
