"""The C-ABI library loads and exports every function include/excmg.h declares
(no compute calls: this runs without a GPU)."""
import ctypes
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for fn in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if not fn.endswith(".h"):
            continue
        text = open(os.path.join(ROOT, "include", fn)).read()
        text = re.sub(r"/\*.*?\*/", " ", text, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][\w\s\*]*?\b([a-z_][a-z0-9_]*)\s*\(", text, flags=re.M):
            name = m.group(1)
            if name not in ("if", "while", "for", "return", "sizeof"):
                names.add(name)
    return names


def test_header_declares_the_hot_path():
    names = declared_functions()
    for required in ("excmg_solve", "stencil_apply", "bicg_solve", "extrapolate_interpolate",
                     "midpoint_extrapolate"):
        assert required in names


def test_library_exports_every_declared_symbol():
    from paper_1901_05118_gb300 import build as b
    lib_path = b.build()
    lib = ctypes.CDLL(lib_path)
    missing = [n for n in sorted(declared_functions()) if not hasattr(lib, n)]
    assert not missing, f"not exported: {missing}"
