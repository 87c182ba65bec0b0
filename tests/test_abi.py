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


def declared_parameters(name):
    """Parameter names of `name` as include/*.h declares it."""
    for fn in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if not fn.endswith(".h"):
            continue
        text = re.sub(r"/\*.*?\*/", " ", open(os.path.join(ROOT, "include", fn)).read(), flags=re.S)
        m = re.search(r"\b" + name + r"\s*\(([^)]*)\)\s*;", text)
        if m:
            params = [p.strip() for p in m.group(1).split(",") if p.strip()]
            return [re.findall(r"[A-Za-z_]\w*", p)[-1] for p in params]
    return None


# The calls of the hot-path boundary, with their parameters in order (the
# problem statement and Alg. 1 fix what each call takes).
HOT_PATH = {
    "excmg_solve": ["n_finest", "n_coarsest", "bc_kind", "f", "g1", "g2", "tol", "u_out"],
    "stencil_apply": ["level", "transpose", "u", "y"],
    "bicg_solve": ["level", "b", "x_inout", "tol", "max_iter", "iters_out", "relres_out"],
    "extrapolate_interpolate": ["n_fine", "u_2h", "u_4h", "g1_fine", "w_h"],
    "midpoint_extrapolate": ["n_fine", "u_h", "u_2h", "u_tilde"],
}


def test_hot_path_signatures():
    for name, params in HOT_PATH.items():
        assert declared_parameters(name) == params, name
