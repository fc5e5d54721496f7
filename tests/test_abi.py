"""The C-ABI library builds for sm_103a, loads, and exports every function that
include/front.h declares (no compute: this runs without a GPU)."""
import ctypes
import os
import re

from paper_2505_06932_gb300 import build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "front.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\**\s*([a-z_][a-z0-9_]*)\s*\(", src, flags=re.M)
    return sorted(set(names))


def test_header_declares_the_five_steps():
    names = declared_functions()
    for step in ("front_bin", "front_volume_fraction", "front_curvature_ppic", "front_csf_force",
                 "front_interp_velocity"):
        assert step in names


def test_library_exports_every_declared_symbol():
    lib = ctypes.CDLL(build.build())
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_status_strings():
    lib = ctypes.CDLL(build.build())
    lib.ft_status_string.restype = ctypes.c_char_p
    assert lib.ft_status_string(0) == b"ok"
    assert b"capacity" in lib.ft_status_string(-3)


def declared_signatures():
    """(name, [parameter declarations]) of every function include/front.h declares."""
    src = open(os.path.join(ROOT, "include", "front.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    out = []
    for m in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\**\s*([a-z_][a-z0-9_]*)\s*\(([^)]*)\)\s*;",
                         src, flags=re.M):
        params = [p.strip() for p in m.group(2).replace("\n", " ").split(",") if p.strip() and p.strip() != "void"]
        out.append((m.group(1), params))
    return out


def _ctype(decl):
    if "*" in decl:
        return ctypes.c_void_p
    if decl.split()[0] in ("int64_t", "size_t"):
        return ctypes.c_int64
    if decl.split()[0] == "double":
        return ctypes.c_double
    return ctypes.c_int32


def test_null_workspace_is_an_argument_error():
    """Every entry point that takes a workspace rejects a NULL one on the host
    with FT_ERR_ARG, before any CUDA call (so this runs without a GPU)."""
    lib = ctypes.CDLL(build.build())
    checked = []
    for name, params in declared_signatures():
        if not params or not re.match(r"^ft_workspace\s*\*\s*ws$", params[0]):
            continue
        fn = getattr(lib, name)
        fn.restype = ctypes.c_int32
        fn.argtypes = [_ctype(p) for p in params]
        args = [None if t is ctypes.c_void_p else 0 for t in fn.argtypes]
        assert fn(*args) == -1, name
        checked.append(name)
    for name in ("front_bin", "front_volume_fraction", "front_curvature_ppic", "front_csf_force",
                 "front_force_clear", "front_csf_force_cells", "front_force_clear_batch",
                 "front_csf_force_cells_batch", "front_bin_batch", "ft_batch_set"):
        assert name in checked
