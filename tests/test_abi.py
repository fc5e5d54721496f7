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
