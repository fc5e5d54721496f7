"""CPU oracle for the front/fluid coupling hot path (plain FP64 C, see oracle.c).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline / reference arm of ``bench.py`` may import this package.  It shares
no code with the CUDA library and never imports it.

``build()`` compiles ``oracle.c`` with gcc (``-std=c11 -ffp-contract=off``: no
fused multiply-add, so the binning predicate rounds as defined); the functions
below wrap the C entry points with numpy arrays.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

DEFAULT_PARAMS = dict(delta_h=2.5, delta_growth=1.25, delta_max_h=4.0, sigma=1.0, fit_min=24)


class _Grid(C.Structure):
    _fields_ = [("n", C.c_int32 * 3), ("pad", C.c_int32), ("origin", C.c_double * 3), ("h", C.c_double)]


class _Params(C.Structure):
    _fields_ = [("delta_h", C.c_double), ("delta_growth", C.c_double), ("delta_max_h", C.c_double),
                ("sigma", C.c_double), ("fit_min", C.c_int32), ("fit_ring", C.c_int32),
                ("frame_angle", C.c_double), ("frame_vertex", C.c_int32), ("pad", C.c_int32)]


def build(force: bool = False) -> str:
    """Compile the oracle into ``oracle/_build/liboracle.so`` (gcc, OpenMP if available)."""
    srcs = [os.path.join(_HERE, "oracle.c"), os.path.join(_HERE, "paraboloid.c")]
    hdr = os.path.join(_HERE, "oracle.h")
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= max([os.path.getmtime(x) for x in srcs] + [os.path.getmtime(hdr)])):
        return _LIB_PATH
    os.makedirs(_BUILD, exist_ok=True)
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    base = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
            *srcs, "-o", tmp, "-lm"]
    try:
        subprocess.run(base[:-3] + ["-fopenmp"] + base[-3:], check=True, capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base, check=True, capture_output=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = C.CDLL(_LIB_PATH)
            P = C.c_void_p
            L.og_bin.restype = C.c_int64
            L.og_bin.argtypes = [P, C.c_int64, P, C.c_int64, P, C.c_int32, C.c_int64, P, P, P]
            L.og_bin_bruteforce.restype = C.c_int64
            L.og_bin_bruteforce.argtypes = [P, C.c_int64, P, C.c_int64, P, C.c_int64, P, P]
            L.og_clip_fragment.restype = C.c_int
            L.og_clip_fragment.argtypes = [P, P, C.c_int32, C.c_int32, C.c_int32, P]
            L.og_alpha.restype = C.c_int
            L.og_alpha.argtypes = [P, C.c_int64, P, C.c_int64, P, C.c_int32, P, P]
            L.og_ppic.restype = C.c_int
            L.og_ppic.argtypes = [P, C.c_int64, P, C.c_int64, P, P, C.c_int64, P, P, P, P, P, P]
            L.og_closest_vertex.restype = None
            L.og_closest_vertex.argtypes = [P, C.c_int64, P, C.c_int64, P, C.c_int64, P, P, P]
            L.og_ring.restype = C.c_int64
            L.og_ring.argtypes = [C.c_int64, P, C.c_int64, C.c_int64, C.c_int32, P, C.c_int64]
            L.og_csf.restype = C.c_int
            L.og_csf.argtypes = [P, P, C.c_int64, P, P, P, C.c_double, P]
            L.og_face_force.restype = C.c_int
            L.og_face_force.argtypes = [P, P, C.c_int64, P, P, P, C.c_double, P, P, P]
            L.og_roughness.restype = C.c_int
            L.og_roughness.argtypes = [P, C.c_int64, P, C.c_int64, P, P, P, P, P, P, P]
            L.og_roughness_smooth.restype = C.c_int
            L.og_roughness_smooth.argtypes = [P, C.c_int64, P, C.c_int64, C.c_double, C.c_double, C.c_int, P]
            L.og_edge_priority.restype = C.c_uint64
            L.og_edge_priority.argtypes = [C.c_uint64]
            L.og_interp.restype = None
            L.og_interp.argtypes = [P, P, P, P, P, C.c_int64, P]
            L.og_advect_rk4.restype = None
            L.og_advect_rk4.argtypes = [P, P, P, P, P, C.c_int64, C.c_double, P, P]
            L.og_green_moments.restype = None
            L.og_paraboloid_cells.argtypes = [C.c_int64, P, P, P, P, P, P, P]
            L.og_paraboloid_cells.restype = None
            L.og_green_moments.argtypes = [P, P, C.c_int, P]
            L.og_signed_volume.restype = C.c_double
            L.og_signed_volume.argtypes = [P, P, C.c_int64]
            L.og_wendland_weight.restype = C.c_double
            L.og_wendland_weight.argtypes = [C.c_double]
            L.og_set_threads.restype = None
            L.og_set_threads.argtypes = [C.c_int]
            L.og_get_threads.restype = C.c_int
            L.og_get_threads.argtypes = []
            _lib = L
    return _lib


def _ptr(a):
    return a.ctypes.data_as(C.c_void_p)


def _grid(g):
    s = _Grid()
    for d in range(3):
        s.n[d] = int(g.n[d])
        s.origin[d] = float(g.origin[d])
    s.h = float(g.h)
    return s


def _front(verts, tris):
    v = np.ascontiguousarray(verts, dtype=np.float64)
    t = np.ascontiguousarray(tris, dtype=np.int32)
    return v, t


def margin_for(delta_max_h: float = DEFAULT_PARAMS["delta_max_h"]) -> int:
    """Cells that must separate the front's candidate cells from the grid boundary."""
    import math
    return 2 + int(math.ceil(delta_max_h))


def set_threads(n: int) -> None:
    lib().og_set_threads(int(n))


def get_threads() -> int:
    return int(lib().og_get_threads())


def bin_pairs(verts, tris, g, margin=None):
    """Sorted (cell key, triangle) pairs of the canonical binning predicate and the status bits."""
    v, t = _front(verts, tris)
    gs = _grid(g)
    m = margin_for() if margin is None else margin
    st = np.zeros(1, np.uint32)
    L = lib()
    cap = max(16, 8 * t.shape[0])
    while True:
        keys = np.empty(cap, np.uint32)
        tid = np.empty(cap, np.int32)
        n = L.og_bin(_ptr(v), v.shape[0], _ptr(t), t.shape[0], C.byref(gs), m, cap, _ptr(keys), _ptr(tid), _ptr(st))
        if n <= cap:
            return keys[:n].copy(), tid[:n].copy(), int(st[0])
        cap = int(n)
        st[0] = 0


def bin_pairs_bruteforce(verts, tris, g):
    v, t = _front(verts, tris)
    gs = _grid(g)
    cap = max(16, 64 * t.shape[0])
    keys = np.empty(cap, np.uint32)
    tid = np.empty(cap, np.int32)
    n = lib().og_bin_bruteforce(_ptr(v), v.shape[0], _ptr(t), t.shape[0], C.byref(gs), cap, _ptr(keys), _ptr(tid))
    assert n <= cap
    return keys[:n].copy(), tid[:n].copy()


def clip_fragment(tri_xyz, g, i, j, k):
    """Fragment polygon (n, 3) of the canonical clip of one triangle against cell (i,j,k), or None."""
    tri = np.ascontiguousarray(tri_xyz, dtype=np.float64).reshape(9)
    out = np.empty((32, 3), np.float64)
    gs = _grid(g)
    n = lib().og_clip_fragment(_ptr(tri), C.byref(gs), int(i), int(j), int(k), _ptr(out))
    return out[:n].copy() if n else None


def interfacial_cells(verts, tris, g, margin=None):
    keys, _, st = bin_pairs(verts, tris, g, margin)
    return np.unique(keys), st


def alpha(verts, tris, g, margin=None):
    """Dense volume fractions (n0, n1, n2) and status bits."""
    v, t = _front(verts, tris)
    gs = _grid(g)
    m = margin_for() if margin is None else margin
    out = np.empty(tuple(int(x) for x in g.n), np.float64)
    st = np.zeros(1, np.uint32)
    lib().og_alpha(_ptr(v), v.shape[0], _ptr(t), t.shape[0], C.byref(gs), m, _ptr(out), _ptr(st))
    return out, int(st[0])


def ppic(verts, tris, g, cells, params=None, frame_angle=0.0, frame=False):
    """PPIC curvature, paraboloid normal, coefficients and status in the given
    cells (and, with ``frame=True``, each cell's frame (t1, t2, n) as (M, 9)).
    params may set fit_ring (0: fragments; k: whole triangles of the k-ring of
    the closest vertex) and frame_vertex (1: the closest vertex's normal)."""
    p = dict(DEFAULT_PARAMS)
    if params:
        p.update(params)
    ps = _Params(p["delta_h"], p["delta_growth"], p["delta_max_h"], p["sigma"], int(p["fit_min"]),
                 int(p.get("fit_ring", 0)), float(frame_angle), int(p.get("frame_vertex", 0)), 0)
    v, t = _front(verts, tris)
    gs = _grid(g)
    cells = np.ascontiguousarray(cells, dtype=np.uint32)
    M = cells.shape[0]
    kappa = np.empty(M, np.float64)
    normal = np.empty((M, 3), np.float64)
    coeffs = np.empty((M, 6), np.float64)
    status = np.empty(M, np.int8)
    fr = np.empty((M, 9), np.float64)
    rc = lib().og_ppic(_ptr(v), v.shape[0], _ptr(t), t.shape[0], C.byref(gs), C.byref(ps), M, _ptr(cells),
                       _ptr(kappa), _ptr(normal), _ptr(coeffs), _ptr(status), _ptr(fr))
    if rc != 0:
        raise ValueError("og_ppic: a listed cell is not interfacial")
    if frame:
        return kappa, normal, coeffs, status, fr
    return kappa, normal, coeffs, status


def closest_vertex(verts, tris, g, cells):
    """Per cell the index of the front vertex closest to its centre and that
    vertex's normal (M, 3)."""
    v, t = _front(verts, tris)
    cells = np.ascontiguousarray(cells, dtype=np.uint32)
    idx = np.empty(cells.shape[0], np.int32)
    nrm = np.empty((cells.shape[0], 3), np.float64)
    lib().og_closest_vertex(_ptr(v), v.shape[0], _ptr(t), t.shape[0], C.byref(_grid(g)), cells.shape[0],
                            _ptr(cells), _ptr(idx), _ptr(nrm))
    return idx, nrm


def ring(verts, tris, v, k):
    """The k-ring of triangles around vertex v, ascending triangle ids."""
    vv, t = _front(verts, tris)
    cap = 4096
    out = np.empty(cap, np.int32)
    n = lib().og_ring(vv.shape[0], _ptr(t), t.shape[0], int(v), int(k), _ptr(out), cap)
    assert n <= cap
    return out[:n].copy()


def csf(g, alpha_dense, cells, kappa, normal, sigma=1.0):
    """Dense CSF force (3, n0, n1, n2)."""
    a = np.ascontiguousarray(alpha_dense, dtype=np.float64)
    cells = np.ascontiguousarray(cells, dtype=np.uint32)
    k = np.ascontiguousarray(kappa, dtype=np.float64)
    n = np.ascontiguousarray(normal, dtype=np.float64)
    out = np.empty((3,) + tuple(int(x) for x in g.n), np.float64)
    gs = _grid(g)
    lib().og_csf(C.byref(gs), _ptr(a), cells.shape[0], _ptr(cells), _ptr(k), _ptr(n), float(sigma), _ptr(out))
    return out


def face_force(g, alpha_dense, cells, kappa, normal, sigma=1.0):
    """Balanced-force face term on the three staggered face arrays (Fx, Fy, Fz)."""
    a = np.ascontiguousarray(alpha_dense, dtype=np.float64)
    cells = np.ascontiguousarray(cells, dtype=np.uint32)
    k = np.ascontiguousarray(kappa, dtype=np.float64)
    nrm = np.ascontiguousarray(normal, dtype=np.float64)
    n = [int(x) for x in g.n]
    out = [np.empty(tuple(n[e] + (1 if e == d else 0) for e in range(3)), np.float64) for d in range(3)]
    gs = _grid(g)
    lib().og_face_force(C.byref(gs), _ptr(a), cells.shape[0], _ptr(cells), _ptr(k), _ptr(nrm), float(sigma),
                        _ptr(out[0]), _ptr(out[1]), _ptr(out[2]))
    return tuple(out)


def interp(g, faces, pts):
    """Divergence-preserving interpolated velocities (np, 3)."""
    U, V, W = (np.ascontiguousarray(f, dtype=np.float64) for f in faces)
    p = np.ascontiguousarray(pts, dtype=np.float64).reshape(-1, 3)
    out = np.empty_like(p)
    gs = _grid(g)
    lib().og_interp(C.byref(gs), _ptr(U), _ptr(V), _ptr(W), _ptr(p), p.shape[0], _ptr(out))
    return out


def advect_rk4(g, faces, pts, dt):
    """One classical RK4 step of the points in the interpolated velocity of the
    (fixed) face field: returns (new positions (np, 3), k1 velocities (np, 3))."""
    U, V, W = (np.ascontiguousarray(f, dtype=np.float64) for f in faces)
    p = np.ascontiguousarray(pts, dtype=np.float64).reshape(-1, 3)
    out = np.empty_like(p)
    vel = np.empty_like(p)
    gs = _grid(g)
    lib().og_advect_rk4(C.byref(gs), _ptr(U), _ptr(V), _ptr(W), _ptr(p), p.shape[0], C.c_double(dt), _ptr(out),
                        _ptr(vel))
    return out, vel


def roughness(verts, tris):
    """Local roughness metrics (Sec. 3.4): dict of gl (nv, 3), rough, r1, r2,
    G, V (nv) and rt (nt)."""
    v = np.ascontiguousarray(verts, dtype=np.float64)
    t = np.ascontiguousarray(tris, dtype=np.int32)
    nv, nt = v.shape[0], t.shape[0]
    out = dict(gl=np.empty((nv, 3)), rough=np.empty(nv), r1=np.empty(nv), r2=np.empty(nv), rt=np.empty(nt),
               G=np.empty(nv), V=np.empty(nv))
    lib().og_roughness(_ptr(v), nv, _ptr(t), nt, _ptr(out["gl"]), _ptr(out["rough"]), _ptr(out["r1"]),
                       _ptr(out["r2"]), _ptr(out["rt"]), _ptr(out["G"]), _ptr(out["V"]))
    return out


def roughness_smooth(verts, tris, gl_thr, r_thr, max_rounds=64):
    """Local roughness smoothing; returns (new verts, rounds, edges moved)."""
    v = np.array(verts, dtype=np.float64, order="C", copy=True)
    t = np.ascontiguousarray(tris, dtype=np.int32)
    moved = C.c_int64(0)
    rounds = lib().og_roughness_smooth(_ptr(v), v.shape[0], _ptr(t), t.shape[0], float(gl_thr), float(r_thr),
                                       int(max_rounds), C.byref(moved))
    return v, rounds, moved.value


def edge_priority(e):
    return int(lib().og_edge_priority(int(e)))


def paraboloid_cells(frame, coeffs):
    """The paper's cut-cell quantities from fitted paraboloids (Sec. 3.2): per
    cell alpha = V_P / V_C, the surface area inside the cell (cell units), the
    area-averaged mean curvature (1 / cell width) and the normalised
    area-integrated normal; status 1 where the surface misses the cell."""
    fr = np.ascontiguousarray(np.asarray(frame, dtype=np.float64).reshape(-1, 9))
    co = np.ascontiguousarray(np.asarray(coeffs, dtype=np.float64).reshape(-1, 6))
    m = fr.shape[0]
    assert co.shape[0] == m
    out = dict(alpha=np.empty(m), area=np.empty(m), kbar=np.empty(m), nbar=np.empty((m, 3)),
               status=np.empty(m, np.int8))
    lib().og_paraboloid_cells(m, _ptr(fr), _ptr(co), _ptr(out["alpha"]), _ptr(out["area"]), _ptr(out["kbar"]),
                              _ptr(out["nbar"]), _ptr(out["status"]))
    return out


def green_moments(x, y):
    x = np.ascontiguousarray(x, dtype=np.float64)
    y = np.ascontiguousarray(y, dtype=np.float64)
    m = np.empty(6, np.float64)
    lib().og_green_moments(_ptr(x), _ptr(y), x.shape[0], _ptr(m))
    return m


def signed_volume(verts, tris):
    v, t = _front(verts, tris)
    return float(lib().og_signed_volume(_ptr(v), _ptr(t), t.shape[0]))


def wendland(q):
    return float(lib().og_wendland_weight(float(q)))
