"""ctypes binding of libfront.so (C ABI in include/front.h).

Argument marshalling only: every step runs in the library's CUDA kernels.  The
functions take torch CUDA tensors (device memory and the current stream come
from PyTorch) and keep the C names.  There is no CPU fallback: if the library
cannot be built or loaded, ``lib()`` raises.
"""
from __future__ import annotations

import ctypes as C
import threading

import torch

from . import build as _build

_lock = threading.Lock()
_lib = None

FT_FP64, FT_FP32C = 0, 1
ST_BITS = {0x01: "capacity", 0x02: "outside_grid", 0x04: "not_closed", 0x08: "orientation",
           0x10: "bad_index", 0x20: "timeout"}


class FtGrid(C.Structure):
    _fields_ = [("n", C.c_int32 * 3), ("pad", C.c_int32), ("origin", C.c_double * 3), ("h", C.c_double)]


class FtFront(C.Structure):
    _fields_ = [("verts", C.c_void_p), ("nv", C.c_int64), ("tris", C.c_void_p), ("nt", C.c_int64)]


class FtParams(C.Structure):
    _fields_ = [("delta_h", C.c_double), ("delta_growth", C.c_double), ("delta_max_h", C.c_double),
                ("sigma", C.c_double), ("fit_min", C.c_int32), ("precision", C.c_int32), ("fit_ring", C.c_int32),
                ("frame", C.c_int32)]


class FtCapacity(C.Structure):
    _fields_ = [("max_nt", C.c_int64), ("max_cand", C.c_int64), ("max_cells", C.c_int64)]


class FtBatchFront(C.Structure):
    _fields_ = [("grid", FtGrid), ("verts", C.c_void_p), ("nv", C.c_int64), ("tris", C.c_void_p), ("nt", C.c_int64),
                ("alpha", C.c_void_p), ("force", C.c_void_p), ("U", C.c_void_p), ("V", C.c_void_p),
                ("W", C.c_void_p), ("vel", C.c_void_p), ("verts_next", C.c_void_p), ("dt", C.c_double),
                ("face_force", C.c_void_p * 3)]


class FtBatchCapacity(C.Structure):
    _fields_ = [("max_fronts", C.c_int32), ("pad", C.c_int32), ("max_grid_cells", C.c_int64),
                ("max_nt", C.c_int64), ("max_cand", C.c_int64), ("max_cells", C.c_int64)]


class FtTuning(C.Structure):
    _fields_ = [("clip_blocks_per_sm", C.c_int32), ("ppic_blocks_per_sm", C.c_int32),
                ("csf_blocks_per_sm", C.c_int32), ("fill_blocks_per_sm", C.c_int32),
                ("ppic_min_blocks", C.c_int32), ("ppic_dynamic", C.c_int32), ("sort_blocks", C.c_int32),
                ("pad", C.c_int32), ("cand_need", C.c_int64), ("cells_need", C.c_int64), ("fit_pairs", C.c_int64),
                ("step_ms", C.c_double)]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_}


class FrontError(RuntimeError):
    pass


def lib():
    """Load libfront.so (building it first if it is missing or stale)."""
    global _lib
    with _lock:
        if _lib is None:
            path = _build.build()
            L = C.CDLL(path)
            P, I64, I32 = C.c_void_p, C.c_int64, C.c_int
            sig = {
                "ft_workspace_create": (I32, [C.POINTER(P), P, P, I32, C.POINTER(C.c_size_t)]),
                "ft_workspace_destroy": (I32, [P]),
                "ft_status": (I32, [P, P, C.POINTER(C.c_uint32)]),
                "ft_counts": (I32, [P, P, P]),
                "ft_status_string": (C.c_char_p, [I32]),
                "ft_bin_pairs": (I32, [P, I64, P, P, P]),
                "front_bin": (I32, [P, P, P, P]),
                "front_volume_fraction": (I32, [P, P, P]),
                "front_curvature_ppic": (I32, [P, P, I64, P, P, P, P, P, P]),
                "front_csf_force": (I32, [P, P, P, P, P, P, P]),
                "front_force_clear": (I32, [P, P, P]),
                "front_csf_prepare": (I32, [P, P]),
                "front_csf_force_cells": (I32, [P, P, P, P, P, P, P]),
                "front_interp_velocity": (I32, [P, P, P, P, P, I64, P, P]),
                "ft_probe_fma_rate": (I32, [I32, I32, C.POINTER(C.c_double)]),
                "ft_launch_count": (I64, []),
                "ft_work_counts": (I32, [P, P, P, I32]),
                "front_csf_force_compact": (I32, [P, P, P, P, P, I64, P, P, P, P]),
                "front_alpha_pack": (I32, [P, P, I64, P, P, P]),
                "ft_trace_start": (I32, [I64]),
                "ft_trace_stop": (I32, [I32, P, P, P, C.POINTER(C.c_int32), C.POINTER(C.c_int64)]),
                "ft_volume_fraction_noalloc": (I32, [P, P, P, P, P, P]),
                "ft_batch_workspace_create": (I32, [C.POINTER(P), P, I32, C.POINTER(C.c_size_t)]),
                "ft_batch_set": (I32, [P, I32, P, P]),
                "front_bin_batch": (I32, [P, P, P]),
                "front_volume_fraction_batch": (I32, [P, P]),
                "front_csf_force_batch": (I32, [P, P, P, P, P]),
                "front_force_clear_batch": (I32, [P, P]),
                "front_csf_force_cells_batch": (I32, [P, P, P, P, P]),
                "front_interp_velocity_batch": (I32, [P, P]),
                "ft_batch_cell_ranges": (I32, [P, P, P]),
                "ft_batch_status": (I32, [P, P, P]),
                "ft_set_tuning": (I32, [P, P]),
                "ft_get_tuning": (I32, [P, P]),
                "ft_autotune": (I32, [P, P, P, I32, P, P]),
                "front_advect_rk4": (I32, [P, P, P, P, P, I64, C.c_double, P, P, P]),
                "front_advect_rk4_batch": (I32, [P, P]),
                "front_face_force": (I32, [P, P, P, P, P, P, P, P, P]),
                "front_face_force_batch": (I32, [P, P, P, P, P]),
                "front_paraboloid_cells": (I32, [P, P, I64, P, P, P, P, P, P]),
                "front_ppic_frame": (I32, [P, I64, P, P]),
                "front_volume_fraction_ppic": (I32, [P, P, I64, P, P, P, P, P, P]),
                "front_volume_fraction_ppic_batch": (I32, [P, P, I64, P, P, P, P, P]),
                "ft_rough_create": (I32, [C.POINTER(P), I64, I64, I32, C.POINTER(C.c_size_t)]),
                "ft_rough_destroy": (I32, [P]),
                "ft_rough_status": (I32, [P, P, C.POINTER(C.c_uint32)]),
                "front_roughness": (I32, [P, P, I64, P, I64, P, P, P, P, P, P, P, P]),
                "front_roughness_smooth": (I32, [P, P, I64, P, I64, C.c_double, C.c_double, I32,
                                                 C.POINTER(C.c_int32), C.POINTER(C.c_int64),
                                                 C.POINTER(C.c_uint32), P]),
            }
            for name, (res, args) in sig.items():
                fn = getattr(L, name)
                fn.restype = res
                fn.argtypes = args
            _lib = L
    return _lib


def _check(rc: int, what: str):
    if rc != 0:
        msg = lib().ft_status_string(rc).decode()
        raise FrontError(f"{what}: {msg} ({rc})")


def _stream(stream=None):
    s = torch.cuda.current_stream() if stream is None else stream
    return C.c_void_p(s.cuda_stream)


def _ptr(t: torch.Tensor, dtype, what: str):
    if t is None:
        return None
    if not t.is_cuda:
        raise FrontError(f"{what} must be a CUDA tensor")
    if t.dtype != dtype:
        raise FrontError(f"{what} must be {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise FrontError(f"{what} must be contiguous")
    return C.c_void_p(t.data_ptr())


def _ptr_faces(t: torch.Tensor, what: str):
    """A face array: a CUDA tensor, or a page-locked host tensor that the
    kernel reads in place (mapped host memory)."""
    if t is not None and not t.is_cuda:
        if not t.is_pinned():
            raise FrontError(f"{what} must be a CUDA tensor or pinned host memory")
        if t.dtype != torch.float64 or not t.is_contiguous():
            raise FrontError(f"{what} must be contiguous float64")
        return C.c_void_p(t.data_ptr())
    return _ptr(t, torch.float64, what)


def make_grid(g) -> FtGrid:
    s = FtGrid()
    for d in range(3):
        s.n[d] = int(g.n[d])
        s.origin[d] = float(g.origin[d])
    s.h = float(g.h)
    return s


FT_FRAME_FRAGMENTS, FT_FRAME_VERTEX = 0, 1


def make_params(delta_h=2.5, delta_growth=1.25, delta_max_h=4.0, sigma=1.0, fit_min=24, precision=FT_FP64,
                fit_ring=0, frame=FT_FRAME_FRAGMENTS):
    """ft_params; fit_ring = k > 0 and frame = FT_FRAME_VERTEX select the
    paper's own PPIC neighbourhood (whole triangles of the k-ring of the
    closest front vertex) and frame (that vertex's normal)."""
    return FtParams(float(delta_h), float(delta_growth), float(delta_max_h), float(sigma), int(fit_min),
                    int(precision), int(fit_ring), int(frame))


class Workspace:
    """Library-owned device memory for one grid shape (ft_workspace_create)."""

    def __init__(self, grid, max_nt: int, max_cand: int = 0, max_cells: int = 0, device: int = 0):
        self.grid = grid
        self._g = make_grid(grid)
        cap = FtCapacity(int(max_nt), int(max_cand), int(max_cells))
        h = C.c_void_p()
        nbytes = C.c_size_t()
        _check(lib().ft_workspace_create(C.byref(h), C.byref(self._g), C.byref(cap), int(device), C.byref(nbytes)),
               "ft_workspace_create")
        self.handle = h
        self.bytes = int(nbytes.value)
        self.device = device

    def close(self):
        if self.handle:
            lib().ft_workspace_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def status(self, stream=None) -> int:
        bits = C.c_uint32()
        _check(lib().ft_status(self.handle, _stream(stream), C.byref(bits)), "ft_status")
        return int(bits.value)

    def counts(self, stream=None) -> dict:
        out = (C.c_int64 * 5)()
        _check(lib().ft_counts(self.handle, _stream(stream), out), "ft_counts")
        return dict(M=out[0], P=out[1], C=out[2], C_need=out[3], fit_pairs=out[4])

    def work_counts(self, stream=None) -> dict:
        """ft_work_counts: the work of the last calls (per-kernel roofline units)."""
        out = (C.c_int64 * 8)()
        _check(lib().ft_work_counts(self.handle, _stream(stream), C.cast(out, C.c_void_p), 8), "ft_work_counts")
        return dict(T=out[0], M=out[1], P=out[2], C=out[3], C_need=out[4], fit_pairs=out[5], clip_f64=out[6],
                    ring=out[7])


class BatchWorkspace(Workspace):
    """Library-owned device memory for a batch of fronts (ft_batch_workspace_create).
    ``set_fronts`` installs the table; the tensors it references are kept alive here."""

    def __init__(self, max_fronts: int, max_grid_cells: int, max_nt: int, max_cand: int = 0, max_cells: int = 0,
                 device: int = 0):
        cap = FtBatchCapacity(int(max_fronts), 0, int(max_grid_cells), int(max_nt), int(max_cand), int(max_cells))
        h = C.c_void_p()
        nbytes = C.c_size_t()
        _check(lib().ft_batch_workspace_create(C.byref(h), C.byref(cap), int(device), C.byref(nbytes)),
               "ft_batch_workspace_create")
        self.handle = h
        self.bytes = int(nbytes.value)
        self.device = device
        self.grid = None
        self.nf = 0
        self._keep = []

    def set_fronts(self, fronts, stream=None):
        """fronts: list of dicts with keys grid, verts, tris and optionally
        alpha, force, U, V, W, vel (CUDA tensors)."""
        arr = (FtBatchFront * len(fronts))()
        keep = []
        for b, f in enumerate(fronts):
            e = arr[b]
            e.grid = make_grid(f["grid"])
            n = f["grid"].n
            e.verts = _ptr(f["verts"], torch.float64, "verts")
            e.nv = f["verts"].shape[0]
            e.tris = _ptr(f["tris"], torch.int32, "tris")
            e.nt = f["tris"].shape[0]
            nc = int(n[0]) * int(n[1]) * int(n[2])
            for name, size in (("alpha", nc), ("force", 3 * nc), ("vel", 3 * e.nv), ("verts_next", 3 * e.nv)):
                t = f.get(name)
                if t is not None and t.numel() != size:
                    raise FrontError(f"front {b}: {name} must hold {size} values")
                setattr(e, name, _ptr(t, torch.float64, name) if t is not None else None)
            for name, shp in (("U", (n[0] + 1, n[1], n[2])), ("V", (n[0], n[1] + 1, n[2])),
                              ("W", (n[0], n[1], n[2] + 1))):
                t = f.get(name)
                if t is not None and tuple(t.shape) != tuple(int(x) for x in shp):
                    raise FrontError(f"front {b}: {name} has the wrong shape")
                setattr(e, name, _ptr(t, torch.float64, name) if t is not None else None)
            e.dt = float(f.get("dt", 0.0))
            ff = f.get("face_force")
            if ff is not None:
                for d in range(3):
                    shp = tuple(int(n[e2]) + (1 if e2 == d else 0) for e2 in range(3))
                    if tuple(ff[d].shape) != shp:
                        raise FrontError(f"front {b}: face_force[{d}] must have shape {shp}")
                    e.face_force[d] = _ptr(ff[d], torch.float64, "face_force")
            keep.append(f)
        _check(lib().ft_batch_set(self.handle, len(fronts), arr, _stream(stream)), "ft_batch_set")
        self._keep = keep
        self.nf = len(fronts)

    def front_status(self, stream=None):
        out = (C.c_uint32 * max(self.nf, 1))()
        _check(lib().ft_batch_status(self.handle, _stream(stream), out), "ft_batch_status")
        return [int(out[b]) for b in range(self.nf)]


def ft_bin_pairs(ws: Workspace, keys: torch.Tensor, tris: torch.Tensor, stream=None):
    cap = min(keys.shape[0], tris.shape[0])
    _check(lib().ft_bin_pairs(ws.handle, cap, _ptr(keys, torch.int32, "keys"), _ptr(tris, torch.int32, "tris"),
                              _stream(stream)), "ft_bin_pairs")


def status_names(bits: int):
    return [v for k, v in ST_BITS.items() if bits & k]


# ---------------------------------------------------------------------------
# the five steps, one C call each
# ---------------------------------------------------------------------------

def front_bin(ws: Workspace, verts: torch.Tensor, tris: torch.Tensor, params: FtParams, stream=None):
    f = FtFront(_ptr(verts, torch.float64, "verts"), verts.shape[0], _ptr(tris, torch.int32, "tris"), tris.shape[0])
    _check(lib().front_bin(ws.handle, C.byref(f), C.byref(params), _stream(stream)), "front_bin")


def front_volume_fraction(ws: Workspace, alpha: torch.Tensor, stream=None):
    if alpha.numel() != ws.grid.ncells:
        raise FrontError("alpha must hold n0*n1*n2 values")
    _check(lib().front_volume_fraction(ws.handle, _ptr(alpha, torch.float64, "alpha"), _stream(stream)),
           "front_volume_fraction")


def front_curvature_ppic(ws: Workspace, params: FtParams, cell_keys, kappa, normal, coeffs, fit_status, stream=None):
    cap = kappa.shape[0]
    if cell_keys.shape[0] < cap or normal.shape[0] < cap or fit_status.shape[0] < cap:
        raise FrontError("PPIC output arrays are shorter than kappa")
    _check(lib().front_curvature_ppic(ws.handle, C.byref(params), cap, _ptr(cell_keys, torch.int32, "cell_keys"),
                                      _ptr(kappa, torch.float64, "kappa"), _ptr(normal, torch.float64, "normal"),
                                      _ptr(coeffs, torch.float64, "coeffs") if coeffs is not None else None,
                                      _ptr(fit_status, torch.int8, "fit_status"), _stream(stream)),
           "front_curvature_ppic")


def front_csf_force(ws: Workspace, params: FtParams, alpha, kappa, normal, force, stream=None):
    if force.numel() != 3 * ws.grid.ncells:
        raise FrontError("force must hold 3*n0*n1*n2 values")
    _check(lib().front_csf_force(ws.handle, C.byref(params), _ptr(alpha, torch.float64, "alpha"),
                                 _ptr(kappa, torch.float64, "kappa"), _ptr(normal, torch.float64, "normal"),
                                 _ptr(force, torch.float64, "force"), _stream(stream)), "front_csf_force")


def front_force_clear(ws: Workspace, force, stream=None):
    """The dense force arrays set to zero (the first half of front_csf_force)."""
    if force.numel() != 3 * ws.grid.ncells:
        raise FrontError("force must hold 3*n0*n1*n2 values")
    _check(lib().front_force_clear(ws.handle, _ptr(force, torch.float64, "force"), _stream(stream)),
           "front_force_clear")


def front_csf_prepare(ws: Workspace, stream=None):
    """The ring cells of the current binning (one-front or batch workspace),
    listed ahead of front_csf_force_cells(_batch); needs only the binning."""
    _check(lib().front_csf_prepare(ws.handle, _stream(stream)), "front_csf_prepare")


def front_csf_force_cells(ws: Workspace, params: FtParams, alpha, kappa, normal, force, stream=None):
    """front_csf_force without the clear and the ring list (front_csf_prepare
    after the last binning): only the cells where the force can be non-zero are
    written (the rest of force must be zero already)."""
    if force.numel() != 3 * ws.grid.ncells:
        raise FrontError("force must hold 3*n0*n1*n2 values")
    _check(lib().front_csf_force_cells(ws.handle, C.byref(params), _ptr(alpha, torch.float64, "alpha"),
                                       _ptr(kappa, torch.float64, "kappa"), _ptr(normal, torch.float64, "normal"),
                                       _ptr(force, torch.float64, "force"), _stream(stream)), "front_csf_force_cells")


def front_csf_force_compact(ws: Workspace, params: FtParams, alpha, kappa, normal, keys, force, count, stream=None):
    """Compact CSF force: keys (int32/uint32 view, cap), force (cap, 3) float64,
    count (1) int64 on the device receives the number of slots."""
    cap = keys.numel()
    if force.numel() < 3 * cap or count.numel() < 1:
        raise FrontError("force must hold 3 values per key slot and count one int64")
    _check(lib().front_csf_force_compact(ws.handle, C.byref(params), _ptr(alpha, torch.float64, "alpha"),
                                         _ptr(kappa, torch.float64, "kappa"), _ptr(normal, torch.float64, "normal"),
                                         cap, _ptr(keys, torch.int32, "keys"), _ptr(force, torch.float64, "force"),
                                         _ptr(count, torch.int64, "count"), _stream(stream)), "front_csf_force_compact")


def front_alpha_pack(ws: Workspace, alpha, full_bits, alpha_cells, stream=None):
    """Compact alpha: full_bits (ceil(ncells/32) int32 words), alpha_cells (cap) float64."""
    if full_bits.numel() < (ws.grid.ncells + 31) // 32:
        raise FrontError("full_bits must hold ceil(n0*n1*n2/32) words")
    _check(lib().front_alpha_pack(ws.handle, _ptr(alpha, torch.float64, "alpha"), alpha_cells.numel(),
                                  _ptr(full_bits, torch.int32, "full_bits"),
                                  _ptr(alpha_cells, torch.float64, "alpha_cells"), _stream(stream)),
           "front_alpha_pack")


def front_face_force(ws: Workspace, params: FtParams, alpha, kappa, normal, fx, fy, fz, stream=None):
    """Balanced-force face term into the staggered arrays fx, fy, fz."""
    n = ws.grid.n
    for d, f in enumerate((fx, fy, fz)):
        shp = tuple(int(n[e]) + (1 if e == d else 0) for e in range(3))
        if tuple(f.shape) != shp:
            raise FrontError(f"face array {d} must have shape {shp}")
    _check(lib().front_face_force(ws.handle, C.byref(params), _ptr(alpha, torch.float64, "alpha"),
                                  _ptr(kappa, torch.float64, "kappa"), _ptr(normal, torch.float64, "normal"),
                                  _ptr(fx, torch.float64, "fx"), _ptr(fy, torch.float64, "fy"),
                                  _ptr(fz, torch.float64, "fz"), _stream(stream)), "front_face_force")


def front_face_force_batch(ws: "BatchWorkspace", params: FtParams, kappa, normal, stream=None):
    _check(lib().front_face_force_batch(ws.handle, C.byref(params), _ptr(kappa, torch.float64, "kappa"),
                                        _ptr(normal, torch.float64, "normal"), _stream(stream)),
           "front_face_force_batch")


FT_PARAB_MISS = 0x1


def front_paraboloid_cells(frame, coeffs, alpha, area=None, kappa=None, normal=None, status=None, stream=None):
    """alpha = V_P / V_C, surface area, surface-averaged curvature and normal
    of the paraboloids coeffs (m, 6) in the frames frame (m, 9) (cell units)."""
    m = frame.shape[0]
    if coeffs.shape[0] != m or alpha.shape[0] < m:
        raise FrontError("frame, coeffs and alpha must describe the same cells")
    _check(lib().front_paraboloid_cells(_ptr(frame, torch.float64, "frame"), _ptr(coeffs, torch.float64, "coeffs"), m,
                                        _ptr(alpha, torch.float64, "alpha"), _ptr(area, torch.float64, "area"),
                                        _ptr(kappa, torch.float64, "kappa"), _ptr(normal, torch.float64, "normal"),
                                        _ptr(status, torch.int8, "status"), _stream(stream)),
           "front_paraboloid_cells")


def front_ppic_frame(ws, frame, stream=None):
    """The (t1, t2, n) frame of every interfacial cell of the last PPIC fit."""
    _check(lib().front_ppic_frame(ws.handle, frame.shape[0], _ptr(frame, torch.float64, "frame"), _stream(stream)),
           "front_ppic_frame")


def front_volume_fraction_ppic(ws, coeffs, alpha, kappa=None, normal=None, area=None, status=None, stream=None):
    """alpha_P of the fitted paraboloids into alpha at the interfacial cells, and
    the surface-averaged kappa, normal and area per interfacial cell."""
    cap = coeffs.shape[0]
    _check(lib().front_volume_fraction_ppic(ws.handle, _ptr(coeffs, torch.float64, "coeffs"), cap,
                                            _ptr(alpha, torch.float64, "alpha"), _ptr(kappa, torch.float64, "kappa"),
                                            _ptr(normal, torch.float64, "normal"), _ptr(area, torch.float64, "area"),
                                            _ptr(status, torch.int8, "status"), _stream(stream)),
           "front_volume_fraction_ppic")


def front_volume_fraction_ppic_batch(ws, coeffs, kappa=None, normal=None, area=None, status=None, stream=None):
    cap = coeffs.shape[0]
    _check(lib().front_volume_fraction_ppic_batch(ws.handle, _ptr(coeffs, torch.float64, "coeffs"), cap,
                                                  _ptr(kappa, torch.float64, "kappa"),
                                                  _ptr(normal, torch.float64, "normal"),
                                                  _ptr(area, torch.float64, "area"), _ptr(status, torch.int8, "status"),
                                                  _stream(stream)),
           "front_volume_fraction_ppic_batch")


def front_interp_velocity(grid, U, V, W, verts, vel, stream=None):
    g = make_grid(grid)
    n = grid.n
    if tuple(U.shape) != (n[0] + 1, n[1], n[2]) or tuple(V.shape) != (n[0], n[1] + 1, n[2]) \
            or tuple(W.shape) != (n[0], n[1], n[2] + 1):
        raise FrontError("face arrays have the wrong shapes")
    _check(lib().front_interp_velocity(C.byref(g), _ptr_faces(U, "U"), _ptr_faces(V, "V"),
                                       _ptr_faces(W, "W"), _ptr(verts, torch.float64, "verts"),
                                       verts.shape[0], _ptr(vel, torch.float64, "vel"), _stream(stream)),
           "front_interp_velocity")


def front_advect_rk4(grid, U, V, W, verts, dt, verts_out, vel=None, stream=None):
    """One RK4 step of the points (verts_out may be verts; vel receives k1)."""
    g = make_grid(grid)
    n = grid.n
    if tuple(U.shape) != (n[0] + 1, n[1], n[2]) or tuple(V.shape) != (n[0], n[1] + 1, n[2]) \
            or tuple(W.shape) != (n[0], n[1], n[2] + 1):
        raise FrontError("face arrays have the wrong shapes")
    if verts_out.shape != verts.shape or (vel is not None and vel.shape != verts.shape):
        raise FrontError("verts_out and vel must have the shape of verts")
    _check(lib().front_advect_rk4(C.byref(g), _ptr(U, torch.float64, "U"), _ptr(V, torch.float64, "V"),
                                  _ptr(W, torch.float64, "W"), _ptr(verts, torch.float64, "verts"), verts.shape[0],
                                  float(dt), _ptr(verts_out, torch.float64, "verts_out"),
                                  _ptr(vel, torch.float64, "vel") if vel is not None else None, _stream(stream)),
           "front_advect_rk4")


def front_advect_rk4_batch(ws: "BatchWorkspace", stream=None):
    """RK4 step of every front of the table with its own dt."""
    _check(lib().front_advect_rk4_batch(ws.handle, _stream(stream)), "front_advect_rk4_batch")


def ft_volume_fraction_noalloc(grid, verts, tris, params: FtParams, alpha, status, stream=None):
    """Binning + volume fraction with the library's static scratch (no device
    allocation); status is a 1-element int32 CUDA tensor receiving FT_ST_* bits."""
    if alpha.numel() != grid.ncells or status.numel() < 1:
        raise FrontError("alpha must hold n0*n1*n2 values and status one word")
    g = make_grid(grid)
    f = FtFront(_ptr(verts, torch.float64, "verts"), verts.shape[0], _ptr(tris, torch.int32, "tris"), tris.shape[0])
    _check(lib().ft_volume_fraction_noalloc(C.byref(g), C.byref(f), C.byref(params),
                                            _ptr(alpha, torch.float64, "alpha"), _ptr(status, torch.int32, "status"),
                                            _stream(stream)), "ft_volume_fraction_noalloc")


def front_bin_batch(ws: BatchWorkspace, params: FtParams, stream=None):
    _check(lib().front_bin_batch(ws.handle, C.byref(params), _stream(stream)), "front_bin_batch")


def front_volume_fraction_batch(ws: BatchWorkspace, stream=None):
    _check(lib().front_volume_fraction_batch(ws.handle, _stream(stream)), "front_volume_fraction_batch")


def front_csf_force_batch(ws: BatchWorkspace, params: FtParams, kappa, normal, stream=None):
    _check(lib().front_csf_force_batch(ws.handle, C.byref(params), _ptr(kappa, torch.float64, "kappa"),
                                       _ptr(normal, torch.float64, "normal"), _stream(stream)),
           "front_csf_force_batch")


def front_force_clear_batch(ws: BatchWorkspace, stream=None):
    _check(lib().front_force_clear_batch(ws.handle, _stream(stream)), "front_force_clear_batch")


def front_csf_force_cells_batch(ws: BatchWorkspace, params: FtParams, kappa, normal, stream=None):
    _check(lib().front_csf_force_cells_batch(ws.handle, C.byref(params), _ptr(kappa, torch.float64, "kappa"),
                                             _ptr(normal, torch.float64, "normal"), _stream(stream)),
           "front_csf_force_cells_batch")


def front_interp_velocity_batch(ws: BatchWorkspace, stream=None):
    _check(lib().front_interp_velocity_batch(ws.handle, _stream(stream)), "front_interp_velocity_batch")


def ft_batch_cell_ranges(ws: BatchWorkspace, off: torch.Tensor, stream=None):
    if off.numel() < ws.nf + 1:
        raise FrontError("off must hold nf + 1 values")
    _check(lib().ft_batch_cell_ranges(ws.handle, _ptr(off, torch.int64, "off"), _stream(stream)),
           "ft_batch_cell_ranges")


def ft_set_tuning(ws: Workspace, clip=4, ppic=4, csf=16, fill=8, ppic_min_blocks=4, ppic_dynamic=0, sort_blocks=0):
    t = FtTuning(int(clip), int(ppic), int(csf), int(fill), int(ppic_min_blocks), int(ppic_dynamic),
                 int(sort_blocks), 0, 0, 0, 0, 0.0)
    _check(lib().ft_set_tuning(ws.handle, C.byref(t)), "ft_set_tuning")


def ft_get_tuning(ws: Workspace) -> dict:
    t = FtTuning()
    _check(lib().ft_get_tuning(ws.handle, C.byref(t)), "ft_get_tuning")
    return t.as_dict()


def ft_autotune(ws: Workspace, params: FtParams, reps: int = 5, verts=None, tris=None, stream=None) -> dict:
    """Times launch shapes on the workspace's workload and installs the fastest
    (verts/tris for a one-front workspace; None for a batch workspace)."""
    t = FtTuning()
    if verts is not None:
        f = FtFront(_ptr(verts, torch.float64, "verts"), verts.shape[0], _ptr(tris, torch.int32, "tris"),
                    tris.shape[0])
        fp = C.byref(f)
    else:
        fp = None
    _check(lib().ft_autotune(ws.handle, fp, C.byref(params), int(reps), C.byref(t), _stream(stream)), "ft_autotune")
    return t.as_dict()


class Roughness:
    """Roughness workspace (ft_rough_create): metrics and smoothing of a front."""

    def __init__(self, max_nv: int, max_nt: int, device: int = 0):
        h = C.c_void_p()
        nbytes = C.c_size_t()
        _check(lib().ft_rough_create(C.byref(h), int(max_nv), int(max_nt), int(device), C.byref(nbytes)),
               "ft_rough_create")
        self.handle = h
        self.bytes = int(nbytes.value)

    def close(self):
        if self.handle:
            lib().ft_rough_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def status(self, stream=None) -> int:
        bits = C.c_uint32()
        _check(lib().ft_rough_status(self.handle, _stream(stream), C.byref(bits)), "ft_rough_status")
        return int(bits.value)

    def metrics(self, verts, tris, stream=None) -> dict:
        nv, nt = verts.shape[0], tris.shape[0]
        dev = verts.device
        out = dict(gl=torch.empty((nv, 3), dtype=torch.float64, device=dev),
                   rough=torch.empty(nv, dtype=torch.float64, device=dev),
                   r1=torch.empty(nv, dtype=torch.float64, device=dev),
                   r2=torch.empty(nv, dtype=torch.float64, device=dev),
                   rt=torch.empty(nt, dtype=torch.float64, device=dev),
                   G=torch.empty(nv, dtype=torch.float64, device=dev),
                   V=torch.empty(nv, dtype=torch.float64, device=dev))
        _check(lib().front_roughness(self.handle, _ptr(verts, torch.float64, "verts"), nv,
                                     _ptr(tris, torch.int32, "tris"), nt, *(C.c_void_p(out[k].data_ptr()) for k in
                                                                             ("gl", "rough", "r1", "r2", "rt", "G",
                                                                              "V")), _stream(stream)),
               "front_roughness")
        return out

    def smooth(self, verts, tris, gl_thr, r_thr, max_rounds=64, stream=None) -> dict:
        """In place on verts; returns rounds, moved, status."""
        rounds, moved, st = C.c_int32(), C.c_int64(), C.c_uint32()
        _check(lib().front_roughness_smooth(self.handle, _ptr(verts, torch.float64, "verts"), verts.shape[0],
                                            _ptr(tris, torch.int32, "tris"), tris.shape[0], float(gl_thr),
                                            float(r_thr), int(max_rounds), C.byref(rounds), C.byref(moved),
                                            C.byref(st), _stream(stream)), "front_roughness_smooth")
        return dict(rounds=int(rounds.value), moved=int(moved.value), status=int(st.value))


def launch_count() -> int:
    return int(lib().ft_launch_count())


TRACE_NAME = 48  # FT_TRACE_NAME


def trace_start(capacity: int = 65536):
    """Open a per-kernel trace: event pairs around the library's launches
    (eager launches only; see ft_trace_start)."""
    _check(lib().ft_trace_start(int(capacity)), "ft_trace_start")


def trace_stop(max_kernels: int = 64) -> dict:
    """Close the trace; returns {kernel name: (launches, summed device ms)}
    in order of first launch, plus the count of launches not traced under the
    key None."""
    names = C.create_string_buffer(max_kernels * TRACE_NAME)
    launches = (C.c_int64 * max_kernels)()
    ms = (C.c_double * max_kernels)()
    nk = C.c_int32(0)
    dropped = C.c_int64(0)
    _check(lib().ft_trace_stop(max_kernels, C.cast(names, C.c_void_p), C.cast(launches, C.c_void_p),
                               C.cast(ms, C.c_void_p), C.byref(nk), C.byref(dropped)), "ft_trace_stop")
    out = {}
    raw = names.raw
    for k in range(nk.value):
        nm = raw[k * TRACE_NAME:(k + 1) * TRACE_NAME].split(b"\0", 1)[0].decode()
        out[nm] = (int(launches[k]), float(ms[k]))
    out[None] = int(dropped.value)
    return out


def probe_fma_rate(kind: int, device: int = 0) -> float:
    out = C.c_double()
    _check(lib().ft_probe_fma_rate(int(kind), int(device), C.byref(out)), "ft_probe_fma_rate")
    return float(out.value)


# ---------------------------------------------------------------------------
# convenience: device buffers for one front and the whole hot path
# ---------------------------------------------------------------------------

class FrontCoupling:
    """Holds a workspace and device output buffers for fronts on one grid and
    runs the five steps in order (bin, alpha, kappa, force, vertex velocity)."""

    def __init__(self, grid, max_nt: int, max_nv: int, max_cand: int = 0, params: FtParams | None = None,
                 device: int = 0):
        self.grid = grid
        self.params = params or make_params()
        self.ws = Workspace(grid, max_nt, max_cand=max_cand, device=device)
        dev = torch.device("cuda", device)
        nc = grid.ncells
        cap = max_cand if max_cand else 16 * max_nt + 1024
        self.cap_cells = cap
        self.alpha = torch.empty(nc, dtype=torch.float64, device=dev)
        self.force = torch.empty(3 * nc, dtype=torch.float64, device=dev)
        self.cell_keys = torch.empty(cap, dtype=torch.int32, device=dev)
        self.kappa = torch.empty(cap, dtype=torch.float64, device=dev)
        self.normal = torch.empty((cap, 3), dtype=torch.float64, device=dev)
        self.coeffs = torch.empty((cap, 6), dtype=torch.float64, device=dev)
        self.fit_status = torch.empty(cap, dtype=torch.int8, device=dev)
        self.vel = torch.empty((max_nv, 3), dtype=torch.float64, device=dev)

    def step(self, verts, tris, faces, stream=None):
        p = self.params
        front_bin(self.ws, verts, tris, p, stream)
        front_volume_fraction(self.ws, self.alpha, stream)
        front_curvature_ppic(self.ws, p, self.cell_keys, self.kappa, self.normal, self.coeffs, self.fit_status, stream)
        front_csf_force(self.ws, p, self.alpha, self.kappa, self.normal, self.force, stream)
        front_interp_velocity(self.grid, faces[0], faces[1], faces[2], verts, self.vel[:verts.shape[0]], stream)

    def results(self, nv: int):
        """Synchronizes and returns host copies (numpy) of every output."""
        c = self.ws.counts()
        M = c["M"]
        n = tuple(int(x) for x in self.grid.n)
        return dict(
            counts=c,
            status=self.ws.status(),
            alpha=self.alpha.view(n).cpu().numpy(),
            cell_keys=self.cell_keys[:M].cpu().numpy().view("uint32"),
            kappa=self.kappa[:M].cpu().numpy(),
            normal=self.normal[:M].cpu().numpy(),
            coeffs=self.coeffs[:M].cpu().numpy(),
            fit_status=self.fit_status[:M].cpu().numpy(),
            force=self.force.view((3,) + n).cpu().numpy(),
            vel=self.vel[:nv].cpu().numpy(),
        )


class BatchCoupling:
    """A batch workspace, per-front device outputs (alpha, force, vel) and the
    batch-wide PPIC outputs; runs the five steps over every front at once."""

    def __init__(self, fronts, params: FtParams | None = None, max_cand: int = 0, max_cells: int = 0,
                 device: int = 0, headroom: float = 1.0):
        """fronts: list of dicts with grid, verts, tris and optional U, V, W.
        max_cand = 0 sizes the candidate buffers exactly: a first binning on a
        small workspace reports the pairs needed (ft_counts), times headroom."""
        self.params = params or make_params()
        dev = torch.device("cuda", device)
        cells = sum(int(f["grid"].ncells) for f in fronts)
        nt = sum(int(f["tris"].shape[0]) for f in fronts)
        if not max_cand:
            # per-triangle counts are exact up to the probe's capacity
            probe = BatchWorkspace(len(fronts), cells, max(nt, 1), max_cand=1 << 20, max_cells=1024, device=device)
            probe.set_fronts([dict(grid=f["grid"], verts=f["verts"], tris=f["tris"]) for f in fronts])
            front_bin_batch(probe, self.params)
            max_cand = int(probe.counts()["C_need"] * headroom) + 1024
            probe.status()
            probe.front_status()
            probe.close()
        self.ws = BatchWorkspace(len(fronts), int(cells * headroom) + 1, int(nt * headroom) + 1,
                                 max_cand=max_cand, max_cells=max_cells, device=device)
        cap = max_cand if max_cand else 16 * (int(nt * headroom) + 1) + 1024
        self.cap_cells = max_cells if max_cells else cap
        self.fronts = []
        for f in fronts:
            g = f["grid"]
            d = dict(f)
            d.setdefault("alpha", torch.empty(g.ncells, dtype=torch.float64, device=dev))
            d.setdefault("force", torch.empty(3 * g.ncells, dtype=torch.float64, device=dev))
            if "U" in f:
                d.setdefault("vel", torch.empty((f["verts"].shape[0], 3), dtype=torch.float64, device=dev))
            self.fronts.append(d)
        self.ws.set_fronts(self.fronts)
        M = self.cap_cells
        self.cell_keys = torch.empty(M, dtype=torch.int32, device=dev)
        self.kappa = torch.empty(M, dtype=torch.float64, device=dev)
        self.normal = torch.empty((M, 3), dtype=torch.float64, device=dev)
        self.coeffs = torch.empty((M, 6), dtype=torch.float64, device=dev)
        self.fit_status = torch.empty(M, dtype=torch.int8, device=dev)
        self.off = torch.empty(len(fronts) + 1, dtype=torch.int64, device=dev)

    def step(self, stream=None, interp: bool = True):
        p, ws = self.params, self.ws
        front_bin_batch(ws, p, stream)
        front_volume_fraction_batch(ws, stream)
        front_curvature_ppic(ws, p, self.cell_keys, self.kappa, self.normal, self.coeffs, self.fit_status, stream)
        front_csf_force_batch(ws, p, self.kappa, self.normal, stream)
        ft_batch_cell_ranges(ws, self.off, stream)
        if interp and all("U" in f for f in self.fronts):
            front_interp_velocity_batch(ws, stream)

    def results(self, b: int):
        """Synchronizes and returns host copies (numpy) of front b's outputs,
        with its cell keys made front-local."""
        off = self.off.cpu().numpy()
        lo, hi = int(off[b]), int(off[b + 1])
        f = self.fronts[b]
        n = tuple(int(x) for x in f["grid"].n)
        kb = sum(int(x["grid"].ncells) for x in self.fronts[:b])
        out = dict(
            alpha=f["alpha"].view(n).cpu().numpy(),
            cell_keys=(self.cell_keys[lo:hi].cpu().numpy().view("uint32").astype("int64") - kb).astype("uint32"),
            kappa=self.kappa[lo:hi].cpu().numpy(),
            normal=self.normal[lo:hi].cpu().numpy(),
            coeffs=self.coeffs[lo:hi].cpu().numpy(),
            fit_status=self.fit_status[lo:hi].cpu().numpy(),
            force=f["force"].view((3,) + n).cpu().numpy(),
        )
        if "vel" in f:
            out["vel"] = f["vel"].cpu().numpy()
        return out
