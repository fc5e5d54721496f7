"""CUDA path (through the C ABI) against the FP64 oracle, element by element.

Bins, the interfacial-cell set and the parity fill must match bit for bit;
floats within: |d alpha| <= 1e-12, |d kappa| <= 1e-9 max(|kappa|, 1),
|d normal| <= 1e-9, |d S| <= 1e-9 max|S|, |d u| <= 1e-12 max|U|.
"""
import numpy as np
import pytest

from paper_2505_06932_gb300 import inputs as I
from gpucase import run_gpu, run_oracle

pytestmark = pytest.mark.gpu

TOL_ALPHA = 1e-12
TOL_KAPPA = 1e-9
TOL_NORMAL = 1e-9
TOL_FORCE = 1e-9
TOL_VEL = 1e-12


def _rotation(seed):
    q, _ = np.linalg.qr(I.rng(seed).normal(size=(3, 3)))
    if np.linalg.det(q) < 0:
        q[:, 0] *= -1
    return q


def _box(rotate):
    g = I.unit_grid(48)
    L = 20 * g.h
    v, t = I.box_front((0.5 - L / 2,) * 3, (0.5 + L / 2,) * 3, 40)
    if rotate:
        v = (v - 0.5) @ _rotation(5).T + 0.5
    gen = I.rng(17)
    faces, _ = I.solid_body_faces(g, np.array([0.5, 0.5, 0.5]), gen)
    return dict(grid=g, verts=np.ascontiguousarray(v), tris=t, faces=faces)


def _general_grid():
    g = I.Grid((40, 36, 44), (-0.3, 0.2, 0.05), 1.0 / 37)
    gen = I.rng(31)
    c = np.array([-0.3 + 20 / 37, 0.2 + 18 / 37, 0.05 + 22 / 37]) + gen.uniform(0, 1 / 37, 3)
    v, t = I.sh_deformed_front(4, 8.0 / 37, c, gen)
    faces, _ = I.solid_body_faces(g, c, gen)
    return dict(grid=g, verts=v, tris=t, faces=faces)


def _far_origin():
    """A grid far from the coordinate origin: |coordinate| / h ~ 6e7, beyond the
    float32 clip's grid bound (2^24), so the FP32 form clips in binary64 there."""
    h = 1.0 / 32
    g = I.Grid((40, 40, 40), (1.0e6, -2.0e6, 3.0e5), h)
    gen = I.rng(41)
    c = np.array(g.origin) + 20 * h + gen.uniform(0, h, 3)
    v, t = I.sh_deformed_front(4, 10 * h, c, gen)
    faces, _ = I.solid_body_faces(g, c, gen)
    return dict(grid=g, verts=v, tris=t, faces=faces)


CASES = {
    "droplet_32": lambda: I.laplace_droplet_32(1),
    "sphere_36_ragged": lambda: I.small_sphere(3, 0.3, 36, seed=4, noise_h=1e-3),
    "sh_droplet_40": lambda: I.sh_droplet_256(seed=9, s=4, N=40),
    "bubble_40": lambda: I.sh_droplet_256(seed=10, bubble=True, s=4, N=40),
    "box_in_grid_planes": lambda: _box(False),
    "box_rotated": lambda: _box(True),
    "general_grid": _general_grid,
}


def _dump(path, gpu, orc):
    """Both sides' arrays of a failing case, into pytest's temporary folder."""
    arrs = {}
    for tag, r in (("gpu", gpu), ("orc", orc)):
        for k, v in r.items():
            if isinstance(v, np.ndarray):
                arrs[f"{tag}_{k}"] = v
    np.savez_compressed(str(path), **arrs)


FP64_TOL = dict(alpha=TOL_ALPHA, kappa=TOL_KAPPA, normal=TOL_NORMAL, coeffs=1e-9, force=TOL_FORCE)
# the FP32-compensated form against the FP64 oracle (stated errors 1e-6 on alpha, 1e-4 on kappa)
FP32_TOL = dict(alpha=1e-6, kappa=1e-4, normal=1e-4, coeffs=1e-3, force=1e-4)


def compare(gpu, orc, full=True, dump=None, tol=FP64_TOL):
    try:
        _compare(gpu, orc, full, tol)
    except AssertionError:
        if dump is not None:
            _dump(dump, gpu, orc)
        raise


def _compare(gpu, orc, full=True, tol=FP64_TOL):
    assert gpu["status"] == 0, gpu["status"]
    assert orc["status"] == 0
    # bins: bit-exact pairs and interfacial set
    assert np.array_equal(gpu["pair_keys"], orc["pair_keys"])
    assert np.array_equal(gpu["pair_tris"], orc["pair_tris"])
    assert np.array_equal(gpu["cell_keys"], orc["cells"])
    # alpha: parity fill bit-exact, cut cells within 1e-12
    ga, oa = gpu["alpha"], orc["alpha"]
    inter = np.zeros(ga.size, bool)
    inter[orc["cells"]] = True
    assert np.array_equal(ga.reshape(-1)[~inter], oa.reshape(-1)[~inter])
    assert np.max(np.abs(ga - oa)) <= tol["alpha"]
    if not full:
        return
    # kappa, normal, coefficients, fit status
    k, ko = gpu["kappa"], orc["kappa"]
    assert np.all(np.abs(k - ko) <= tol["kappa"] * np.maximum(np.abs(ko), 1.0))
    assert np.max(np.abs(gpu["normal"] - orc["normal"])) <= tol["normal"]
    assert np.all(np.abs(gpu["coeffs"] - orc["coeffs"]) <= tol["coeffs"] * np.maximum(np.abs(orc["coeffs"]), 1.0))
    assert np.array_equal(gpu["fit_status"], orc["fit_status"])
    # CSF force
    fo = orc["force"]
    assert np.max(np.abs(gpu["force"] - fo)) <= tol["force"] * max(np.abs(fo).max(), 1e-300)
    # vertex velocities
    if "vel" in orc:
        umax = max(np.abs(f).max() for f in orc_faces(orc))
        assert np.max(np.abs(gpu["vel"] - orc["vel"])) <= tol.get("vel", TOL_VEL) * umax


def orc_faces(orc):
    return orc["_faces"]


@pytest.mark.parametrize("name", list(CASES))
def test_parity_small_cases(name, tmp_path):
    w = CASES[name]()
    gpu = run_gpu(w)
    orc = run_oracle(w)
    orc["_faces"] = w["faces"]
    compare(gpu, orc, dump=tmp_path / f"fail_{name}.npz")


@pytest.mark.parametrize("make", [I.rough_sphere_128, I.ellipsoid_128], ids=["rough_sphere_128", "ellipsoid_128"])
def test_parity_128(make):
    """The 128^3 workloads (81,920 triangles) in full."""
    w = make()
    gpu = run_gpu(w)
    orc = run_oracle(w)
    orc["_faces"] = w["faces"]
    compare(gpu, orc)


_ORACLE_256 = {}


def _oracle_256(bubble):
    """The oracle's five steps on the 256^3 SH droplet or dimpled bubble (every
    interfacial cell fitted), computed once per module."""
    if bubble not in _ORACLE_256:
        w = I.sh_droplet_256(seed=4, bubble=bubble)
        orc = run_oracle(w)
        orc["_faces"] = w["faces"]
        _ORACLE_256[bubble] = (w, orc)
    return _ORACLE_256[bubble]


@pytest.mark.parametrize("precision", ["fp64", "fp32c"])
@pytest.mark.parametrize("bubble", [False, True], ids=["sh_droplet_256", "bubble_256"])
def test_parity_256(bubble, precision, tmp_path):
    """The 256^3 workloads (327,680 triangles; the oscillating-droplet and
    rising-bubble shapes) in full, in both forms: pairs, interfacial cells and
    parity fill bit for bit; alpha, kappa, normal, coefficients and fit status of
    every interfacial cell, the CSF force in every cell and the velocity at every
    vertex within the form's stated tolerance."""
    from paper_2505_06932_gb300 import _front as F
    w, orc = _oracle_256(bubble)
    prec = F.FT_FP64 if precision == "fp64" else F.FT_FP32C
    gpu = run_gpu(w, precision=prec)
    assert len(orc["cells"]) > 40000
    compare(gpu, orc, dump=tmp_path / "fail_256.npz", tol=FP64_TOL if precision == "fp64" else FP32_TOL)


def test_support_growth_parity():
    """Coarse front with fit_min above the fragment count: delta grows."""
    w = I.small_sphere(1, 0.25, 32, seed=2)
    p = dict(fit_min=60)
    gpu = run_gpu(w, params=p, max_cand=200000)
    orc = run_oracle(w, params=p)
    orc["_faces"] = w["faces"]
    assert np.mean((gpu["fit_status"] & 1) != 0) > 0.5
    compare(gpu, orc)


@pytest.mark.parametrize("name", ["droplet_32", "sh_droplet_40", "bubble_40", "box_in_grid_planes", "box_rotated",
                                  "general_grid"])
def test_fp32c_small_cases(name, tmp_path):
    """FP32-compensated form: identical bins and parity fill, |d alpha| <= 1e-6,
    |d kappa| <= 1e-4 max(|kappa|, 1) against the FP64 oracle."""
    from paper_2505_06932_gb300 import _front as F
    w = CASES[name]()
    gpu = run_gpu(w, precision=F.FT_FP32C)
    orc = run_oracle(w)
    orc["_faces"] = w["faces"]
    compare(gpu, orc, dump=tmp_path / f"fail_fp32c_{name}.npz", tol=FP32_TOL)


@pytest.mark.parametrize("make", [I.rough_sphere_128, I.ellipsoid_128], ids=["rough_sphere_128", "ellipsoid_128"])
def test_fp32c_128(make):
    from paper_2505_06932_gb300 import _front as F
    w = make()
    gpu = run_gpu(w, precision=F.FT_FP32C)
    orc = run_oracle(w)
    orc["_faces"] = w["faces"]
    compare(gpu, orc, tol=FP32_TOL)


@pytest.mark.parametrize("precision", ["fp64", "fp32c"])
def test_far_origin_grid(precision, tmp_path):
    """A grid whose coordinates are 6.4e7 cells from the origin (beyond the
    float32 clip's bound, so the FP32 form clips in binary64 there): bins,
    interfacial set and parity fill still bit for bit; the floats within their
    tolerances widened by the rounding of the coordinates themselves (binary64
    coordinates carry eps |x| / h = 7e-9 cells there; the oracle and the CUDA
    path round them in different places), 200 eps |x| / h."""
    from paper_2505_06932_gb300 import _front as F
    w = _far_origin()
    g = w["grid"]
    ext = max(abs(o) + n * g.h for o, n in zip(g.origin, g.n)) / g.h
    floor = 200 * np.finfo(float).eps * ext
    base = FP64_TOL if precision == "fp64" else FP32_TOL
    tol = {k: max(v, floor) for k, v in base.items()}
    tol["vel"] = max(TOL_VEL, floor)
    gpu = run_gpu(w, precision=F.FT_FP64 if precision == "fp64" else F.FT_FP32C)
    orc = run_oracle(w)
    orc["_faces"] = w["faces"]
    compare(gpu, orc, dump=tmp_path / f"fail_far_origin_{precision}.npz", tol=tol)


# ---------------------------------------------------------------------------
# edge cases
# ---------------------------------------------------------------------------

def test_empty_front():
    g = I.unit_grid(16)
    w = dict(grid=g, verts=np.zeros((0, 3)), tris=np.zeros((0, 3), np.int32))
    gpu = run_gpu(w)
    assert gpu["status"] == 0
    assert gpu["counts"]["M"] == 0 and gpu["counts"]["P"] == 0
    assert np.all(gpu["alpha"] == 0.0) and np.all(gpu["force"] == 0.0)


def test_outside_grid_flagged():
    w = I.laplace_droplet_32(1)
    w["verts"] = w["verts"] + np.array([0.3, 0.0, 0.0])
    gpu = run_gpu(w)
    assert gpu["status"] & 0x02


def test_open_front_flagged():
    w = I.laplace_droplet_32(2)
    w["tris"] = np.ascontiguousarray(np.delete(w["tris"], 17, axis=0))
    gpu = run_gpu(w)
    assert gpu["status"] & 0x04


def test_inverted_front_flagged():
    w = I.laplace_droplet_32(2)
    w["tris"] = np.ascontiguousarray(w["tris"][:, ::-1])
    gpu = run_gpu(w)
    assert gpu["status"] & 0x08


def test_bad_vertex_index_flagged():
    w = I.laplace_droplet_32(2)
    t = w["tris"].copy()
    t[5, 1] = len(w["verts"]) + 7
    w["tris"] = t
    gpu = run_gpu(w)
    assert gpu["status"] & 0x10


def test_capacity_overflow_flagged_not_faulting():
    w = I.laplace_droplet_32(3)
    gpu = run_gpu(w, max_cand=1000)
    assert gpu["status"] & 0x01
    assert gpu["counts"]["C_need"] > 1000 and gpu["counts"]["M"] == 0
