"""Pins of the oracle's volume fraction alpha_C = (1/V_C) int_C I dx (Sec. 3.2)."""
import math

import numpy as np
import pytest

import oracle
from paper_2505_06932_gb300 import inputs as I
import geomref


@pytest.mark.parametrize("make", [
    lambda: I.laplace_droplet_32(1),
    lambda: I.small_sphere(3, 0.3, 36, seed=4, noise_h=1e-3),
    lambda: I.sh_droplet_256(seed=9, s=4, N=40),
    lambda: I.sh_droplet_256(seed=10, bubble=True, s=4, N=40),
])
def test_total_volume_equals_mesh_volume(make):
    """sum alpha h^3 = (1/6) sum_t x_a . (x_b x x_c) to 1e-12 relative; alpha in [0,1]."""
    w = make()
    g = w["grid"]
    a, st = oracle.alpha(w["verts"], w["tris"], g)
    assert st == 0
    vol = I.signed_volume(w["verts"], w["tris"])
    assert abs(a.sum() * g.h ** 3 - vol) <= 1e-12 * abs(vol)
    assert a.min() >= 0.0 and a.max() <= 1.0


def _plane_cut_front(cell_lo, h, nvec, d):
    lo = np.asarray(cell_lo) - 2 * h
    hi = np.asarray(cell_lo) + 3 * h
    planes = [(np.array([1.0, 0, 0]), hi[0]), (np.array([-1.0, 0, 0]), -lo[0]),
              (np.array([0, 1.0, 0]), hi[1]), (np.array([0, -1.0, 0]), -lo[1]),
              (np.array([0, 0, 1.0]), hi[2]), (np.array([0, 0, -1.0]), -lo[2]),
              (np.asarray(nvec, dtype=np.float64), d)]
    return geomref.convex_polyhedron_mesh(planes)


@pytest.mark.parametrize("seed", range(6))
def test_plane_cut_of_one_cube(seed):
    """A closed convex front whose only face through cell C is the plane n.x = d:
    alpha_C equals the corner-simplex volume of the plane-cut cube."""
    gen = I.rng(100 + seed)
    g = I.unit_grid(24)
    h = g.h
    ijk = np.array([11, 11, 11])
    cell_lo = ijk * h
    nvec = gen.uniform(0.2, 1.0, size=3)
    nvec /= np.linalg.norm(nvec)
    frac = gen.uniform(0.05, 0.95)
    dloc = frac * nvec.sum()              # plane offset in cell-local units of h
    d = float(nvec @ cell_lo) + dloc * h
    v, t = _plane_cut_front(cell_lo, h, nvec, d)
    a, st = oracle.alpha(v, t, g, margin=3)
    assert st == 0
    want = geomref.plane_cut_unit_cube(nvec, dloc)
    assert abs(a[tuple(ijk)] - want) < 1e-13


def test_integer_cell_translation():
    w = I.small_sphere(3, 0.2, 32, seed=7)
    g = w["grid"]
    a0, st0 = oracle.alpha(w["verts"], w["tris"], g)
    shift = np.array([2, -1, 1])
    a1, st1 = oracle.alpha(w["verts"] + shift * g.h, w["tris"], g)
    assert st0 == 0 and st1 == 0
    b = np.roll(a0, tuple(shift), axis=(0, 1, 2))
    assert np.max(np.abs(a1 - b)) < 1e-13


def test_convex_clip_agreement():
    """For a convex front, alpha_C = vol(cube cut by every face plane)/h^3."""
    w = I.small_sphere(2, 0.3, 14, seed=3)
    g, v, t = w["grid"], w["verts"], w["tris"]
    a, _ = oracle.alpha(v, t, g)
    cells, _ = oracle.interfacial_cells(v, t, g)
    n, d = geomref.face_planes(v, t)
    planes = list(zip(n, d))
    h = g.h
    for key in cells[::3]:
        i, j, k = key // (g.n[1] * g.n[2]), (key // g.n[2]) % g.n[1], key % g.n[2]
        lo = np.array([i, j, k]) * h
        want = geomref.convex_cell_fraction(lo, h, planes)
        assert abs(a[i, j, k] - want) < 1e-12, (i, j, k)


def test_parity_fill_matches_winding_number():
    """Cells without front: alpha is exactly the winding number (0 or 1) at the centre."""
    w = I.sh_droplet_256(seed=12, s=3, N=32)
    g, v, t = w["grid"], w["verts"], w["tris"]
    a, st = oracle.alpha(v, t, g)
    assert st == 0
    cells, _ = oracle.interfacial_cells(v, t, g)
    empty = np.ones(g.ncells, bool)
    empty[cells] = False
    idx = np.nonzero(empty)[0]
    ii, jj, kk = idx // (g.n[1] * g.n[2]), (idx // g.n[2]) % g.n[1], idx % g.n[2]
    pts = (np.stack([ii, jj, kk], 1) + 0.5) * g.h
    wn = geomref.winding_numbers(v, t, pts)
    assert np.max(np.abs(wn - np.round(wn))) < 1e-6
    assert np.array_equal(a.reshape(-1)[idx], np.round(wn))


def test_open_and_inverted_fronts_flagged():
    w = I.laplace_droplet_32(2)
    g, v, t = w["grid"], w["verts"], w["tris"]
    _, st = oracle.alpha(v, np.delete(t, 17, axis=0), g)
    assert st & 2  # not closed
    _, st = oracle.alpha(v, t[:, ::-1].copy(), g)
    assert st & 4  # orientation
