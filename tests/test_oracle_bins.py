"""Pins of the oracle's binning (interfacial cells, Sec. 3.2) against brute force,
an independent separating-axis overlap test and area-partition identities."""
import numpy as np
import pytest

import oracle
from paper_2505_06932_gb300 import inputs as I
import geomref


def _decode(key, g):
    n1, n2 = g.n[1], g.n[2]
    return key // (n1 * n2), (key // n2) % n1, key % n2


def _tri_area_vec(v, t):
    a, b, c = v[t[:, 0]], v[t[:, 1]], v[t[:, 2]]
    return 0.5 * np.cross(b - a, c - a)


def _poly_area_vec(p):
    p0 = p[0]
    s = np.zeros(3)
    for a, b in zip(p[1:-1], p[2:]):
        s += np.cross(a - p0, b - p0)
    return 0.5 * s


def test_candidate_restriction_matches_bruteforce():
    """Binning only tests cells whose box meets the triangle's bounding box;
    evaluating the predicate on every cell of the grid gives the same pairs."""
    w = I.small_sphere(1, 0.3, 10, seed=5)
    k1, t1, st = oracle.bin_pairs(w["verts"], w["tris"], w["grid"], margin=0)
    k2, t2 = oracle.bin_pairs_bruteforce(w["verts"], w["tris"], w["grid"])
    assert st == 0
    assert np.array_equal(k1, k2) and np.array_equal(t1, t2)


def test_bins_match_separating_axis_overlap():
    """A pair is binned iff the triangle and the cell overlap with positive area
    (generic input: no contact is within 1e-9 h of degenerate)."""
    w = I.small_sphere(2, 0.27, 12, seed=11)
    g, v, t = w["grid"], w["verts"], w["tris"]
    keys, tids, st = oracle.bin_pairs(v, t, g, margin=0)
    got = set(zip(keys.tolist(), tids.tolist()))
    want = set()
    h = g.h
    for ti, tri in enumerate(t):
        p = v[tri]
        lo = np.floor(p.min(0) / h).astype(int) - 1
        hi = np.floor(p.max(0) / h).astype(int) + 1
        for i in range(lo[0], hi[0] + 1):
            for j in range(lo[1], hi[1] + 1):
                for k in range(lo[2], hi[2] + 1):
                    clo = np.array([i, j, k]) * h
                    if geomref.tri_box_overlap(p, clo, clo + h, eps=-1e-9 * h):
                        want.add(((i * g.n[1] + j) * g.n[2] + k, ti))
    assert got == want


def test_fragments_partition_each_triangle():
    """Sum of fragment areas of a triangle = its area; fragment area vectors of a
    closed front sum to zero."""
    w = I.laplace_droplet_32(1)
    g, v, t = w["grid"], w["verts"], w["tris"]
    keys, tids, _ = oracle.bin_pairs(v, t, g)
    area = np.zeros(len(t))
    total = np.zeros(3)
    for key, ti in zip(keys, tids):
        i, j, k = _decode(int(key), g)
        poly = oracle.clip_fragment(v[t[ti]], g, i, j, k)
        assert poly is not None
        av = _poly_area_vec(poly)
        area[ti] += np.linalg.norm(av)
        total += av
    ref = np.linalg.norm(_tri_area_vec(v, t), axis=1)
    assert np.max(np.abs(area - ref) / ref) < 1e-12
    assert np.linalg.norm(total) < 1e-13 * ref.sum()


def test_bins_contain_vertex_cells():
    w = I.laplace_droplet_32(3)
    g, v, t = w["grid"], w["verts"], w["tris"]
    keys, tids, _ = oracle.bin_pairs(v, t, g)
    cells = set(keys.tolist())
    ijk = np.floor(v / g.h).astype(np.int64)
    vk = (ijk[:, 0] * g.n[1] + ijk[:, 1]) * g.n[2] + ijk[:, 2]
    assert set(vk.tolist()) <= cells


def test_in_face_fragments_owned_once():
    """A front whose faces lie exactly in grid planes: each in-face fragment is
    owned by one cell only, so fragment areas still sum to the front area."""
    g = I.unit_grid(16)
    v, t = I.box_front((6 / 16, 6 / 16, 6 / 16), (10 / 16, 9 / 16, 11 / 16), 6)
    keys, tids, st = oracle.bin_pairs(v, t, g, margin=2)
    assert st == 0
    tot = 0.0
    for key, ti in zip(keys, tids):
        i, j, k = _decode(int(key), g)
        tot += np.linalg.norm(_poly_area_vec(oracle.clip_fragment(v[t[ti]], g, i, j, k)))
    ref = np.linalg.norm(_tri_area_vec(v, t), axis=1).sum()
    assert abs(tot - ref) < 1e-13 * ref


def test_outside_grid_and_bad_index_flagged():
    w = I.laplace_droplet_32(1)
    g, v, t = w["grid"], w["verts"].copy(), w["tris"].copy()
    v2 = v + np.array([0.3, 0.0, 0.0])
    _, _, st = oracle.bin_pairs(v2, t, g)
    assert st & 1
    t2 = t.copy()
    t2[5, 1] = len(v) + 7
    _, _, st2 = oracle.bin_pairs(v, t2, g)
    assert st2 & 8
