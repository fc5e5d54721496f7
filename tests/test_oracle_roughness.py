"""Pins of the oracle's local roughness detection and smoothing (Sec. 3.4,
Appendix A; Kuprat et al. 2001, Algorithm 4)."""
import numpy as np

import oracle
from paper_2505_06932_gb300 import inputs as I


def _box(n=6):
    return I.box_front((0.2, 0.25, 0.3), (0.7, 0.65, 0.8), n)


def test_planar_grid_faces_are_smooth_and_box_edges_are_right_angles():
    """On the faces of a triangulated box, interior vertices have a zero
    geometric Laplacian and zero edge roughness; an edge along a box edge has
    R_e = 1 - cos(90 deg) = 1."""
    v, t = _box()
    r = oracle.roughness(v, t)
    lo, hi = v.min(0), v.max(0)
    on_face = np.isclose(v, lo).astype(int) + np.isclose(v, hi).astype(int)
    interior = on_face.sum(1) == 1          # on exactly one face: not on a box edge
    assert interior.sum() > 0
    assert np.max(np.abs(r["gl"][interior])) <= 1e-15
    assert np.max(np.abs(r["G"][interior])) <= 1e-15 and np.max(r["V"][interior]) <= 1e-15
    # a vertex on a box edge (not a corner) has right-angle edges (R_e = 1) among
    # its edges, the others lie in a face (R_e = 0)
    edge = on_face.sum(1) == 2
    assert np.all(r["G"][edge] > 0.0)
    # every edge roughness value is 0 or 1 on a box
    G, V = r["G"][edge], r["V"][edge]
    # with k of m edges at 1 and the rest at 0: G = k/m, V = G (1 - G)
    assert np.allclose(V, G * (1.0 - G), atol=1e-15)


def test_edge_roughness_measures_curvature_on_spheres():
    """Appendix A: the dihedral angle arccos(1 - R_e) over the distance d between
    neighbouring triangle centres approximates the mean curvature 1/R (error of
    a few percent, independent of the refinement)."""
    for s, R in ((3, 0.3), (4, 0.25), (5, 0.2)):
        v, t = I.sphere_front(s, R, (0.5, 0.5, 0.5))
        r = oracle.roughness(v, t)
        # the mean edge roughness G_i relates to the mean dihedral angle; the mean
        # centre distance of the triangles around a vertex is about the edge
        # length over sqrt(3)
        e = np.linalg.norm(v[t[:, 0]] - v[t[:, 1]], axis=1).mean()
        d = e / np.sqrt(3.0)
        k = np.arccos(1.0 - r["G"]) / d
        assert abs(np.median(k) * R - 1.0) < 0.02, (s, np.median(k) * R)


def test_geometric_laplacian_points_outward_on_a_sphere():
    v, t = I.sphere_front(4, 0.25, (0.5, 0.5, 0.5))
    r = oracle.roughness(v, t)
    radial = v - 0.5
    assert np.all(np.einsum("ij,ij->i", r["gl"], radial) > 0.0)


def test_triangle_roughness_is_the_variance_weighted_mean():
    """R_t = sum G_i V_i / sum V_i: between the smallest and largest G of its
    vertices; with every V_i = 0 (box faces) the plain mean."""
    v, t = I.sphere_front(3, 0.3, (0.5, 0.5, 0.5), radial_noise=0.01, gen=I.rng(3))
    r = oracle.roughness(v, t)
    g = r["G"][t]
    assert np.all(r["rt"] >= g.min(1) - 1e-15) and np.all(r["rt"] <= g.max(1) + 1e-15)
    vb, tb = _box()
    rb = oracle.roughness(vb, tb)
    flat = np.all(rb["V"][tb] == 0.0, axis=1)
    assert np.allclose(rb["rt"][flat], rb["G"][tb][flat].mean(1), atol=1e-16)
    assert np.all(rb["rough"] == np.maximum(rb["r1"], rb["r2"]))


def _bumpy(seed=5):
    v, t = I.sphere_front(4, 0.25, (0.5, 0.5, 0.5))
    gen = I.rng(seed)
    idx = gen.choice(v.shape[0], 12, replace=False)
    v = v.copy()
    v[idx] = 0.5 + (v[idx] - 0.5) * (1.0 + gen.uniform(0.03, 0.06, (12, 1)))
    return v, t, idx


def test_smoothing_conserves_volume_and_removes_spikes():
    v, t, idx = _bumpy()
    r0 = oracle.roughness(*I.sphere_front(4, 0.25, (0.5, 0.5, 0.5)))
    gl_thr = 1.3 * np.linalg.norm(r0["gl"], axis=1).max()
    r_thr = 1.3 * r0["rough"].max()
    rb = oracle.roughness(v, t)
    assert np.linalg.norm(rb["gl"], axis=1).max() > gl_thr
    vol0 = oracle.signed_volume(v, t)
    vs, rounds, moved = oracle.roughness_smooth(v, t, gl_thr, r_thr)
    assert moved > 0 and 1 <= rounds < 64
    # every move keeps the enclosed volume (Kuprat's volume-conserving step)
    assert abs(oracle.signed_volume(vs, t) / vol0 - 1.0) <= 1e-13
    # the spikes are gone: the geometric Laplacian at the bumped vertices shrinks
    ra = oracle.roughness(vs, t)
    assert np.linalg.norm(ra["gl"][idx], axis=1).max() < 0.5 * np.linalg.norm(rb["gl"][idx], axis=1).max()
    # untouched far away: vertices whose stars contain no flagged edge do not move
    still = np.all(vs == v, axis=1)
    assert still.sum() > 0.5 * v.shape[0]


def test_smoothing_of_a_smooth_front_moves_nothing():
    v, t = I.sphere_front(4, 0.25, (0.5, 0.5, 0.5))
    r = oracle.roughness(v, t)
    vs, rounds, moved = oracle.roughness_smooth(v, t, 1.3 * np.linalg.norm(r["gl"], axis=1).max(),
                                                1.3 * r["rough"].max())
    assert moved == 0 and rounds == 0 and np.array_equal(vs, v)


def test_edge_priorities_are_distinct():
    p = [oracle.edge_priority(e) for e in range(20000)]
    assert len(set(p)) == len(p)
