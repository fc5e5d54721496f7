"""Independent geometric references used to pin the oracle (numpy only).

None of these share code with the oracle or the CUDA path; each is a textbook
construction chosen so that a mistake in the oracle shows up against it:
  * convex polyhedron clipping (cell cube cut by the faces of a convex front),
  * generalized winding numbers (Van Oosterom & Strackee solid angles),
  * the separating-axis triangle/box overlap test,
  * the corner-simplex (inclusion-exclusion) volume of a plane-cut cube,
  * an exact quadrature rule for quadratics on triangles.
"""
from __future__ import annotations

import itertools
import math

import numpy as np


# ---------------------------------------------------------------------------
# convex polyhedra as face lists
# ---------------------------------------------------------------------------

def cube_faces(lo, hi):
    """Faces (counter-clockwise seen from outside) of the box [lo, hi]."""
    x0, y0, z0 = lo
    x1, y1, z1 = hi
    P = lambda x, y, z: np.array([x, y, z], dtype=np.float64)
    return [
        [P(x0, y0, z0), P(x0, y1, z0), P(x1, y1, z0), P(x1, y0, z0)],  # -z
        [P(x0, y0, z1), P(x1, y0, z1), P(x1, y1, z1), P(x0, y1, z1)],  # +z
        [P(x0, y0, z0), P(x1, y0, z0), P(x1, y0, z1), P(x0, y0, z1)],  # -y
        [P(x0, y1, z0), P(x0, y1, z1), P(x1, y1, z1), P(x1, y1, z0)],  # +y
        [P(x0, y0, z0), P(x0, y0, z1), P(x0, y1, z1), P(x0, y1, z0)],  # -x
        [P(x1, y0, z0), P(x1, y1, z0), P(x1, y1, z1), P(x1, y0, z1)],  # +x
    ]


def _clip_poly_plane(poly, n, d):
    """Keep the part of a planar polygon with n.x <= d."""
    out = []
    m = len(poly)
    for i in range(m):
        a, b = poly[i - 1], poly[i]
        fa, fb = float(n @ a) - d, float(n @ b) - d
        if fb <= 0.0:
            if fa > 0.0:
                t = fa / (fa - fb)
                out.append(a + t * (b - a))
            out.append(b)
        elif fa <= 0.0:
            t = fa / (fa - fb)
            out.append(a + t * (b - a))
    return out


def clip_polyhedron(faces, n, d):
    """Convex polyhedron (face list) cut by the half-space n.x <= d."""
    n = np.asarray(n, dtype=np.float64)
    new = []
    cap = []
    for f in faces:
        c = _clip_poly_plane(f, n, d)
        if len(c) >= 3:
            new.append(c)
        for p in c:
            if abs(float(n @ p) - d) <= 1e-13 * max(1.0, abs(d)):
                cap.append(p)
    if len(cap) >= 3:
        cap = np.array(cap)
        ctr = cap.mean(axis=0)
        u = cap[0] - ctr
        if np.linalg.norm(u) == 0.0:
            u = cap[1] - ctr
        u /= np.linalg.norm(u)
        v = np.cross(n / np.linalg.norm(n), u)
        ang = np.arctan2((cap - ctr) @ v, (cap - ctr) @ u)
        order = np.argsort(ang)
        ring = [cap[i] for i in order]
        # drop duplicates
        ring2 = [ring[0]]
        for p in ring[1:]:
            if np.linalg.norm(p - ring2[-1]) > 1e-15:
                ring2.append(p)
        if len(ring2) >= 3:
            new.append(ring2)  # counter-clockwise about +n = outward for the cap
    return new


def polyhedron_volume(faces):
    """Divergence theorem: V = (1/3) sum_f c_f . A_f."""
    vol = 0.0
    for f in faces:
        p0 = f[0]
        for a, b in zip(f[1:-1], f[2:]):
            vol += float(p0 @ np.cross(a, b)) / 6.0
    return vol


def convex_cell_fraction(cell_lo, h, planes):
    """vol(cell cap convex region)/h^3, the region being the intersection of
    the half-spaces n.x <= d in ``planes`` (list of (n, d))."""
    faces = cube_faces(cell_lo, np.asarray(cell_lo) + h)
    corners = np.array(list(itertools.product(*[(c, c + h) for c in cell_lo])))
    for n, d in planes:
        s = corners @ n - d
        if np.all(s <= 0.0):
            continue
        if np.all(s >= 0.0) and np.any(s > 0.0) and np.min(s) > 0.0:
            return 0.0
        faces = clip_polyhedron(faces, n, d)
        if not faces:
            return 0.0
    return polyhedron_volume(faces) / h ** 3


def face_planes(verts, tris):
    """(outward unit normal, offset) of every triangle of a convex closed mesh."""
    a, b, c = verts[tris[:, 0]], verts[tris[:, 1]], verts[tris[:, 2]]
    n = np.cross(b - a, c - a)
    n /= np.linalg.norm(n, axis=1, keepdims=True)
    d = np.einsum("ij,ij->i", n, a)
    return n, d


def convex_polyhedron_mesh(planes, big=10.0):
    """Closed triangle mesh (outward counter-clockwise) of the convex region
    bounded by the half-spaces n.x <= d."""
    faces = cube_faces((-big, -big, -big), (big, big, big))
    for n, d in planes:
        faces = clip_polyhedron(faces, np.asarray(n, dtype=np.float64), float(d))
    verts, tris = [], []
    for f in faces:
        base = len(verts)
        verts.extend(f)
        for m in range(1, len(f) - 1):
            tris.append((base, base + m, base + m + 1))
    return np.array(verts), np.array(tris, dtype=np.int32)


# ---------------------------------------------------------------------------
# winding numbers
# ---------------------------------------------------------------------------

def winding_numbers(verts, tris, pts, chunk=2048):
    """Generalized winding number of a closed mesh at each point:
    (1/4pi) sum_t solid angle, with tan(Omega/2) = a.(b x c) /
    (|a||b||c| + (a.b)|c| + (a.c)|b| + (b.c)|a|)  (Van Oosterom & Strackee 1983)."""
    A, B, Cc = verts[tris[:, 0]], verts[tris[:, 1]], verts[tris[:, 2]]
    out = np.empty(len(pts))
    for s in range(0, len(pts), chunk):
        p = pts[s:s + chunk, None, :]
        a, b, c = A[None] - p, B[None] - p, Cc[None] - p
        la, lb, lc = (np.linalg.norm(x, axis=2) for x in (a, b, c))
        num = np.einsum("ptk,ptk->pt", a, np.cross(b, c))
        den = (la * lb * lc + np.einsum("ptk,ptk->pt", a, b) * lc + np.einsum("ptk,ptk->pt", a, c) * lb
               + np.einsum("ptk,ptk->pt", b, c) * la)
        out[s:s + chunk] = np.sum(2.0 * np.arctan2(num, den), axis=1) / (4.0 * math.pi)
    return out


# ---------------------------------------------------------------------------
# triangle / box overlap (separating axis theorem)
# ---------------------------------------------------------------------------

def tri_box_overlap(tri, lo, hi, eps=0.0):
    """True iff the closed triangle and the closed box are not separated by
    any of the 13 axes (box normals, triangle normal, 9 edge cross products).
    With eps > 0 a separation by less than eps is ignored (touching counts)."""
    c = (np.asarray(lo) + np.asarray(hi)) / 2.0
    e = (np.asarray(hi) - np.asarray(lo)) / 2.0
    v = np.asarray(tri) - c
    edges = [v[1] - v[0], v[2] - v[1], v[0] - v[2]]
    axes = [np.eye(3)[i] for i in range(3)] + [np.cross(edges[0], edges[1])]
    for i in range(3):
        for ed in edges:
            axes.append(np.cross(np.eye(3)[i], ed))
    for ax in axes:
        nn = np.linalg.norm(ax)
        if nn == 0.0:
            continue
        p = v @ ax
        r = float(np.abs(ax) @ e)
        if p.min() > r + eps * nn or p.max() < -r - eps * nn:
            return False
    return True


# ---------------------------------------------------------------------------
# closed forms and quadrature
# ---------------------------------------------------------------------------

def plane_cut_unit_cube(nvec, d):
    """Volume of {x in [0,1]^3 : n.x <= d} for n with positive components
    (inclusion-exclusion over the cube corners)."""
    n1, n2, n3 = nvec
    H = lambda s: s ** 3 if s > 0.0 else 0.0
    s = H(d) - H(d - n1) - H(d - n2) - H(d - n3) + H(d - n1 - n2) + H(d - n1 - n3) + H(d - n2 - n3) \
        - H(d - n1 - n2 - n3)
    return s / (6.0 * n1 * n2 * n3)


def triangle_quadratic_integrals(a, b, c):
    """[int 1, int x, int y, int x^2, int xy, int y^2] over the 2D triangle (a,b,c),
    signed by orientation, with the edge-midpoint rule (exact for quadratics)."""
    a, b, c = (np.asarray(x, dtype=np.float64) for x in (a, b, c))
    area = 0.5 * ((b[0] - a[0]) * (c[1] - a[1]) - (b[1] - a[1]) * (c[0] - a[0]))
    mids = [(a + b) / 2, (b + c) / 2, (c + a) / 2]
    f = lambda p: np.array([1.0, p[0], p[1], p[0] ** 2, p[0] * p[1], p[1] ** 2])
    return area / 3.0 * sum(f(m) for m in mids)


def ellipsoid_mean_curvature_at(p, axes):
    """kappa = div n (= 2H, > 0 on convex surfaces) of x^2/a^2 + y^2/b^2 + z^2/c^2 = 1
    at the surface point p:  (a^2+b^2+c^2-|p|^2) / (a^2 b^2 c^2 (x^2/a^4+y^2/b^4+z^2/c^4)^{3/2})."""
    a, b, c = axes
    x, y, z = p
    q = x * x / a ** 4 + y * y / b ** 4 + z * z / c ** 4
    return (a * a + b * b + c * c - (x * x + y * y + z * z)) / (a * a * b * b * c * c * q ** 1.5)


def closest_point_on_ellipsoid(p, axes, iters=60):
    """Closest point of the ellipsoid to p (Newton on the Lagrange parameter)."""
    a = np.asarray(axes, dtype=np.float64)
    p = np.asarray(p, dtype=np.float64)
    t = 0.0
    for _ in range(iters):
        x = a * a * p / (a * a + t)
        f = np.sum((x / a) ** 2) - 1.0
        df = -2.0 * np.sum(a * a * p * p / (a * a + t) ** 3)
        t -= f / df
    return a * a * p / (a * a + t)
