"""Seeded synthetic inputs for the front/fluid coupling hot path.

This module only *generates* inputs: closed triangulated fronts, uniform
Cartesian grids and staggered face-velocity fields.  It holds none of the
method's arithmetic (no clipping, no volume fractions, no fits), so both the
CUDA path and the CPU oracle can take their inputs from here.

Shapes follow the workloads of the paper (arXiv 2505.06932):
  * spherical droplets at Laplace equilibrium (Sec. 4.1) -> icospheres,
  * an oscillating droplet (Sec. 4.3) -> spherical-harmonic deformation,
  * rising bubbles (Sec. 4.4) -> a flattened sphere with a dimpled base.
Every generator draws from ``numpy.random.Generator(PCG64(seed))``.
"""
from __future__ import annotations

import functools
import math
from dataclasses import dataclass

import numpy as np


@dataclass(frozen=True)
class Grid:
    """Uniform Cartesian grid of ``n[0] x n[1] x n[2]`` cubic cells of edge ``h``.

    Cell (i, j, k) spans ``origin + h*[i, i+1] x h*[j, j+1] x h*[k, k+1]``;
    the cell key is ``(i*n1 + j)*n2 + k`` (k fastest).
    """
    n: tuple
    origin: tuple
    h: float

    @property
    def ncells(self) -> int:
        return int(self.n[0]) * int(self.n[1]) * int(self.n[2])


def unit_grid(N: int) -> Grid:
    """The unit cube split into N^3 cells (h = 1/N)."""
    return Grid((N, N, N), (0.0, 0.0, 0.0), 1.0 / N)


def rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


# ----------------------------------------------------------------------------
# fronts
# ----------------------------------------------------------------------------

def icosphere(s: int):
    """Unit icosphere after ``s`` 4-to-1 subdivisions (fresh copies of a cached mesh).

    Returns ``verts (10*4^s+2, 3) float64`` on the unit sphere and
    ``tris (20*4^s, 3) int32`` ordered counter-clockwise seen from outside.
    """
    v, t = _icosphere(s)
    return v.copy(), t.copy()


@functools.lru_cache(maxsize=None)
def _icosphere(s: int):
    """Unit icosphere after ``s`` 4-to-1 subdivisions.

    Returns ``verts (10*4^s+2, 3) float64`` on the unit sphere and
    ``tris (20*4^s, 3) int32`` ordered counter-clockwise seen from outside.
    """
    t = (1.0 + 5.0 ** 0.5) / 2.0
    v = np.array([[-1, t, 0], [1, t, 0], [-1, -t, 0], [1, -t, 0],
                  [0, -1, t], [0, 1, t], [0, -1, -t], [0, 1, -t],
                  [t, 0, -1], [t, 0, 1], [-t, 0, -1], [-t, 0, 1]], dtype=np.float64)
    v /= np.linalg.norm(v, axis=1, keepdims=True)
    f = np.array([[0, 11, 5], [0, 5, 1], [0, 1, 7], [0, 7, 10], [0, 10, 11],
                  [1, 5, 9], [5, 11, 4], [11, 10, 2], [10, 7, 6], [7, 1, 8],
                  [3, 9, 4], [3, 4, 2], [3, 2, 6], [3, 6, 8], [3, 8, 9],
                  [4, 9, 5], [2, 4, 11], [6, 2, 10], [8, 6, 7], [9, 8, 1]], dtype=np.int64)
    for _ in range(s):
        a, b, c = f[:, 0], f[:, 1], f[:, 2]
        edges = np.concatenate([np.stack([a, b], 1), np.stack([b, c], 1), np.stack([c, a], 1)])
        es = np.sort(edges, axis=1)
        uniq, inv = np.unique(es, axis=0, return_inverse=True)
        inv = inv.reshape(-1)
        mid = v[uniq[:, 0]] + v[uniq[:, 1]]
        mid /= np.linalg.norm(mid, axis=1, keepdims=True)
        base = v.shape[0]
        v = np.concatenate([v, mid])
        T = f.shape[0]
        ab, bc, ca = base + inv[:T], base + inv[T:2 * T], base + inv[2 * T:]
        f = np.concatenate([np.stack([a, ab, ca], 1), np.stack([b, bc, ab], 1),
                            np.stack([c, ca, bc], 1), np.stack([ab, bc, ca], 1)])
    return np.ascontiguousarray(v), np.ascontiguousarray(f.astype(np.int32))


def sphere_front(s: int, R: float, centre, radial_noise: float = 0.0, gen=None):
    """Icosphere of radius ``R`` about ``centre``; optional radial noise U[-a, a]."""
    v, f = icosphere(s)
    r = np.full(v.shape[0], R)
    if radial_noise:
        r = r + gen.uniform(-radial_noise, radial_noise, size=v.shape[0])
    return np.ascontiguousarray(np.asarray(centre)[None, :] + v * r[:, None]), f


def real_sph_harm(l: int, m: int, theta: np.ndarray, phi: np.ndarray) -> np.ndarray:
    """Orthonormal real spherical harmonic Y_lm (theta polar, phi azimuth)."""
    from scipy.special import lpmv
    am = abs(m)
    norm = math.sqrt((2 * l + 1) / (4 * math.pi) * math.factorial(l - am) / math.factorial(l + am))
    p = lpmv(am, l, np.cos(theta))
    if m == 0:
        return norm * p
    if m > 0:
        return math.sqrt(2.0) * norm * p * np.cos(m * phi)
    return math.sqrt(2.0) * norm * p * np.sin(am * phi)


def sh_deformed_front(s: int, R: float, centre, gen, lmin: int = 2, lmax: int = 8,
                      rel_sigma: float = 0.05):
    """Icosphere with radius r(theta, phi) = R + sum_{l,m} c_lm Y_lm, c ~ N(0, (rel_sigma R)^2)."""
    v, f = icosphere(s)
    theta = np.arccos(np.clip(v[:, 2], -1.0, 1.0))
    phi = np.arctan2(v[:, 1], v[:, 0])
    r = np.full(v.shape[0], R)
    for l in range(lmin, lmax + 1):
        for m in range(-l, l + 1):
            r = r + gen.normal(0.0, rel_sigma * R) * real_sph_harm(l, m, theta, phi)
    if np.any(r <= 0.0):
        raise ValueError("spherical-harmonic deformation produced a non-positive radius")
    return np.ascontiguousarray(np.asarray(centre)[None, :] + v * r[:, None]), f


def bubble_front(verts: np.ndarray, centre, R: float, flatten: float = 0.7,
                 dent_depth: float = 0.1, dent_width: float = 0.3):
    """Flatten a front by z -> flatten*z about ``centre`` and dimple its base.

    Vertices below the centre are raised by a Gaussian dent of depth
    ``dent_depth*R`` and width ``dent_width*R`` about the vertical axis.
    """
    c = np.asarray(centre)
    p = verts - c[None, :]
    p[:, 2] *= flatten
    rho2 = p[:, 0] ** 2 + p[:, 1] ** 2
    below = p[:, 2] < 0.0
    p[below, 2] += dent_depth * R * np.exp(-rho2[below] / (2.0 * (dent_width * R) ** 2))
    return np.ascontiguousarray(p + c[None, :])


def box_front(lo, hi, ncell):
    """Closed axis-aligned box [lo, hi] with each face split into ncell x ncell
    quads (two triangles each); counter-clockwise seen from outside."""
    lo = np.asarray(lo, dtype=np.float64)
    hi = np.asarray(hi, dtype=np.float64)
    verts, tris = [], []

    def face(origin, du, dv):
        base = sum(len(x) for x in verts)
        u = np.linspace(0.0, 1.0, ncell + 1)
        uu, vv = np.meshgrid(u, u, indexing="ij")
        pts = origin[None, :] + uu.reshape(-1, 1) * du[None, :] + vv.reshape(-1, 1) * dv[None, :]
        verts.append(pts)
        idx = np.arange((ncell + 1) ** 2).reshape(ncell + 1, ncell + 1) + base
        a = idx[:-1, :-1].ravel()
        b = idx[1:, :-1].ravel()
        c = idx[1:, 1:].ravel()
        d = idx[:-1, 1:].ravel()
        tris.append(np.stack([a, b, c], 1))
        tris.append(np.stack([a, c, d], 1))

    ex = np.array([hi[0] - lo[0], 0, 0])
    ey = np.array([0, hi[1] - lo[1], 0])
    ez = np.array([0, 0, hi[2] - lo[2]])
    # each face: du x dv points outward
    face(lo, ey, ex)                       # z = lo (normal -z)
    face(lo + ez, ex, ey)                  # z = hi (+z)
    face(lo, ex, ez)                       # y = lo (-y)
    face(lo + ey, ez, ex)                  # y = hi (+y)
    face(lo, ez, ey)                       # x = lo (-x)
    face(lo + ex, ey, ez)                  # x = hi (+x)
    v = np.concatenate(verts)
    t = np.concatenate(tris)
    # weld duplicated edge vertices so the surface is closed
    key = np.round(v * 1e12).astype(np.int64)
    _, first, inv = np.unique(key, axis=0, return_index=True, return_inverse=True)
    inv = inv.reshape(-1)
    vw = v[first]
    tw = inv[t]
    return np.ascontiguousarray(vw), np.ascontiguousarray(tw.astype(np.int32))


def signed_volume(verts: np.ndarray, tris: np.ndarray) -> float:
    """(1/6) sum_t x_a . (x_b x x_c): the divergence-theorem volume of a closed mesh."""
    a, b, c = verts[tris[:, 0]], verts[tris[:, 1]], verts[tris[:, 2]]
    return float(np.sum(np.einsum("ij,ij->i", a, np.cross(b, c))) / 6.0)


# ----------------------------------------------------------------------------
# staggered face velocities: U (n0+1, n1, n2), V (n0, n1+1, n2), W (n0, n1, n2+1)
# ----------------------------------------------------------------------------

def face_centres(g: Grid, axis: int):
    """Coordinates (X, Y, Z) of the centres of the faces normal to ``axis``."""
    n = list(g.n)
    ax = [np.arange(n[d], dtype=np.float64) + 0.5 for d in range(3)]
    ax[axis] = np.arange(n[axis] + 1, dtype=np.float64)
    X, Y, Z = np.meshgrid(*ax, indexing="ij")
    return (g.origin[0] + X * g.h, g.origin[1] + Y * g.h, g.origin[2] + Z * g.h)


def solid_body_faces(g: Grid, centre, gen, omega: float = 1.0, noise: float = 1e-3):
    """Solid-body rotation u = omega * a x (x - c) about a seeded unit axis a,
    sampled at face centres, plus N(0, noise^2) on every face value."""
    a = gen.normal(size=3)
    a /= np.linalg.norm(a)
    w = omega * a
    c = np.asarray(centre, dtype=np.float64)
    out = []
    for axis in range(3):
        X, Y, Z = face_centres(g, axis)
        r = np.stack([X - c[0], Y - c[1], Z - c[2]], -1)
        u = np.cross(np.broadcast_to(w, r.shape), r)[..., axis]
        if noise:
            u = u + gen.normal(0.0, noise, size=u.shape)
        out.append(np.ascontiguousarray(u))
    return tuple(out), w


def taylor_green_faces(g: Grid, gen, amp: float = 1.0):
    """Divergence-free Taylor-Green field with seeded phases:
    u = A sin(2pi x') cos(2pi y') cos(2pi z'), v = -A cos(2pi x') sin(2pi y') cos(2pi z'),
    w = 0, with x' = x + phi_x etc."""
    ph = gen.uniform(0.0, 1.0, size=3)
    tp = 2.0 * math.pi
    out = []
    for axis in range(3):
        X, Y, Z = face_centres(g, axis)
        xs, ys, zs = X + ph[0], Y + ph[1], Z + ph[2]
        if axis == 0:
            u = amp * np.sin(tp * xs) * np.cos(tp * ys) * np.cos(tp * zs)
        elif axis == 1:
            u = -amp * np.cos(tp * xs) * np.sin(tp * ys) * np.cos(tp * zs)
        else:
            u = np.zeros_like(X)
        out.append(np.ascontiguousarray(u))
    return tuple(out), ph


# ----------------------------------------------------------------------------
# the workloads (all seeded)
# ----------------------------------------------------------------------------

def laplace_droplet_32(seed: int = 1):
    """Icosphere s=4 (5,120 triangles), R=0.25, centre 0.5 + U[0,h)^3, 32^3 grid,
    solid-body rotation + N(0, 1e-3) face noise (Laplace-equilibrium droplet)."""
    g = unit_grid(32)
    gen = rng(seed)
    centre = 0.5 + gen.uniform(0.0, g.h, size=3)
    verts, tris = sphere_front(4, 0.25, centre)
    faces, omega = solid_body_faces(g, centre, gen)
    return dict(name="icosphere_s4_R0.25_32^3", grid=g, verts=verts, tris=tris,
                faces=faces, centre=centre, R=0.25, omega=omega)


def rough_sphere_128(seed: int = 2):
    """Icosphere s=6 (81,920 triangles), R=0.2, radial noise U[-1e-3 h, 1e-3 h], 128^3."""
    g = unit_grid(128)
    gen = rng(seed)
    centre = 0.5 + gen.uniform(0.0, g.h, size=3)
    verts, tris = sphere_front(6, 0.2, centre, radial_noise=1e-3 * g.h, gen=gen)
    faces, omega = solid_body_faces(g, centre, gen)
    return dict(name="rough_icosphere_s6_R0.2_128^3", grid=g, verts=verts, tris=tris,
                faces=faces, centre=centre, R=0.2, omega=omega)


def ellipsoid_128(seed: int = 3):
    """The s=6 icosphere of radius 0.2 scaled by (1.5, 1.0, 0.75): semi-axes (0.3, 0.2, 0.15), 128^3."""
    g = unit_grid(128)
    gen = rng(seed)
    centre = 0.5 + gen.uniform(0.0, g.h, size=3)
    v, tris = icosphere(6)
    axes = np.array([0.3, 0.2, 0.15])
    verts = np.ascontiguousarray(centre[None, :] + v * axes[None, :])
    faces, omega = solid_body_faces(g, centre, gen)
    return dict(name="ellipsoid_s6_0.3x0.2x0.15_128^3", grid=g, verts=verts, tris=tris,
                faces=faces, centre=centre, axes=axes, omega=omega)


def sh_droplet_256(seed: int = 4, bubble: bool = False, s: int = 7, N: int = 256):
    """Icosphere s=7 (327,680 triangles), R=0.2, real-SH deformation l=2..8 with
    c_lm ~ N(0, (0.05R)^2), optionally flattened and dimpled (rising bubble);
    Taylor-Green faces of amplitude 1 on a 256^3 grid."""
    g = unit_grid(N)
    gen = rng(seed)
    centre = 0.5 + gen.uniform(0.0, g.h, size=3)
    verts, tris = sh_deformed_front(s, 0.2, centre, gen)
    if bubble:
        verts = bubble_front(verts, centre, 0.2)
    faces, phase = taylor_green_faces(g, gen)
    name = ("bubble" if bubble else "sh_droplet") + f"_s{s}_R0.2_{N}^3"
    return dict(name=name, grid=g, verts=verts, tris=tris, faces=faces, centre=centre, R=0.2)


def small_sphere(s: int, R: float, N: int, seed: int = 0, noise_h: float = 0.0):
    """A seeded icosphere of radius R on an N^3 unit grid with face velocities
    (used for parity cases at oracle-friendly sizes)."""
    g = unit_grid(N)
    gen = rng(seed)
    centre = 0.5 + gen.uniform(0.0, g.h, size=3)
    verts, tris = sphere_front(s, R, centre, radial_noise=noise_h * g.h, gen=gen)
    faces, omega = solid_body_faces(g, centre, gen)
    return dict(name=f"icosphere_s{s}_R{R}_{N}^3", grid=g, verts=verts, tris=tris,
                faces=faces, centre=centre, R=R, omega=omega)


# ----------------------------------------------------------------------------
# batched form: many independent fronts of uneven size
# ----------------------------------------------------------------------------

def batch_fronts(seed: int = 5, count: int = 512, delta_max_h: float = 4.0, s_choices=(3, 4, 5, 6),
                 n_choices=(32, 48, 64, 96), rmin_h: float = 3.0, rmax_h: float = 20.0, noise_h: float = 1e-3):
    """``count`` independent rough icospheres, each on its own unit grid:
    subdivision s ~ U(s_choices), N ~ U(n_choices), radius log-uniform in
    [rmin_h h, rmax_h h] capped so that the front keeps the grid margin
    2 + ceil(delta_max/h) (plus one cell), centre uniform where it fits,
    radial roughness U[-noise_h h, noise_h h] per vertex.  Returns a list of
    dicts (grid, verts, tris, centre, R, s, omega: the solid-body rotation
    vector used for face velocities, capped: whether the radius was capped)."""
    gen = rng(seed)
    margin = 2 + math.ceil(delta_max_h)
    out = []
    for b in range(count):
        s = int(gen.choice(s_choices))
        N = int(gen.choice(n_choices))
        g = unit_grid(N)
        h = g.h
        r = math.exp(gen.uniform(math.log(rmin_h * h), math.log(rmax_h * h)))
        rcap = (N / 2 - margin - 2) * h
        capped = r > rcap
        r = min(r, rcap)
        lo = (margin + 1) * h + r + 2 * noise_h * h
        hi = 1.0 - lo
        centre = np.array([gen.uniform(lo, hi) if hi > lo else 0.5 for _ in range(3)])
        verts, tris = sphere_front(s, r, centre, radial_noise=noise_h * h, gen=gen)
        a = gen.normal(size=3)
        a /= np.linalg.norm(a)
        out.append(dict(name=f"batch{b}_s{s}_N{N}", grid=g, verts=verts, tris=tris, centre=centre, R=r, s=s,
                        omega=a, capped=capped))
    return out


def solid_body_faces_exact(g: Grid, centre, omega):
    """Noise-free solid-body rotation u = omega x (x - c) at the face centres
    (a linear divergence-free field, reproduced exactly by the interpolation)."""
    w = np.asarray(omega, dtype=np.float64)
    c = np.asarray(centre, dtype=np.float64)
    out = []
    for axis in range(3):
        X, Y, Z = face_centres(g, axis)
        r = np.stack([X - c[0], Y - c[1], Z - c[2]], -1)
        out.append(np.ascontiguousarray(np.cross(np.broadcast_to(w, r.shape), r)[..., axis]))
    return tuple(out)


# ----------------------------------------------------------------------------
# served form: a stream of requests
# ----------------------------------------------------------------------------

def served_requests(seed: int = 11, count: int = 48, rate: float = 100.0, s_choices=(4, 5, 6, 7, 8),
                    n_choices=(32, 64, 128, 256, 512), max_steps: int = 50, pool_per_s: int = 2,
                    delta_max_h: float = 4.0):
    """A request stream: Poisson arrivals of the given rate (requests/s); each
    request a spherical-harmonic-deformed icosphere (l = 2..8, c ~ N(0, (0.05R)^2),
    the oscillating-droplet shape) with s ~ U(s_choices), on a unit grid with
    N ~ U(n_choices), taking steps ~ U{1..max_steps} time steps of dt = 0.25 h,
    advected by a solid-body rotation about its centre (speed 1 at 1.5 R, a
    seeded axis).  The deformed shapes come from a pool of pool_per_s shapes per
    subdivision (unit radius), scaled to R = 0.2 or less, so that the front keeps
    the grid margin 2 + ceil(delta_max/h) plus two cells.  Returns dicts with
    grid, verts, tris, steps, arrival, dt, centre, omega, s, R."""
    gen = rng(seed)
    pool = {}
    for s in s_choices:
        for k in range(pool_per_s):
            v, t = sh_deformed_front(s, 1.0, np.zeros(3), rng(1000 * s + k))
            pool[(s, k)] = (v, t, float(np.linalg.norm(v, axis=1).max()))
    margin = 2 + math.ceil(delta_max_h)
    out = []
    t = 0.0
    for i in range(count):
        t += gen.exponential(1.0 / rate)
        s = int(gen.choice(s_choices))
        k = int(gen.integers(pool_per_s))
        N = int(gen.choice(n_choices))
        g = unit_grid(N)
        v, tri, rmax = pool[(s, k)]
        R = min(0.2, (N / 2 - margin - 2) * g.h / rmax)
        centre = 0.5 + gen.uniform(0.0, g.h, size=3)
        a = gen.normal(size=3)
        a *= 1.0 / (1.5 * R * np.linalg.norm(a))
        out.append(dict(rid=i, grid=g, verts=np.ascontiguousarray(centre + R * v), tris=tri,
                        steps=int(gen.integers(1, max_steps + 1)), arrival=t, dt=0.25 * g.h,
                        centre=centre, omega=a, s=s, R=R))
    return out


def random_frames(gen, m: int) -> np.ndarray:
    """m random right-handed orthonormal frames, rows (t1, t2, n), as (m, 9)."""
    out = np.empty((m, 9))
    for c in range(m):
        Q, R = np.linalg.qr(gen.normal(size=(3, 3)))
        Q = Q * np.sign(np.diag(R))
        if np.linalg.det(Q) < 0:
            Q[:, 2] = -Q[:, 2]
        out[c] = Q.T.reshape(9)
    return out


def paraboloid_cells(seed: int = 21, m: int = 512):
    """Cut-cell paraboloids in cell units: random frames and coefficients of
    z = a1 + a2 x + a3 y + a4 x^2 + a5 x y + a6 y^2 spanning planes, the
    curvatures of fitted fronts (|a4..a6| up to 0.06 for R >= 8h), strongly
    curved patches (up to 0.4), steep slopes and heights that cut the cell
    anywhere from a corner to the middle; every fifth cell is axis-aligned
    (a signed permutation frame), where degenerate cases (faces parallel to
    the tangent plane) occur."""
    gen = rng(seed)
    fr = random_frames(gen, m)
    perms = [(0, 1, 2), (1, 2, 0), (2, 0, 1)]
    for c in range(0, m, 5):
        p = perms[(c // 5) % 3]
        s = gen.choice([-1.0, 1.0], 2)
        E = np.eye(3)[list(p)]
        E[0] *= s[0]
        E[1] *= s[1]
        E[2] = np.cross(E[0], E[1])
        fr[c] = E.reshape(9)
    co = np.zeros((m, 6))
    co[:, 0] = gen.uniform(-0.6, 0.6, m)
    co[:, 1:3] = gen.uniform(-0.5, 0.5, (m, 2)) * gen.choice([0.0, 0.1, 1.0], (m, 1))
    co[:, 3:] = gen.uniform(-1.0, 1.0, (m, 3)) * gen.choice([0.0, 0.01, 0.06, 0.4], (m, 1))
    return fr, co
