"""Pins of the oracle's paraboloid cut-cell quantities (Sec. 3.2: alpha = V_P/V_C
of the cell below the fitted paraboloid, curvature and normal averaged over
the paraboloid surface inside the cell), against closed forms, identities and
brute force that do not use the oracle's own integration."""
import itertools

import numpy as np
from numpy.polynomial.legendre import leggauss

import oracle
from paper_2505_06932_gb300 import inputs as I


def _plane_volume(m, c):
    """|{X in [-1/2,1/2]^3 : m.X <= c}| for m with no zero component: the
    inclusion-exclusion formula over the corners of the unit cube."""
    m = np.array(m, float)
    cc = c + 0.5 * m.sum()          # Y = X + 1/2 in [0, 1]^3
    for d in range(3):              # reflect axes with m_d < 0
        if m[d] < 0:
            cc -= m[d]
            m[d] = -m[d]
    tot = 0.0
    for e in itertools.product((0, 1), repeat=3):
        v = cc - np.dot(m, e)
        if v > 0:
            tot += (-1) ** sum(e) * v ** 3
    return tot / (6.0 * m[0] * m[1] * m[2])


def _plane_area(m, c):
    """Area of {m.X = c} inside the cube: the polygon of its cube-edge crossings."""
    m = np.asarray(m, float)
    nm = np.linalg.norm(m)
    m, c = m / nm, c / nm
    P = []
    for f in range(3):
        d, e = (f + 1) % 3, (f + 2) % 3
        for s1, s2 in itertools.product((-0.5, 0.5), repeat=2):
            t = (c - m[d] * s1 - m[e] * s2) / m[f]
            if -0.5 <= t <= 0.5:
                X = np.zeros(3)
                X[d], X[e], X[f] = s1, s2, t
                P.append(X)
    P = np.array(P)
    ctr = P.mean(0)
    u = (P[0] - ctr) / np.linalg.norm(P[0] - ctr)
    v = np.cross(m, u)
    P = P[np.argsort(np.arctan2((P - ctr) @ v, (P - ctr) @ u))]
    return 0.5 * np.linalg.norm(sum(np.cross(P[i], P[(i + 1) % len(P)]) for i in range(len(P))))


def _frames(seed, m):
    return I.random_frames(I.rng(seed), m)


def test_planes_match_the_cube_cut_closed_forms():
    """a4 = a5 = a6 = 0: the surface is the plane n.X - a2 t1.X - a3 t2.X = a1;
    V by inclusion-exclusion, the area of the section polygon, kbar = 0 and
    nbar = the plane's unit normal."""
    gen = I.rng(31)
    fr = _frames(31, 40)
    co = np.zeros((40, 6))
    co[:, 0] = gen.uniform(-0.5, 0.5, 40)
    co[:, 1:3] = gen.uniform(-0.6, 0.6, (40, 2))
    o = oracle.paraboloid_cells(fr, co)
    for c in range(40):
        t1, t2, n = fr[c].reshape(3, 3)
        m = n - co[c, 1] * t1 - co[c, 2] * t2
        assert abs(o["alpha"][c] - _plane_volume(m, co[c, 0])) <= 1e-13
        if o["status"][c] == 0:
            assert abs(o["area"][c] - _plane_area(m, co[c, 0])) <= 1e-12
            assert abs(o["kbar"][c]) <= 1e-15
            assert np.max(np.abs(o["nbar"][c] - m / np.linalg.norm(m))) <= 1e-13
        else:
            assert o["area"][c] == 0.0 and _plane_volume(m, co[c, 0]) in (0.0, 1.0)


def _whole_square(co, nq=64):
    """A, kbar and int n dA of z = P(x, y) over the whole square [-1/2, 1/2]^2
    by a tensor Gauss-Legendre rule (the integrands are smooth there)."""
    x, w = leggauss(nq)
    x, w = 0.5 * x, 0.5 * w
    X, Y = np.meshgrid(x, x, indexing="ij")
    W2 = np.outer(w, w)
    a = co
    px = a[1] + 2 * a[3] * X + a[4] * Y
    py = a[2] + a[4] * X + 2 * a[5] * Y
    G = np.sqrt(1 + px ** 2 + py ** 2)
    kap = -((1 + py ** 2) * 2 * a[3] - 2 * px * py * a[4] + (1 + px ** 2) * 2 * a[5]) / G ** 3
    A = (W2 * G).sum()
    N = np.array([(W2 * -px).sum(), (W2 * -py).sum(), W2.sum()])
    return A, (W2 * kap * G).sum() / A, N / np.linalg.norm(N)


def test_paraboloid_over_the_whole_cell_matches_tensor_quadrature():
    """In an axis-aligned frame a paraboloid with |P| < 1/2 on the whole square
    crosses every vertical column once: V = a1 + 1/2 + (a4 + a6)/12 exactly,
    and the surface integrals are smooth integrals over the square.  Every
    right-handed signed permutation frame (a cube symmetry) gives the same V,
    A and kbar, and the normal turns with the frame."""
    cases = [np.array([0.1, 0.05, -0.08, 0.2, 0.1, -0.15]), np.array([-0.2, 0.0, 0.0, 0.06, 0.0, 0.06]),
             np.array([0.0, 0.3, 0.2, -0.1, 0.05, 0.1])]
    frames = []
    for p in itertools.permutations(range(3)):
        for s in itertools.product((-1.0, 1.0), repeat=2):
            E = np.eye(3)[list(p)]
            E[0] *= s[0]
            E[1] *= s[1]
            E[2] = np.cross(E[0], E[1])
            frames.append(E)
    for co in cases:
        A, kb, nl = _whole_square(co)
        fr = np.array([E.reshape(9) for E in frames])
        o = oracle.paraboloid_cells(fr, np.tile(co, (len(frames), 1)))
        assert np.max(np.abs(o["alpha"] - (co[0] + 0.5 + (co[3] + co[5]) / 12.0))) <= 1e-13
        assert np.max(np.abs(o["area"] - A)) <= 1e-12
        assert np.max(np.abs(o["kbar"] - kb)) <= 1e-12
        for E, nb in zip(frames, o["nbar"]):
            assert np.max(np.abs(nb - E.T @ nl)) <= 1e-13


def test_complement_and_rotation_about_the_normal():
    """(t2, t1, -n) with P'(x', y') = -P(y', x') bounds the complement:
    V + V' = 1, the same surface (A' = A), kbar' = -kbar, nbar' = -nbar.
    Rotating (t1, t2) by theta about n and re-expressing P in the new frame
    changes none of V, A, kbar, nbar."""
    fr, co = I.paraboloid_cells(seed=32, m=64)
    o = oracle.paraboloid_cells(fr, co)
    frc = np.concatenate([fr[:, 3:6], fr[:, 0:3], -fr[:, 6:9]], 1)
    coc = -co[:, [0, 2, 1, 5, 4, 3]]
    oc = oracle.paraboloid_cells(frc, coc)
    assert np.max(np.abs(o["alpha"] + oc["alpha"] - 1.0)) <= 1e-12
    assert np.max(np.abs(o["area"] - oc["area"])) <= 1e-12
    hit = o["status"] == 0
    assert np.array_equal(hit, oc["status"] == 0)
    assert np.max(np.abs(o["kbar"][hit] + oc["kbar"][hit])) <= 1e-11
    assert np.max(np.abs(o["nbar"][hit] + oc["nbar"][hit])) <= 1e-11
    # rotation: x = c x' - s y', y = s x' + c y'; new coefficients by a fit at six points
    th = 0.7
    cs, sn = np.cos(th), np.sin(th)
    frr = np.concatenate([cs * fr[:, 0:3] + sn * fr[:, 3:6], -sn * fr[:, 0:3] + cs * fr[:, 3:6], fr[:, 6:9]], 1)
    pts = np.array([[0, 0], [1, 0], [0, 1], [1, 1], [-1, 0.5], [0.5, -1]], float)
    B = np.stack([np.ones(6), pts[:, 0], pts[:, 1], pts[:, 0] ** 2, pts[:, 0] * pts[:, 1], pts[:, 1] ** 2], 1)
    x = cs * pts[:, 0] - sn * pts[:, 1]
    y = sn * pts[:, 0] + cs * pts[:, 1]
    Bxy = np.stack([np.ones(6), x, y, x * x, x * y, y * y], 1)
    cor = np.linalg.solve(B, Bxy @ co.T).T
    orr = oracle.paraboloid_cells(frr, cor)
    assert np.max(np.abs(orr["alpha"] - o["alpha"])) <= 1e-12
    assert np.max(np.abs(orr["area"] - o["area"])) <= 1e-12
    assert np.max(np.abs(orr["kbar"][hit] - o["kbar"][hit])) <= 1e-11
    assert np.max(np.abs(orr["nbar"][hit] - o["nbar"][hit])) <= 1e-11


def test_vector_area_closes_the_region_below():
    """The boundary of {X in cell : below the surface} has zero vector area, so
    int_S n dA = -sum over faces of nu_f |face part below| (brute force on a
    600 x 600 midpoint grid per face; sign and direction of nbar and the area
    scale)."""
    fr, co = I.paraboloid_cells(seed=33, m=8)
    o = oracle.paraboloid_cells(fr, co)
    g = (np.arange(600) + 0.5) / 600 - 0.5
    U, V = np.meshgrid(g, g, indexing="ij")
    for c in range(8):
        if o["status"][c]:
            continue
        t1, t2, n = fr[c].reshape(3, 3)
        a = co[c]
        N = np.zeros(3)
        for d in range(3):
            p, q = (d + 1) % 3, (d + 2) % 3
            for s in (-0.5, 0.5):
                X = np.zeros((3,) + U.shape)
                X[d], X[p], X[q] = s, U, V
                x, y, z = (np.tensordot(t, X, 1) for t in (t1, t2, n))
                below = a[0] + a[1] * x + a[2] * y + a[3] * x * x + a[4] * x * y + a[5] * y * y - z > 0
                N[d] -= np.sign(s) * below.mean()
        # |int n dA| <= A, with equality only for a plane
        Nv = o["nbar"][c] * np.linalg.norm(N)
        assert np.max(np.abs(Nv - N)) <= 4e-3
        assert np.linalg.norm(N) <= o["area"][c] + 4e-3


def test_surface_missing_the_cell():
    fr = _frames(34, 4)
    co = np.array([[2.0, 0, 0, 0.1, 0, 0.1], [-2.0, 0, 0, 0.1, 0, 0.1], [3.0, 0.1, 0, 0, 0, 0],
                   [-3.0, 0, 0.1, 0, 0, 0]])
    o = oracle.paraboloid_cells(fr, co)
    assert np.array_equal(o["alpha"], [1.0, 0.0, 1.0, 0.0])
    assert np.all(o["area"] == 0.0) and np.all(o["status"] == 1)
    # the point values at the origin: kappa of z = 0.1 (x^2 + y^2) is -0.4
    assert abs(o["kbar"][0] + 0.4) <= 1e-15


def test_volume_grows_with_the_height():
    fr, co = I.paraboloid_cells(seed=35, m=12)
    prev = None
    for h in np.linspace(-1.2, 1.2, 9):
        c2 = co.copy()
        c2[:, 0] = h
        v = oracle.paraboloid_cells(fr, c2)["alpha"]
        if prev is not None:
            assert np.all(v >= prev - 1e-15)
        prev = v


def test_paraboloid_alpha_of_a_fitted_droplet_is_close_to_the_exact_alpha():
    """On the fitted droplet the paraboloid alpha differs from the exact alpha
    only by the fit error (a sign error or a swapped side would be O(1))."""
    w = I.laplace_droplet_32(1)
    g = w["grid"]
    a, _ = oracle.alpha(w["verts"], w["tris"], g)
    cells, _ = oracle.interfacial_cells(w["verts"], w["tris"], g)
    k, n, co, st, fr = oracle.ppic(w["verts"], w["tris"], g, cells, frame=True)
    o = oracle.paraboloid_cells(fr, co)
    d = o["alpha"] - a.reshape(-1)[cells]
    assert np.max(np.abs(d)) < 0.02 and np.mean(np.abs(d)) < 2e-3
    # the surface-averaged curvature of a sphere of radius R is close to 2/R
    hit = o["status"] == 0
    kb = o["kbar"][hit] / g.h
    assert abs(np.median(kb) * w["R"] / 2.0 - 1.0) < 0.02


def test_surfaces_lying_in_cube_faces_and_diagonal_planes():
    """Planes in the cube's faces (area 1, alpha 1 or 0 up to the face itself)
    and through two opposite edges (area sqrt 2, alpha 1/2): the domain of the
    surface integral is bounded there by a coordinate that does not depend on
    x, a degenerate case of its breakpoints."""
    E = np.eye(3).reshape(9)
    co = np.array([[0.5, 0, 0, 0, 0, 0], [-0.5, 0, 0, 0, 0, 0], [0.0, 1.0, 0, 0, 0, 0], [0.0, 0, 1.0, 0, 0, 0]])
    o = oracle.paraboloid_cells(np.tile(E, (4, 1)), co)
    assert np.max(np.abs(o["area"] - [1.0, 1.0, np.sqrt(2.0), np.sqrt(2.0)])) <= 1e-14
    assert np.max(np.abs(o["alpha"] - [1.0, 0.0, 0.5, 0.5])) <= 1e-15
