"""Pins of the oracle's CSF force (Eq. csf, Sec. 3.3) and of the divergence-
preserving velocity interpolation (Sec. 3.1)."""
import numpy as np
import pytest

import oracle
from paper_2505_06932_gb300 import inputs as I


def _droplet():
    w = I.laplace_droplet_32(1)
    g = w["grid"]
    a, _ = oracle.alpha(w["verts"], w["tris"], g)
    cells, _ = oracle.interfacial_cells(w["verts"], w["tris"], g)
    k, n, _, _ = oracle.ppic(w["verts"], w["tris"], g, cells)
    return w, g, a, cells, k, n


def test_csf_constant_curvature_sums_to_zero():
    """With kappa constant, sum_P S_P h^3 = sigma kappa sum_P grad alpha_P h^3 = 0
    (central differences telescope; alpha = 0 outside the domain)."""
    w, g, a, cells, k, n = _droplet()
    f = oracle.csf(g, a, cells, np.full_like(k, 3.0), n, sigma=0.7)
    tot = f.reshape(3, -1).sum(axis=1)
    assert np.max(np.abs(tot)) <= 1e-13 * np.abs(f).max() * np.count_nonzero(f[0])


def test_csf_points_inward_and_is_local():
    """On a sphere S = sigma kappa grad alpha points to the centre, and it is zero
    outside the interfacial cells and their 26 neighbours."""
    w, g, a, cells, k, n = _droplet()
    f = oracle.csf(g, a, cells, k, n, sigma=1.0)
    N = g.n[0]
    nz = np.nonzero(np.any(f.reshape(3, -1) != 0.0, axis=0))[0]
    ijk = np.stack([nz // (N * N), (nz // N) % N, nz % N], 1)
    x = (ijk + 0.5) * g.h - w["centre"]
    s = np.einsum("ij,ji->i", x, f.reshape(3, -1)[:, nz])
    assert np.all(s < 0.0)
    near = np.zeros((N, N, N), bool)
    ci = np.stack([cells // (N * N), (cells // N) % N, cells % N], 1)
    for d in np.array(np.meshgrid([-1, 0, 1], [-1, 0, 1], [-1, 0, 1], indexing="ij")).reshape(3, -1).T:
        q = ci + d
        near[q[:, 0], q[:, 1], q[:, 2]] = True
    assert np.all(near.reshape(-1)[nz])


def test_csf_smoothing_weights_example():
    """Sec. 3.3: kbar_P = sum kappa_Q w_Q / sum w_Q, w_Q = |s_Q . n_Q|/|s_Q|,
    on a hand-built neighbourhood of one non-interfacial cell."""
    g = I.unit_grid(5)
    a = np.zeros((5, 5, 5))
    a[1, 2, 2] = 1.0  # grad alpha at (2,2,2) = (-1/(2h), 0, 0)
    key = lambda i, j, k: (i * 5 + j) * 5 + k
    cells = np.array([key(3, 2, 2), key(2, 3, 3)], np.uint32)
    kap = np.array([2.0, 5.0])
    nrm = np.array([[1.0, 0.0, 0.0], [0.0, 1.0, 0.0]])
    f = oracle.csf(g, a, cells, kap, nrm, sigma=1.5)
    w1, w2 = 1.0, 1.0 / np.sqrt(2.0)
    kbar = (2.0 * w1 + 5.0 * w2) / (w1 + w2)
    assert abs(f[0, 2, 2, 2] - 1.5 * kbar * (-1.0 / (2 * g.h))) < 1e-12 * abs(f[0, 2, 2, 2])
    assert f[1, 2, 2, 2] == 0.0 and f[2, 2, 2, 2] == 0.0


def _random_faces(g, seed):
    gen = I.rng(seed)
    n0, n1, n2 = g.n
    return (gen.normal(size=(n0 + 1, n1, n2)), gen.normal(size=(n0, n1 + 1, n2)), gen.normal(size=(n0, n1, n2 + 1)))


def test_interp_reproduces_face_values():
    g = I.unit_grid(8)
    F = _random_faces(g, 3)
    pts, want = [], []
    for (i, j, k) in [(0, 3, 4), (3, 5, 1), (7, 2, 6), (8, 4, 4)]:
        # x-face (i, j, k): centre (X_i, y_j+1/2, z_k+1/2)
        pts.append([i * g.h, (j + 0.5) * g.h, (k + 0.5) * g.h])
        want.append(F[0][i, j, k])
    u = oracle.interp(g, F, np.array(pts))[:, 0]
    assert np.max(np.abs(u - np.array(want))) < 1e-13


def test_interp_preserves_discrete_divergence():
    """div u(x) inside a cell equals (dU + dV + dW)/h (Sec. 3.1); the interpolant
    is at most quadratic along each axis, so central differences are exact."""
    g = I.unit_grid(8)
    F = _random_faces(g, 4)
    gen = I.rng(5)
    h = g.h
    for _ in range(40):
        c = gen.integers(0, 8, 3)
        x = (c + gen.uniform(0.2, 0.8, 3)) * h
        s = 0.1 * h
        div = 0.0
        for d in range(3):
            e = np.eye(3)[d] * s
            up = oracle.interp(g, F, (x + e)[None])[0, d]
            dn = oracle.interp(g, F, (x - e)[None])[0, d]
            div += (up - dn) / (2 * s)
        i, j, k = c
        want = (F[0][i + 1, j, k] - F[0][i, j, k] + F[1][i, j + 1, k] - F[1][i, j, k]
                + F[2][i, j, k + 1] - F[2][i, j, k]) / h
        assert abs(div - want) < 1e-9 * max(1.0, abs(want))


def test_interp_exact_for_solid_body_rotation():
    """A linear divergence-free field is reproduced exactly everywhere."""
    g = I.unit_grid(16)
    gen = I.rng(6)
    c = np.array([0.5, 0.45, 0.55])
    F, w = I.solid_body_faces(g, c, gen, noise=0.0)
    pts = gen.uniform(0.0, 1.0, size=(500, 3))
    got = oracle.interp(g, F, pts)
    want = np.cross(np.broadcast_to(w, pts.shape), pts - c)
    assert np.max(np.abs(got - want)) < 1e-13


def test_interp_normal_component_continuous_across_faces():
    g = I.unit_grid(8)
    F = _random_faces(g, 7)
    gen = I.rng(8)
    for _ in range(20):
        x = gen.uniform(0.1, 0.9, 3)
        d = gen.integers(0, 3)
        x[d] = np.round(x[d] / g.h) * g.h
        e = np.eye(3)[d] * 1e-9 * g.h
        a = oracle.interp(g, F, (x - e)[None])[0, d]
        b = oracle.interp(g, F, (x + e)[None])[0, d]
        assert abs(a - b) < 1e-6
