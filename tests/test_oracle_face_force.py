"""Pins of the oracle's balanced-force face term (Sec. 3.3, Eq. mwi_disc):
S_f = sigma kbar_f (alpha_Q - alpha_P)/h on every face, kbar_f the mean of the
two cells' curvatures (own kappa in interfacial cells, the smoothed kbar of
Sec. 3.3 elsewhere)."""
import numpy as np

import oracle
from paper_2505_06932_gb300 import inputs as I


def _droplet():
    w = I.laplace_droplet_32(1)
    g = w["grid"]
    a, _ = oracle.alpha(w["verts"], w["tris"], g)
    cells, _ = oracle.interfacial_cells(w["verts"], w["tris"], g)
    k, n, _, _ = oracle.ppic(w["verts"], w["tris"], g, cells)
    return w, g, a, cells, k, n


def test_constant_curvature_telescopes_along_grid_lines():
    """With kappa constant the face terms of each grid line sum to
    sigma kappa (alpha_out - alpha_out)/h = 0."""
    w, g, a, cells, k, n = _droplet()
    F = oracle.face_force(g, a, cells, np.full_like(k, 4.0), n, sigma=0.7)
    for d in range(3):
        s = F[d].sum(axis=d)
        assert np.max(np.abs(s)) <= 1e-13 * np.abs(F[d]).max()
    assert max(np.abs(f).max() for f in F) > 0.0


def test_constant_curvature_field_is_curl_free():
    """With kappa constant the face field is sigma kappa times the discrete
    gradient of alpha, so its circulation around every cell edge vanishes."""
    w, g, a, cells, k, n = _droplet()
    Fx, Fy, Fz = oracle.face_force(g, a, cells, np.full_like(k, 4.0), n)
    # Fx[i, j, k] lies between cells i-1 and i; around the edge at x_i, y_j:
    # Fx(i, j) - Fx(i, j-1) - Fy(i, j) + Fy(i-1, j) = 0
    c = Fx[1:-1, 1:, :] - Fx[1:-1, :-1, :] - Fy[1:, 1:-1, :] + Fy[:-1, 1:-1, :]
    assert np.max(np.abs(c)) <= 1e-13 * np.abs(Fx).max()
    c = Fy[:, 1:-1, 1:] - Fy[:, 1:-1, :-1] - Fz[:, 1:, 1:-1] + Fz[:, :-1, 1:-1]
    assert np.max(np.abs(c)) <= 1e-13 * np.abs(Fy).max()


def test_cell_average_of_faces_is_the_csf_force_for_constant_curvature():
    """(S_{i-1/2} + S_{i+1/2})/2 = sigma kappa (alpha_{i+1} - alpha_{i-1})/(2h),
    the CSF force of Eq. csf, wherever kappa is the constant."""
    w, g, a, cells, k, n = _droplet()
    kc = np.full_like(k, 2.5)
    F = oracle.face_force(g, a, cells, kc, n, sigma=1.3)
    S = oracle.csf(g, a, cells, kc, n, sigma=1.3)
    for d in range(3):
        lo = [slice(None)] * 3
        hi = [slice(None)] * 3
        lo[d] = slice(0, -1)
        hi[d] = slice(1, None)
        avg = 0.5 * (F[d][tuple(lo)] + F[d][tuple(hi)])
        # the CSF force is zero where the whole gradient vanishes; compare where it does not
        mask = np.any(S != 0.0, axis=0)
        assert np.max(np.abs(avg[mask] - S[d][mask])) <= 1e-13 * np.abs(S[d]).max()


def test_face_force_points_inward_on_a_sphere():
    w, g, a, cells, k, n = _droplet()
    F = oracle.face_force(g, a, cells, k, n)
    c = w["centre"]
    nz = 0
    for d in range(3):
        idx = np.nonzero(F[d])
        x = [(np.asarray(idx[e]) + (0.0 if e == d else 0.5)) * g.h - c[e] for e in range(3)]
        assert np.all(F[d][idx] * x[d] < 0.0)
        nz += len(idx[0])
    assert nz > 100


def test_face_force_is_local_to_the_interface():
    """Only faces between cells of different alpha carry a force, and every one
    of them touches an interfacial cell or a neighbour of one."""
    w, g, a, cells, k, n = _droplet()
    F = oracle.face_force(g, a, cells, k, n)
    N = g.n[0]
    near = np.zeros((N, N, N), bool)
    ci = np.stack([cells // (N * N), (cells // N) % N, cells % N], 1)
    for di in (-1, 0, 1):
        for dj in (-1, 0, 1):
            for dk in (-1, 0, 1):
                near[tuple((ci + [di, dj, dk]).T)] = True
    for d in range(3):
        idx = np.array(np.nonzero(F[d]))
        q = idx.copy()
        p = idx.copy()
        p[d] -= 1
        ok = near[tuple(np.clip(q, 0, N - 1))] | near[tuple(np.clip(p, 0, N - 1))]
        assert np.all(ok)
