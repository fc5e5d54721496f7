"""Pins of the oracle's front advection: one classical fourth-order Runge-Kutta
step of dx/dt = u(x) in the interpolated velocity (Sec. 3.1).

The divergence-preserving interpolation reproduces linear fields exactly, and
RK4 applied to the linear system dx/dt = A (x - c) is exactly the degree-4
Taylor polynomial P(dt A) = I + dt A + (dt A)^2/2 + (dt A)^3/6 + (dt A)^4/24 of
the flow map.  So for a uniform or solid-body field the result has a closed form
computed here with plain matrix arithmetic, and the volume enclosed by a front
scales by det P(dt A) per step."""
import numpy as np

import oracle
from paper_2505_06932_gb300 import inputs as I


def _cross_matrix(w):
    return np.array([[0.0, -w[2], w[1]], [w[2], 0.0, -w[0]], [-w[1], w[0], 0.0]])


def _taylor4(M):
    E = np.eye(3)
    P = np.eye(3)
    for k in range(1, 5):
        E = E @ M / k
        P = P + E
    return P


def test_rk4_uniform_field_translates():
    g = I.unit_grid(24)
    u = np.array([0.3, -0.7, 1.1])
    faces = tuple(np.full(tuple(g.n[d] + (1 if d == a else 0) for d in range(3)), u[a]) for a in range(3))
    pts = I.rng(1).uniform(0.2, 0.8, size=(500, 3))
    dt = 0.25 * g.h
    out, vel = oracle.advect_rk4(g, faces, pts, dt)
    assert np.max(np.abs(out - (pts + dt * u))) <= 1e-15
    assert np.max(np.abs(vel - u)) <= 1e-14


def test_rk4_solid_body_is_the_taylor_polynomial_of_the_flow():
    g = I.unit_grid(32)
    gen = I.rng(4)
    c = 0.5 + gen.uniform(0, g.h, 3)
    w = gen.normal(size=3)
    w *= 3.0 / np.linalg.norm(w)
    faces = I.solid_body_faces_exact(g, c, w)
    pts = c + gen.uniform(-0.3, 0.3, size=(2000, 3))
    for dt in (0.25 * g.h, 0.1, 0.3):
        out, vel = oracle.advect_rk4(g, faces, pts, dt)
        P = _taylor4(dt * _cross_matrix(w))
        expect = c + (pts - c) @ P.T
        assert np.max(np.abs(out - expect)) <= 1e-13, dt
        assert np.max(np.abs(vel - np.cross(w, pts - c))) <= 1e-13


def test_rk4_volume_factor_of_a_rotation():
    """det P(dt A) = |P(i theta)|^2 with theta = |w| dt (the rotation axis keeps
    its length); a closed front's enclosed volume follows it step by step."""
    g = I.unit_grid(32)
    c = np.array([0.5, 0.5, 0.5])
    w = np.array([0.0, 2.0, 1.0])
    faces = I.solid_body_faces_exact(g, c, w)
    v, t = I.sphere_front(3, 0.25, c + 0.3 * g.h)
    dt = 0.2
    theta = np.linalg.norm(w) * dt
    z = 1j * theta
    p = 1 + z + z ** 2 / 2 + z ** 3 / 6 + z ** 4 / 24
    v0 = oracle.signed_volume(v, t)
    x = v
    for n in range(1, 13):
        x, _ = oracle.advect_rk4(g, faces, x, dt)
        assert abs(oracle.signed_volume(x, t) / v0 - abs(p) ** (2 * n)) <= 1e-12, n
    # and the factor is not 1: the pin sees a dropped stage
    assert abs(abs(p) ** 24 - 1.0) > 1e-4


def test_rk4_velocity_is_the_interpolation_at_the_start():
    w = I.laplace_droplet_32(1)
    g = w["grid"]
    out, vel = oracle.advect_rk4(g, w["faces"], w["verts"], 0.25 * g.h)
    assert np.array_equal(vel, oracle.interp(g, w["faces"], w["verts"]))
    # moved by about dt |u| (|u| <= |w| r ~ 0.25)
    assert 0.0 < np.max(np.linalg.norm(out - w["verts"], axis=1)) < 0.25 * g.h * 0.3
