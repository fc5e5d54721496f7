"""Front advection (one RK4 step in the interpolated velocity, Sec. 3.1): the
CUDA path against the FP64 oracle, in place and out of place, one front and a
batch of fronts."""
import numpy as np
import pytest
import torch

import oracle
from paper_2505_06932_gb300 import _front as F
from paper_2505_06932_gb300 import inputs as I

pytestmark = pytest.mark.gpu

DEV = torch.device("cuda", 0)


def _cases():
    return [I.laplace_droplet_32(1), I.sh_droplet_256(seed=9, s=4, N=40),
            I.small_sphere(3, 0.3, 36, seed=4, noise_h=1e-3)]


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


def _tol(w, dt):
    umax = max(np.abs(f).max() for f in w["faces"])
    return 1e-12 * dt * umax + 4e-16 * np.abs(w["verts"]).max(), 1e-12 * umax


@pytest.mark.parametrize("case", [0, 1, 2])
def test_advect_matches_oracle(case):
    w = _cases()[case]
    g = w["grid"]
    dt = 0.25 * g.h / max(np.abs(f).max() for f in w["faces"])
    x = _dev(w["verts"])
    fa = [_dev(f) for f in w["faces"]]
    out = torch.empty_like(x)
    vel = torch.empty_like(x)
    F.front_advect_rk4(g, fa[0], fa[1], fa[2], x, dt, out, vel)
    xo, vo = oracle.advect_rk4(g, w["faces"], w["verts"], dt)
    tx, tv = _tol(w, dt)
    assert np.max(np.abs(out.cpu().numpy() - xo)) <= tx
    assert np.max(np.abs(vel.cpu().numpy() - vo)) <= tv
    # in place: the same positions
    F.front_advect_rk4(g, fa[0], fa[1], fa[2], x, dt, x)
    assert torch.equal(x, out)


def test_advect_batch_equals_one_front():
    ws = _cases()
    dt = [0.25 * w["grid"].h / max(np.abs(f).max() for f in w["faces"]) for w in ws]
    fronts = []
    for w, dts in zip(ws, dt):
        d = dict(grid=w["grid"], verts=_dev(w["verts"]), tris=_dev(w["tris"]))
        d["U"], d["V"], d["W"] = (_dev(f) for f in w["faces"])
        d["vel"] = torch.empty_like(d["verts"])
        d["verts_next"] = torch.empty_like(d["verts"])
        d["dt"] = dts
        fronts.append(d)
    nc = sum(w["grid"].ncells for w in ws)
    nt = sum(w["tris"].shape[0] for w in ws)
    bw = F.BatchWorkspace(len(ws), nc, nt)
    bw.set_fronts(fronts)
    F.front_advect_rk4_batch(bw)
    torch.cuda.synchronize()
    for w, d, dts in zip(ws, fronts, dt):
        out = torch.empty_like(d["verts"])
        vel = torch.empty_like(d["verts"])
        F.front_advect_rk4(w["grid"], d["U"], d["V"], d["W"], d["verts"], dts, out, vel)
        assert torch.equal(out, d["verts_next"])
        assert torch.equal(vel, d["vel"])
        xo, _ = oracle.advect_rk4(w["grid"], w["faces"], w["verts"], dts)
        tx, _ = _tol(w, dts)
        assert np.max(np.abs(d["verts_next"].cpu().numpy() - xo)) <= tx
    bw.close()
