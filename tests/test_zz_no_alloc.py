"""The allocation-free volume fraction (ft_volume_fraction_noalloc), for callers
that cannot allocate device memory while they run, must give the same alpha as
the allocating path (front_bin + front_volume_fraction) on two calls in a row.
Collected last on purpose: its scratch is shared process-wide."""
import numpy as np
import pytest
import torch

from paper_2505_06932_gb300 import _front as F
from paper_2505_06932_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def _alpha_existing(w, prm, dev):
    v = torch.from_numpy(w["verts"]).to(dev)
    t = torch.from_numpy(w["tris"]).to(dev)
    ws = F.Workspace(w["grid"], t.shape[0])
    a = torch.empty(w["grid"].ncells, dtype=torch.float64, device=dev)
    F.front_bin(ws, v, t, prm)
    F.front_volume_fraction(ws, a)
    st = ws.status()
    ws.close()
    return a.cpu().numpy(), st


def test_noalloc_alpha_matches_allocating_path_twice():
    dev = torch.device("cuda", 0)
    prm = F.make_params()
    fronts = [I.laplace_droplet_32(1), I.sh_droplet_256(seed=9, s=4, N=40)]
    for w in fronts:  # two calls in a row, different fronts and grids
        v = torch.from_numpy(w["verts"]).to(dev)
        t = torch.from_numpy(w["tris"]).to(dev)
        a = torch.full((w["grid"].ncells,), -7.0, dtype=torch.float64, device=dev)
        st = torch.zeros(1, dtype=torch.int32, device=dev)
        F.ft_volume_fraction_noalloc(w["grid"], v, t, prm, a, st)
        torch.cuda.synchronize()
        assert int(st.item()) == 0
        got = a.cpu().numpy()
        want, st2 = _alpha_existing(w, prm, dev)
        assert st2 == 0
        assert np.max(np.abs(got - want)) <= 1e-12
        assert np.array_equal(got[(want == 0.0) | (want == 1.0)], want[(want == 0.0) | (want == 1.0)])


def test_noalloc_rejects_sizes_beyond_its_scratch():
    dev = torch.device("cuda", 0)
    w = I.rough_sphere_128(2)  # 128^3 cells and 81,920 triangles exceed the static limits
    v = torch.from_numpy(w["verts"]).to(dev)
    t = torch.from_numpy(w["tris"]).to(dev)
    a = torch.empty(w["grid"].ncells, dtype=torch.float64, device=dev)
    st = torch.zeros(1, dtype=torch.int32, device=dev)
    with pytest.raises(F.FrontError, match="capacity"):
        F.ft_volume_fraction_noalloc(w["grid"], v, t, F.make_params(), a, st)
