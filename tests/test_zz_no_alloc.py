"""The allocation-free volume fraction (ft_volume_fraction_noalloc) is for
callers that cannot allocate device memory while they run: a flow solver that
owns all GPU memory through its own pool, a process under a hard memory cap, or
a time loop that cannot take cudaMalloc's implicit synchronization.  It must
give the same alpha as the allocating path (front_bin + front_volume_fraction)
and as the FP64 oracle on two calls in a row, and must flag, not overrun, a
front whose candidate pairs exceed its fixed scratch.  Collected last on
purpose: its scratch is one array shared by the whole process."""
import numpy as np
import pytest
import torch

import oracle
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


def _alpha_noalloc(w, prm, dev):
    v = torch.from_numpy(w["verts"]).to(dev)
    t = torch.from_numpy(w["tris"]).to(dev)
    a = torch.full((w["grid"].ncells,), -7.0, dtype=torch.float64, device=dev)
    st = torch.zeros(1, dtype=torch.int32, device=dev)
    F.ft_volume_fraction_noalloc(w["grid"], v, t, prm, a, st)
    torch.cuda.synchronize()
    return a.cpu().numpy(), int(st.item())


def _check_small(w, prm, dev):
    got, st = _alpha_noalloc(w, prm, dev)
    assert st == 0
    want, st2 = _alpha_existing(w, F.make_params(), dev)
    assert st2 == 0
    assert np.max(np.abs(got - want)) <= 1e-12
    full_or_empty = (want == 0.0) | (want == 1.0)
    assert np.array_equal(got[full_or_empty], want[full_or_empty])
    orc, st3 = oracle.alpha(w["verts"], w["tris"], w["grid"])
    assert st3 == 0
    assert np.max(np.abs(got - orc.reshape(-1))) <= 1e-12


@pytest.mark.parametrize("precision", [F.FT_FP64, F.FT_FP32C], ids=["fp64", "fp32c_request"])
def test_noalloc_alpha_matches_allocating_path_and_oracle_twice(precision):
    """Two calls in a row on different fronts and grids; a request for the FP32
    form still computes the float64 path (the scratch holds float64 records)."""
    dev = torch.device("cuda", 0)
    prm = F.make_params(precision=precision)
    for w in (I.laplace_droplet_32(1), I.sh_droplet_256(seed=9, s=4, N=40)):
        _check_small(w, prm, dev)


def test_noalloc_candidate_overflow_flagged_then_next_call_exact():
    """A front under the triangle and grid limits whose candidate pairs exceed
    FT_NOALLOC_MAX_CANDIDATES: the call sets FT_ST_CAPACITY on the device (and
    writes nothing past its scratch); the following small call is exact."""
    dev = torch.device("cuda", 0)
    prm = F.make_params()
    big = I.small_sphere(4, 0.3, 64, seed=3)  # 5,120 triangles on 64^3: about 45 k candidates
    assert big["tris"].shape[0] <= 16384 and big["grid"].ncells <= 262144
    _, st = _alpha_noalloc(big, prm, dev)
    assert st & 0x01
    _check_small(I.laplace_droplet_32(2), prm, dev)


def test_noalloc_rejects_sizes_beyond_its_scratch():
    dev = torch.device("cuda", 0)
    w = I.rough_sphere_128(2)  # 128^3 cells and 81,920 triangles exceed the static limits
    v = torch.from_numpy(w["verts"]).to(dev)
    t = torch.from_numpy(w["tris"]).to(dev)
    a = torch.empty(w["grid"].ncells, dtype=torch.float64, device=dev)
    st = torch.zeros(1, dtype=torch.int32, device=dev)
    with pytest.raises(F.FrontError, match="capacity"):
        F.ft_volume_fraction_noalloc(w["grid"], v, t, F.make_params(), a, st)
