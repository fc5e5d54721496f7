"""front_interp_velocity with the face velocities left in page-locked host
memory (read in place by the kernel) gives, bit for bit, what it gives with
the faces copied to the device; and the binding refuses pageable host arrays."""
import numpy as np
import pytest
import torch

from paper_2505_06932_gb300 import _front as F
from paper_2505_06932_gb300 import inputs as I


@pytest.mark.gpu
@pytest.mark.parametrize("make", [lambda: I.rough_sphere_128(2), lambda: I.laplace_droplet_32(1)],
                         ids=["rough_sphere_128", "droplet_32"])
def test_faces_in_pinned_host_memory_equal_device_faces(make):
    w = make()
    dev = torch.device("cuda", 0)
    v = torch.from_numpy(w["verts"]).to(dev)
    fd = [torch.from_numpy(f).to(dev) for f in w["faces"]]
    fh = [torch.from_numpy(f).pin_memory() for f in w["faces"]]
    a = torch.empty((v.shape[0], 3), dtype=torch.float64, device=dev)
    b = torch.full((v.shape[0], 3), float("nan"), dtype=torch.float64, device=dev)
    F.front_interp_velocity(w["grid"], fd[0], fd[1], fd[2], v, a)
    s = torch.cuda.Stream(device=dev)
    with torch.cuda.stream(s):
        F.front_interp_velocity(w["grid"], fh[0], fh[1], fh[2], v, b)
    torch.cuda.synchronize()
    assert torch.equal(a.view(torch.int64), b.view(torch.int64))
    # also inside a captured graph, replayed after the host field changed
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        F.front_interp_velocity(w["grid"], fh[0], fh[1], fh[2], v, b)
    for f in fh:
        f.mul_(-2.0)
    g.replay()
    for f in fd:
        f.mul_(-2.0)
    F.front_interp_velocity(w["grid"], fd[0], fd[1], fd[2], v, a)
    torch.cuda.synchronize()
    assert torch.equal(a.view(torch.int64), b.view(torch.int64))


def test_pageable_host_faces_are_refused():
    w = I.laplace_droplet_32(1)
    fh = [torch.from_numpy(f) for f in w["faces"]]  # pageable
    v = torch.from_numpy(w["verts"])
    with pytest.raises(F.FrontError):
        F._ptr_faces(fh[0], "U")
    assert not fh[0].is_pinned()
    assert v.shape[1] == 3
