"""Compact outputs for callers that move results off the device: the CSF force
at the interfacial and ring cells only (front_csf_force_compact) and alpha as
one bit per cell plus the interfacial values (front_alpha_pack) must carry
exactly the dense outputs' information, bit for bit."""
import numpy as np
import pytest
import torch

from paper_2505_06932_gb300 import _front as F
from paper_2505_06932_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("make,precision", [(lambda: I.laplace_droplet_32(1), F.FT_FP64),
                                            (lambda: I.rough_sphere_128(2), F.FT_FP32C),
                                            (lambda: I.sh_droplet_256(seed=9, s=4, N=40), F.FT_FP64)],
                         ids=["droplet_32", "rough_sphere_128_fp32c", "sh_droplet_40"])
def test_compact_outputs_equal_the_dense_ones(make, precision):
    w = make()
    dev = torch.device("cuda", 0)
    v = torch.from_numpy(w["verts"]).to(dev)
    t = torch.from_numpy(w["tris"]).to(dev)
    fa = [torch.from_numpy(f).to(dev) for f in w["faces"]]
    prm = F.make_params(precision=precision)
    fc = F.FrontCoupling(w["grid"], t.shape[0], v.shape[0], params=prm)
    fc.step(v, t, fa)
    M = fc.ws.counts()["M"]
    N = w["grid"].ncells
    cap = 8 * M
    keys = torch.empty(cap, dtype=torch.int32, device=dev)
    force = torch.empty((cap, 3), dtype=torch.float64, device=dev)
    count = torch.zeros(1, dtype=torch.int64, device=dev)
    F.front_csf_force_compact(fc.ws, prm, fc.alpha, fc.kappa, fc.normal, keys, force, count)
    bits = torch.empty((N + 31) // 32, dtype=torch.int32, device=dev)
    acells = torch.empty(M, dtype=torch.float64, device=dev)
    F.front_alpha_pack(fc.ws, fc.alpha, bits, acells)
    torch.cuda.synchronize()
    assert fc.ws.status() == 0
    n = int(count.item())
    k = keys[:n].cpu().numpy().view(np.uint32).astype(np.int64)
    fcomp = force[:n].cpu().numpy()
    dense = fc.force.view(3, N).cpu().numpy()
    cells = fc.cell_keys[:M].cpu().numpy().view(np.uint32).astype(np.int64)
    assert np.array_equal(k[:M], cells)
    assert len(np.unique(k)) == n
    # scattered back, the compact force is the dense one bit for bit
    back = np.zeros_like(dense)
    back[:, k] = fcomp.T
    assert np.array_equal(back.view(np.int64), dense.view(np.int64))
    assert np.all(np.any(dense != 0.0, axis=0) <= np.isin(np.arange(N), k))
    # alpha: the bits and the interfacial values rebuild it bit for bit
    alpha = fc.alpha.cpu().numpy()
    b = bits.cpu().numpy().view(np.uint32)
    full = ((b[np.arange(N) // 32] >> (np.arange(N) % 32)) & 1).astype(np.float64)
    rebuilt = full.copy()
    rebuilt[cells] = acells.cpu().numpy()
    assert np.array_equal(rebuilt.view(np.int64), alpha.view(np.int64))
    # the compact force and alpha are far smaller than the dense arrays
    assert (n * 28 + (N // 32) * 4 + M * 8) * 10 < 32 * N
    fc.ws.close()


def test_compact_force_capacity_flagged():
    w = I.laplace_droplet_32(1)
    dev = torch.device("cuda", 0)
    v = torch.from_numpy(w["verts"]).to(dev)
    t = torch.from_numpy(w["tris"]).to(dev)
    fa = [torch.from_numpy(f).to(dev) for f in w["faces"]]
    prm = F.make_params()
    fc = F.FrontCoupling(w["grid"], t.shape[0], v.shape[0], params=prm)
    fc.step(v, t, fa)
    M = fc.ws.counts()["M"]
    keys = torch.full((M + 5,), -1, dtype=torch.int32, device=dev)
    force = torch.empty((M + 5, 3), dtype=torch.float64, device=dev)
    count = torch.zeros(1, dtype=torch.int64, device=dev)
    F.front_csf_force_compact(fc.ws, prm, fc.alpha, fc.kappa, fc.normal, keys, force, count)
    assert fc.ws.status() & 0x01
    assert int(count.item()) > M + 5
    assert np.array_equal(keys[:M].cpu().numpy().view(np.uint32), fc.cell_keys[:M].cpu().numpy().view(np.uint32))
    fc.ws.close()


@pytest.mark.parametrize("precision", [F.FT_FP64, F.FT_FP32C], ids=["fp64", "fp32c"])
def test_split_force_equals_front_csf_force(precision):
    """front_force_clear + front_csf_prepare + front_csf_force_cells (the clear
    on a side stream forked before the binning, alpha and the ring list on
    another beside the fit, both joined before the force, as the bench's graph
    step runs them, also captured in a CUDA graph) give front_csf_force's array
    bit for bit, whatever the array held before; the cells call without a ring
    list for the current binning is a call-order error."""
    w = I.rough_sphere_128(2)
    dev = torch.device("cuda", 0)
    v = torch.from_numpy(w["verts"]).to(dev)
    t = torch.from_numpy(w["tris"]).to(dev)
    fa = [torch.from_numpy(f).to(dev) for f in w["faces"]]
    prm = F.make_params(precision=precision)
    fc = F.FrontCoupling(w["grid"], t.shape[0], v.shape[0], params=prm)
    fc.step(v, t, fa)
    torch.cuda.synchronize()
    assert fc.ws.status() == 0
    ref = fc.force.clone()
    side, side2 = torch.cuda.Stream(device=dev), torch.cuda.Stream(device=dev)

    def split():
        cs = torch.cuda.current_stream()
        side.wait_stream(cs)
        with torch.cuda.stream(side):
            F.front_force_clear(fc.ws, fc.force)
        F.front_bin(fc.ws, v, t, prm)
        side2.wait_stream(cs)
        with torch.cuda.stream(side2):
            F.front_volume_fraction(fc.ws, fc.alpha)
            F.front_csf_prepare(fc.ws)  # beside the fit
        F.front_curvature_ppic(fc.ws, prm, fc.cell_keys, fc.kappa, fc.normal, fc.coeffs, fc.fit_status)
        cs.wait_stream(side)
        cs.wait_stream(side2)
        F.front_csf_force_cells(fc.ws, prm, fc.alpha, fc.kappa, fc.normal, fc.force)

    fc.force.fill_(float("nan"))
    split()
    torch.cuda.synchronize()
    assert torch.equal(fc.force.view(torch.int64), ref.view(torch.int64))
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        split()
    fc.force.fill_(-7.0)
    g.replay()
    torch.cuda.synchronize()
    assert fc.ws.status() == 0
    assert torch.equal(fc.force.view(torch.int64), ref.view(torch.int64))
    # a new binning makes the ring list stale: the cells call is refused until
    # front_csf_prepare lists it again
    F.front_bin(fc.ws, v, t, prm)
    with pytest.raises(F.FrontError):
        F.front_csf_force_cells(fc.ws, prm, fc.alpha, fc.kappa, fc.normal, fc.force)
    F.front_curvature_ppic(fc.ws, prm, fc.cell_keys, fc.kappa, fc.normal, fc.coeffs, fc.fit_status)
    F.front_csf_prepare(fc.ws)
    # the cells call alone leaves every cell where the force is zero as it was
    fc.force.fill_(3.0)
    F.front_csf_force_cells(fc.ws, prm, fc.alpha, fc.kappa, fc.normal, fc.force)
    torch.cuda.synchronize()
    nz = (ref.view(3, -1) != 0).any(dim=0)
    got = fc.force.view(3, -1)
    assert torch.equal(got[:, nz].view(torch.int64), ref.view(3, -1)[:, nz].view(torch.int64))
    assert int((got[:, ~nz] == 3.0).all(dim=0).sum()) >= int((~nz).sum()) - 8 * fc.ws.counts()["M"]
    fc.ws.close()


def test_split_force_batch_equals_front_csf_force_batch():
    dev = torch.device("cuda", 0)
    wl = [I.laplace_droplet_32(1), I.small_sphere(3, 0.3, 36, seed=4, noise_h=1e-3),
          I.small_sphere(2, 0.12, 24, seed=6)]
    fr = []
    for w in wl:
        fr.append(dict(grid=w["grid"], verts=torch.from_numpy(w["verts"]).to(dev),
                       tris=torch.from_numpy(w["tris"]).to(dev)))
    prm = F.make_params(precision=F.FT_FP32C)
    bc = F.BatchCoupling(fr, params=prm)
    bc.step()
    torch.cuda.synchronize()
    assert bc.ws.status() == 0
    ref = [f["force"].clone() for f in bc.fronts]
    for f in bc.fronts:
        f["force"].fill_(float("nan"))
    side = torch.cuda.Stream(device=dev)
    cs = torch.cuda.current_stream()
    side.wait_stream(cs)
    with torch.cuda.stream(side):
        F.front_force_clear_batch(bc.ws)
    F.front_bin_batch(bc.ws, prm)
    F.front_volume_fraction_batch(bc.ws)
    F.front_csf_prepare(bc.ws)
    F.front_curvature_ppic(bc.ws, prm, bc.cell_keys, bc.kappa, bc.normal, bc.coeffs, bc.fit_status)
    cs.wait_stream(side)
    F.front_csf_force_cells_batch(bc.ws, prm, bc.kappa, bc.normal)
    torch.cuda.synchronize()
    assert bc.ws.status() == 0
    for f, r in zip(bc.fronts, ref):
        assert torch.equal(f["force"].view(torch.int64), r.view(torch.int64))
    # a one-front call on a batch workspace is an argument error (FT_ERR_ARG)
    assert F.lib().front_force_clear(bc.ws.handle, bc.fronts[0]["force"].data_ptr(), None) == -1
    bc.ws.close()
