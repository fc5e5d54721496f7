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
