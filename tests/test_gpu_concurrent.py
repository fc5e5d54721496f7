"""After front_bin (or front_bin_batch) a workspace may serve the volume
fraction and the PPIC fit on two streams at once: the two steps read the binned
fragments and write disjoint outputs, and the CSF force waits for both.  The
results must equal, bit for bit, those of the five calls in order."""
import numpy as np
import pytest
import torch

from paper_2505_06932_gb300 import _front as F
from paper_2505_06932_gb300 import inputs as I

pytestmark = pytest.mark.gpu

DEV = torch.device("cuda", 0)
FIELDS = ("alpha", "cell_keys", "kappa", "normal", "coeffs", "fit_status", "force")


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


def _fronts():
    return [I.small_sphere(4, 0.22, 48, seed=8, noise_h=1e-3),
            I.sh_droplet_256(seed=9, s=4, N=40),
            I.small_sphere(3, 0.3, 36, seed=4, noise_h=1e-3)]


def _one(w, precision, forked, reps=1):
    prm = F.make_params(precision=precision)
    verts, tris = _dev(w["verts"]), _dev(w["tris"])
    fc = F.FrontCoupling(w["grid"], tris.shape[0], verts.shape[0], params=prm)
    s0, s1 = torch.cuda.Stream(device=DEV), torch.cuda.Stream(device=DEV)
    s0.wait_stream(torch.cuda.current_stream())
    for _ in range(reps):
        with torch.cuda.stream(s0):
            F.front_bin(fc.ws, verts, tris, prm)
        if forked:
            s1.wait_stream(s0)
            with torch.cuda.stream(s1):
                F.front_volume_fraction(fc.ws, fc.alpha)
            with torch.cuda.stream(s0):
                F.front_curvature_ppic(fc.ws, prm, fc.cell_keys, fc.kappa, fc.normal, fc.coeffs, fc.fit_status)
            s0.wait_stream(s1)
        else:
            with torch.cuda.stream(s0):
                F.front_volume_fraction(fc.ws, fc.alpha)
                F.front_curvature_ppic(fc.ws, prm, fc.cell_keys, fc.kappa, fc.normal, fc.coeffs, fc.fit_status)
        with torch.cuda.stream(s0):
            F.front_csf_force(fc.ws, prm, fc.alpha, fc.kappa, fc.normal, fc.force)
    torch.cuda.current_stream().wait_stream(s0)
    torch.cuda.synchronize()
    res = fc.results(verts.shape[0])
    fc.ws.close()
    return res


@pytest.mark.parametrize("precision", [F.FT_FP32C, F.FT_FP64])
def test_alpha_beside_ppic_one_front(precision):
    for w in _fronts():
        ref = _one(w, precision, forked=False)
        got = _one(w, precision, forked=True, reps=3)
        assert got["status"] == ref["status"] == 0
        for k in FIELDS:
            np.testing.assert_array_equal(got[k], ref[k], err_msg=k)


def test_alpha_beside_ppic_batch():
    ws = _fronts()
    prm = F.make_params(precision=F.FT_FP32C)
    def fronts():  # each coupling keeps its own output arrays in its front dicts
        return [dict(grid=w["grid"], verts=_dev(w["verts"]), tris=_dev(w["tris"])) for w in ws]

    ref = F.BatchCoupling(fronts(), params=prm)
    ref.step(interp=False)
    torch.cuda.synchronize()
    bc = F.BatchCoupling(fronts(), params=prm)
    s0, s1 = torch.cuda.Stream(device=DEV), torch.cuda.Stream(device=DEV)
    s0.wait_stream(torch.cuda.current_stream())
    for _ in range(3):
        with torch.cuda.stream(s0):
            F.front_bin_batch(bc.ws, prm, s0)
        s1.wait_stream(s0)
        with torch.cuda.stream(s1):
            F.front_volume_fraction_batch(bc.ws, s1)
        with torch.cuda.stream(s0):
            F.front_curvature_ppic(bc.ws, prm, bc.cell_keys, bc.kappa, bc.normal, bc.coeffs, bc.fit_status, s0)
        s0.wait_stream(s1)
        with torch.cuda.stream(s0):
            F.front_csf_force_batch(bc.ws, prm, bc.kappa, bc.normal, s0)
            F.ft_batch_cell_ranges(bc.ws, bc.off, s0)
    torch.cuda.current_stream().wait_stream(s0)
    torch.cuda.synchronize()
    for b in range(len(ws)):
        r, g = ref.results(b), bc.results(b)
        for k in FIELDS:
            np.testing.assert_array_equal(g[k], r[k], err_msg=f"front {b} {k}")
