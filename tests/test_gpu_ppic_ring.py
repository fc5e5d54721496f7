"""The paper's own PPIC neighbourhood and frame on the GPU (Sec. 3.2): whole
triangles of the k-ring around the front vertex closest to the cell centre,
that vertex's normal as the frame normal, against the oracle's fit in every
interfacial cell (kappa, normal, coefficients, fit status)."""
import numpy as np
import pytest

import oracle
from paper_2505_06932_gb300 import _front as F
from paper_2505_06932_gb300 import inputs as I
from gpucase import run_gpu, run_oracle

pytestmark = pytest.mark.gpu

VARIANTS = {
    "ring3_vertex": dict(fit_ring=3, frame_vertex=1),
    "ring2_vertex": dict(fit_ring=2, frame_vertex=1),
    "ring3_fragment_frame": dict(fit_ring=3, frame_vertex=0),
    "fragments_vertex_frame": dict(fit_ring=0, frame_vertex=1),
}

SHAPES = {
    "droplet_32": lambda: I.laplace_droplet_32(1),
    "sh_droplet_40": lambda: I.sh_droplet_256(seed=9, s=4, N=40),
}


def _gpu_params(v, precision=F.FT_FP64):
    return dict(fit_ring=v["fit_ring"], frame=F.FT_FRAME_VERTEX if v["frame_vertex"] else F.FT_FRAME_FRAGMENTS)


@pytest.mark.parametrize("shape", list(SHAPES))
@pytest.mark.parametrize("variant", list(VARIANTS))
def test_paper_neighbourhood_matches_oracle(shape, variant):
    w = SHAPES[shape]()
    v = VARIANTS[variant]
    gpu = run_gpu(w, params=_gpu_params(v))
    assert gpu["status"] == 0
    cells = np.unique(oracle.bin_pairs(w["verts"], w["tris"], w["grid"])[0])
    assert np.array_equal(gpu["cell_keys"], cells)
    k, n, a, st = oracle.ppic(w["verts"], w["tris"], w["grid"], cells, params=v)
    assert np.array_equal(gpu["fit_status"], st)
    ok = (st & 2) == 0   # singular systems (the 1-ring) fall back to a plane on both sides
    assert np.all(np.abs(gpu["kappa"] - k) <= 1e-9 * np.maximum(np.abs(k), 1.0))
    assert np.max(np.abs(gpu["normal"] - n)) <= 1e-9
    assert np.all(np.abs(gpu["coeffs"][ok] - a[ok]) <= 1e-9 * np.maximum(np.abs(a[ok]), 1.0))


def test_one_ring_fit():
    """The 1-ring (five or six triangles) never reaches fit_min = 24, so the
    support grows to delta_max in every cell; its 6x6 systems are nearly
    singular on a curved front, so the two sides agree on the cells they both
    solve only to the conditioning; on a flat face both give kappa = 0."""
    w = I.laplace_droplet_32(1)
    v = dict(fit_ring=1, frame_vertex=1)
    gpu = run_gpu(w, params=_gpu_params(v))
    cells = np.unique(oracle.bin_pairs(w["verts"], w["tris"], w["grid"])[0])
    k, n, a, st = oracle.ppic(w["verts"], w["tris"], w["grid"], cells, params=v)
    assert np.all(gpu["fit_status"] & 1) and np.all(st & 1)
    both = ((gpu["fit_status"] & 2) == 0) & ((st & 2) == 0)
    close = np.abs(gpu["kappa"] - k) <= 1e-6 * np.maximum(np.abs(k), 1.0)
    assert np.mean(close[both]) > 0.95
    g = I.unit_grid(48)
    L = 20 * g.h
    bv, bt = I.box_front((0.5 - L / 2,) * 3, (0.5 + L / 2,) * 3, 40)
    box = dict(grid=g, verts=np.ascontiguousarray(bv), tris=bt)
    gb = run_gpu(box, params=_gpu_params(v))
    assert gb["status"] == 0
    x = (np.stack([gb["cell_keys"] // (48 * 48), (gb["cell_keys"] // 48) % 48, gb["cell_keys"] % 48], 1) + 0.5) \
        * g.h - 0.5
    top = (np.abs(x[:, 0]) < L / 2 - 6.5 * g.h) & (np.abs(x[:, 1]) < L / 2 - 6.5 * g.h) & (x[:, 2] > 0)
    assert top.sum() >= 16
    assert np.max(np.abs(gb["kappa"][top])) <= 1e-10 / g.h


@pytest.mark.parametrize("variant", ["ring3_vertex", "fragments_vertex_frame"])
def test_paper_neighbourhood_fp32_form(variant):
    """In the FP32 form the ring fit stays float64 (same tolerance as the plain
    path); the fragment fit in the vertex frame runs in float32 (1e-4)."""
    w = I.laplace_droplet_32(1)
    v = VARIANTS[variant]
    gpu = run_gpu(w, params=_gpu_params(v), precision=F.FT_FP32C)
    assert gpu["status"] == 0
    cells = np.unique(oracle.bin_pairs(w["verts"], w["tris"], w["grid"])[0])
    k, n, a, st = oracle.ppic(w["verts"], w["tris"], w["grid"], cells, params=v)
    tol = 1e-9 if v["fit_ring"] else 1e-4
    assert np.array_equal(gpu["fit_status"], st)
    assert np.all(np.abs(gpu["kappa"] - k) <= tol * np.maximum(np.abs(k), 1.0))
    assert np.max(np.abs(gpu["normal"] - n)) <= tol


def test_paper_neighbourhood_is_refused_on_a_batch():
    import torch
    w = I.laplace_droplet_32(1)
    dev = torch.device("cuda", 0)
    dl = [dict(grid=w["grid"], verts=torch.from_numpy(w["verts"]).to(dev), tris=torch.from_numpy(w["tris"]).to(dev))]
    bc = F.BatchCoupling(dl, params=F.make_params())
    bc.step(interp=False)
    prm = F.make_params(fit_ring=3, frame=F.FT_FRAME_VERTEX)
    with pytest.raises(F.FrontError):
        F.front_curvature_ppic(bc.ws, prm, bc.cell_keys, bc.kappa, bc.normal, bc.coeffs, bc.fit_status)
    bc.ws.close()
