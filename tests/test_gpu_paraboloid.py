"""The paper's own cut-cell quantities (Sec. 3.2: alpha = V_P / V_C of the cell
below its fitted paraboloid, curvature and normal averaged over the paraboloid
surface inside the cell) on the GPU against the FP64 oracle.

Tolerances: the oracle integrates to about 1e-12 (its adaptive tolerance); the
kernel's graded Gauss rules agree with it to a few 1e-15 on these inputs, so
the per-cell comparison uses 1e-11.  Through the whole chain (fit, frame,
paraboloid) the GPU and oracle fits differ by the fit's own rounding (FP64)
or by the float32 accumulation (FP32 form), and alpha_P, kbar and nbar inherit
that difference: about the coefficient difference times an O(1) sensitivity."""
import numpy as np
import pytest
import torch

import oracle
from paper_2505_06932_gb300 import _front as F
from paper_2505_06932_gb300 import inputs as I

pytestmark = pytest.mark.gpu

DEV = torch.device("cuda", 0)


def _cells_gpu(fr, co):
    m = fr.shape[0]
    f = torch.from_numpy(np.ascontiguousarray(fr)).to(DEV)
    c = torch.from_numpy(np.ascontiguousarray(co)).to(DEV)
    out = dict(alpha=torch.empty(m, dtype=torch.float64, device=DEV),
               area=torch.empty(m, dtype=torch.float64, device=DEV),
               kappa=torch.empty(m, dtype=torch.float64, device=DEV),
               normal=torch.empty((m, 3), dtype=torch.float64, device=DEV),
               status=torch.empty(m, dtype=torch.int8, device=DEV))
    F.front_paraboloid_cells(f, c, out["alpha"], out["area"], out["kappa"], out["normal"], out["status"])
    torch.cuda.synchronize()
    return {k: v.cpu().numpy() for k, v in out.items()}


def test_paraboloid_cells_match_oracle():
    fr, co = I.paraboloid_cells()
    ref = oracle.paraboloid_cells(fr, co)
    got = _cells_gpu(fr, co)
    assert np.array_equal(got["status"], ref["status"])
    hit = ref["status"] == 0
    assert np.max(np.abs(got["alpha"] - ref["alpha"])) <= 1e-11
    assert np.max(np.abs(got["area"] - ref["area"])) <= 1e-11
    assert np.max(np.abs(got["kappa"] - ref["kbar"]) / np.maximum(1.0, np.abs(ref["kbar"]))) <= 1e-11
    assert np.max(np.abs(got["normal"][hit] - ref["nbar"][hit])) <= 1e-11
    # the misses report the point values at the origin, area 0, alpha 0 or 1
    miss = ~hit
    assert np.all(got["area"][miss] == 0.0) and np.all(np.isin(got["alpha"][miss], (0.0, 1.0)))
    assert np.max(np.abs(got["kappa"][miss] - ref["kbar"][miss])) <= 1e-15


def test_paraboloid_cells_degenerate_cases():
    """Axis-aligned planes and paraboloids (faces parallel to the tangent plane,
    surfaces through cube edges and corners, exact halves) and an empty call."""
    E = np.eye(3).reshape(9)
    cases = np.array([[0.0, 0, 0, 0, 0, 0],        # the mid plane: alpha = 1/2
                      [0.5, 0, 0, 0, 0, 0],        # the top face
                      [-0.5, 0, 0, 0, 0, 0],       # the bottom face
                      [0.0, 1.0, 0, 0, 0, 0],      # the diagonal plane z = x through two edges
                      [0.0, 1.0, 1.0, 0, 0, 0],    # z = x + y through a corner
                      [0.25, 0, 0, 0.5, 0, 0.5],   # a paraboloid crossing the top face
                      [0.0, 0, 0, 1.0, 0, -1.0]])  # a saddle through the centre
    fr = np.tile(E, (len(cases), 1))
    ref = oracle.paraboloid_cells(fr, cases)
    got = _cells_gpu(fr, cases)
    assert got["alpha"][0] == 0.5 and abs(got["alpha"][3] - 0.5) <= 1e-15
    assert np.max(np.abs(got["alpha"] - ref["alpha"])) <= 1e-12
    assert np.array_equal(got["status"], ref["status"])
    hit = ref["status"] == 0
    # the oracle integrates to about 1e-12 (its adaptive tolerance)
    assert np.max(np.abs(got["area"] - ref["area"])) <= 1e-11
    assert np.max(np.abs(got["kappa"][hit] - ref["kbar"][hit])) <= 1e-11
    F.front_paraboloid_cells(torch.empty((0, 9), dtype=torch.float64, device=DEV),
                             torch.empty((0, 6), dtype=torch.float64, device=DEV),
                             torch.empty(0, dtype=torch.float64, device=DEV))


def _chain(w, precision):
    g = w["grid"]
    prm = F.make_params(precision=precision)
    v = torch.from_numpy(w["verts"]).to(DEV)
    t = torch.from_numpy(w["tris"]).to(DEV)
    fc = F.FrontCoupling(g, t.shape[0], v.shape[0], params=prm)
    F.front_bin(fc.ws, v, t, prm)
    F.front_volume_fraction(fc.ws, fc.alpha)
    F.front_curvature_ppic(fc.ws, prm, fc.cell_keys, fc.kappa, fc.normal, fc.coeffs, fc.fit_status)
    exact = fc.alpha.clone()
    cap = fc.coeffs.shape[0]
    frame = torch.empty((cap, 9), dtype=torch.float64, device=DEV)
    F.front_ppic_frame(fc.ws, frame)
    kb = torch.empty(cap, dtype=torch.float64, device=DEV)
    nb = torch.empty((cap, 3), dtype=torch.float64, device=DEV)
    ar = torch.empty(cap, dtype=torch.float64, device=DEV)
    st = torch.empty(cap, dtype=torch.int8, device=DEV)
    F.front_volume_fraction_ppic(fc.ws, fc.coeffs, fc.alpha, kb, nb, ar, st)
    assert fc.ws.status() == 0
    M = fc.ws.counts()["M"]
    keys = fc.cell_keys[:M].cpu().numpy().view(np.uint32)
    out = dict(keys=keys, alpha=fc.alpha.cpu().numpy(), exact=exact.cpu().numpy(), frame=frame[:M].cpu().numpy(),
               kbar=kb[:M].cpu().numpy(), nbar=nb[:M].cpu().numpy(), area=ar[:M].cpu().numpy(),
               status=st[:M].cpu().numpy())
    fc.ws.close()
    return out


CASES = {"droplet_32": lambda: I.laplace_droplet_32(1),
         "sh_droplet_40": lambda: I.sh_droplet_256(seed=9, s=4, N=40)}


@pytest.mark.parametrize("case", list(CASES))
@pytest.mark.parametrize("precision", [F.FT_FP64, F.FT_FP32C], ids=["fp64", "fp32c"])
def test_volume_fraction_ppic_matches_oracle(case, precision):
    w = CASES[case]()
    g = w["grid"]
    cells, _ = oracle.interfacial_cells(w["verts"], w["tris"], g)
    k, n, co, fst, fr = oracle.ppic(w["verts"], w["tris"], g, cells, frame=True)
    ref = oracle.paraboloid_cells(fr, co)
    got = _chain(w, precision)
    assert np.array_equal(got["keys"], cells)
    fp64 = precision == F.FT_FP64
    # the frames: the same construction from the (float-summed in FP32) normal
    assert np.max(np.abs(got["frame"] - fr)) <= (1e-12 if fp64 else 1e-5)
    # alpha_P replaces alpha exactly at the interfacial cells; the rest is untouched
    other = np.ones(got["alpha"].shape, bool)
    other[cells] = False
    assert np.array_equal(got["alpha"][other], got["exact"][other])
    assert np.max(np.abs(got["alpha"][cells] - ref["alpha"])) <= (1e-9 if fp64 else 2e-5)
    hit = (ref["status"] == 0) & (got["status"] == 0)
    # status may differ only where the patch is within the fit difference of missing the cell
    assert np.all(ref["area"][ref["status"] != got["status"]] < 1e-3)
    kref = ref["kbar"] / g.h
    tol_k = 1e-7 if fp64 else 2e-3
    assert np.max(np.abs(got["kbar"][hit] - kref[hit]) / np.maximum(np.abs(kref[hit]), 1.0 / g.h)) <= tol_k
    assert np.max(np.abs(got["nbar"][hit] - ref["nbar"][hit])) <= (1e-8 if fp64 else 2e-4)
    assert np.max(np.abs(got["area"] - ref["area"] * g.h * g.h)) <= (1e-9 if fp64 else 2e-5) * g.h * g.h


def test_volume_fraction_ppic_batch_equals_one_front():
    ws = [I.laplace_droplet_32(1), I.sh_droplet_256(seed=9, s=4, N=40)]
    prm = F.make_params()
    fronts = [dict(grid=w["grid"], verts=torch.from_numpy(w["verts"]).to(DEV),
                   tris=torch.from_numpy(w["tris"]).to(DEV)) for w in ws]
    bc = F.BatchCoupling(fronts, params=prm)
    bc.step(interp=False)
    cap = bc.coeffs.shape[0]
    kb = torch.empty(cap, dtype=torch.float64, device=DEV)
    nb = torch.empty((cap, 3), dtype=torch.float64, device=DEV)
    ar = torch.empty(cap, dtype=torch.float64, device=DEV)
    F.front_volume_fraction_ppic_batch(bc.ws, bc.coeffs, kb, nb, ar)
    torch.cuda.synchronize()
    assert bc.ws.status() == 0
    off = 0
    for w, d in zip(ws, bc.fronts):
        one = _chain(w, F.FT_FP64)
        M = one["keys"].shape[0]
        assert np.array_equal(d["alpha"].cpu().numpy().reshape(-1), one["alpha"])
        assert np.array_equal(kb[off:off + M].cpu().numpy(), one["kbar"])
        assert np.array_equal(nb[off:off + M].cpu().numpy(), one["nbar"])
        assert np.array_equal(ar[off:off + M].cpu().numpy(), one["area"])
        off += M


def test_volume_fraction_ppic_needs_a_fit():
    w = I.laplace_droplet_32(1)
    g = w["grid"]
    prm = F.make_params()
    v = torch.from_numpy(w["verts"]).to(DEV)
    t = torch.from_numpy(w["tris"]).to(DEV)
    fc = F.FrontCoupling(g, t.shape[0], v.shape[0], params=prm)
    F.front_bin(fc.ws, v, t, prm)
    with pytest.raises(F.FrontError):
        F.front_volume_fraction_ppic(fc.ws, fc.coeffs, fc.alpha)
    fc.ws.close()
