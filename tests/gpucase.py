"""Run one front through the CUDA path (C ABI) and through the oracle."""
import numpy as np
import torch

import oracle
from paper_2505_06932_gb300 import _front as F


def run_gpu(w, params=None, max_cand=0, precision=F.FT_FP64):
    g = w["grid"]
    p = params or {}
    prm = F.make_params(precision=precision, **p)
    dev = torch.device("cuda", 0)
    verts = torch.from_numpy(np.ascontiguousarray(w["verts"])).to(dev)
    tris = torch.from_numpy(np.ascontiguousarray(w["tris"])).to(dev)
    faces = [torch.from_numpy(np.ascontiguousarray(f)).to(dev) for f in w["faces"]] if "faces" in w else None
    fc = F.FrontCoupling(g, max(1, tris.shape[0]), max(1, verts.shape[0]), max_cand=max_cand, params=prm)
    F.front_bin(fc.ws, verts, tris, prm)
    F.front_volume_fraction(fc.ws, fc.alpha)
    F.front_curvature_ppic(fc.ws, prm, fc.cell_keys, fc.kappa, fc.normal, fc.coeffs, fc.fit_status)
    F.front_csf_force(fc.ws, prm, fc.alpha, fc.kappa, fc.normal, fc.force)
    if faces is not None and verts.shape[0] > 0:
        F.front_interp_velocity(g, faces[0], faces[1], faces[2], verts, fc.vel[:verts.shape[0]])
    res = fc.results(verts.shape[0])
    P = res["counts"]["P"]
    keys = torch.empty(max(1, P), dtype=torch.int32, device=dev)
    tids = torch.empty(max(1, P), dtype=torch.int32, device=dev)
    F.ft_bin_pairs(fc.ws, keys, tids)
    res["pair_keys"] = keys[:P].cpu().numpy().view(np.uint32)
    res["pair_tris"] = tids[:P].cpu().numpy()
    res["status"] |= fc.ws.status()
    fc.ws.close()
    return res


def run_oracle(w, params=None, cells=None, need=("alpha", "ppic", "csf", "interp")):
    g = w["grid"]
    p = dict(oracle.DEFAULT_PARAMS)
    if params:
        p.update(params)
    margin = oracle.margin_for(p["delta_max_h"])
    keys, tids, st = oracle.bin_pairs(w["verts"], w["tris"], g, margin)
    out = dict(pair_keys=keys, pair_tris=tids, status=st, cells=np.unique(keys))
    if "alpha" in need:
        out["alpha"], st2 = oracle.alpha(w["verts"], w["tris"], g, margin)
        out["status"] |= st2
    if "ppic" in need:
        c = out["cells"] if cells is None else cells
        out["kappa"], out["normal"], out["coeffs"], out["fit_status"] = oracle.ppic(w["verts"], w["tris"], g, c, p)
    if "csf" in need and "alpha" in out and "kappa" in out and cells is None:
        out["force"] = oracle.csf(g, out["alpha"], out["cells"], out["kappa"], out["normal"], p["sigma"])
    if "interp" in need and "faces" in w:
        out["vel"] = oracle.interp(g, w["faces"], w["verts"])
    return out
