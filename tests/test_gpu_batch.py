"""Batched form: many independent fronts, each on its own grid, in one launch
sequence (front_bin_batch ... front_interp_velocity_batch).

Every front's outputs must equal, bit for bit, those of the one-front entry
points on that front alone (each cell's sums run over the same fragments in the
same order), and match the FP64 oracle within the parity tolerances.  Errors of
one front must not touch the others.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2505_06932_gb300 import _front as F
from paper_2505_06932_gb300 import inputs as I
from gpucase import run_gpu, run_oracle
from test_gpu_parity import FP32_TOL, FP64_TOL, compare

pytestmark = pytest.mark.gpu

DEV = torch.device("cuda", 0)
FIELDS = ("alpha", "cell_keys", "kappa", "normal", "coeffs", "fit_status", "force", "vel")


def _dev(a, dtype=None):
    t = torch.from_numpy(np.ascontiguousarray(a))
    return t.to(DEV) if dtype is None else t.to(DEV, dtype)


def _to_device(w):
    d = dict(grid=w["grid"], verts=_dev(w["verts"]), tris=_dev(w["tris"]))
    if "faces" in w:
        d["U"], d["V"], d["W"] = (_dev(f) for f in w["faces"])
    return d


def _uneven_fronts():
    """Six fronts of uneven size on different grids (with face velocities)."""
    ws = [
        I.laplace_droplet_32(1),
        I.small_sphere(3, 0.3, 36, seed=4, noise_h=1e-3),
        I.sh_droplet_256(seed=9, s=4, N=40),
        I.small_sphere(2, 0.12, 24, seed=6),
        I.sh_droplet_256(seed=10, bubble=True, s=4, N=40),
        I.small_sphere(4, 0.22, 48, seed=8, noise_h=1e-3),
    ]
    return ws


def _run_batch(ws_list, precision=F.FT_FP64, **kw):
    prm = F.make_params(precision=precision)
    bc = F.BatchCoupling([_to_device(w) for w in ws_list], params=prm, **kw)
    bc.step()
    torch.cuda.synchronize()
    return bc


def _batch_pairs(bc, b):
    """Sorted (cell, triangle) pairs of front b, front-local."""
    P = bc.ws.counts()["P"]
    keys = torch.empty(max(P, 1), dtype=torch.int32, device=DEV)
    tids = torch.empty(max(P, 1), dtype=torch.int32, device=DEV)
    F.ft_bin_pairs(bc.ws, keys, tids)
    k = keys[:P].cpu().numpy().view(np.uint32).astype(np.int64)
    t = tids[:P].cpu().numpy().astype(np.int64)
    kb = sum(int(f["grid"].ncells) for f in bc.fronts[:b])
    tb = sum(int(f["tris"].shape[0]) for f in bc.fronts[:b])
    sel = (k >= kb) & (k < kb + bc.fronts[b]["grid"].ncells)
    return (k[sel] - kb).astype(np.uint32), (t[sel] - tb).astype(np.int32)


def _assert_same(batch_res, single_res, pairs, name):
    for f in FIELDS:
        if f in batch_res and f in single_res:
            assert np.array_equal(batch_res[f], single_res[f]), f"{name}: {f} differs from the one-front path"
    assert np.array_equal(pairs[0], single_res["pair_keys"]), f"{name}: pair keys"
    assert np.array_equal(pairs[1], single_res["pair_tris"]), f"{name}: pair triangles"


@pytest.mark.parametrize("precision", [F.FT_FP64, F.FT_FP32C], ids=["fp64", "fp32c"])
def test_batch_equals_one_front_path(precision):
    wl = _uneven_fronts()
    bc = _run_batch(wl, precision)
    assert bc.ws.status() == 0
    assert bc.ws.front_status() == [0] * len(wl)
    for b, w in enumerate(wl):
        single = run_gpu(w, precision=precision)
        assert single["status"] == 0
        _assert_same(bc.results(b), single, _batch_pairs(bc, b), f"front {b}")


def test_batch_fronts_match_oracle():
    """Three fronts of the batch against the FP64 oracle, every output."""
    wl = _uneven_fronts()
    bc = _run_batch(wl)
    for b in (0, 3, 4):
        w = wl[b]
        gpu = bc.results(b)
        gpu["status"] = bc.ws.front_status()[b]
        gpu["pair_keys"], gpu["pair_tris"] = _batch_pairs(bc, b)
        orc = run_oracle(w)
        orc["_faces"] = w["faces"]
        compare(gpu, orc)


def test_batch_cell_ranges():
    wl = _uneven_fronts()
    bc = _run_batch(wl)
    off = bc.off.cpu().numpy()
    M = bc.ws.counts()["M"]
    assert off[0] == 0 and off[-1] == M
    keys = bc.cell_keys[:M].cpu().numpy().view(np.uint32).astype(np.int64)
    assert np.all(np.diff(keys) > 0)
    kb = 0
    for b, w in enumerate(wl):
        seg = keys[off[b]:off[b + 1]]
        assert np.all((seg >= kb) & (seg < kb + w["grid"].ncells))
        kb += w["grid"].ncells


def test_batch_isolates_bad_fronts():
    """A front outside the grid margin, an inverted front and a front with a bad
    vertex index are flagged on their own; the other fronts are unchanged."""
    good = _uneven_fronts()[:3]
    big = I.small_sphere(3, 0.47, 32, seed=2)  # reaches into the margin
    inv = I.small_sphere(3, 0.25, 32, seed=3)
    inv = dict(inv, tris=np.ascontiguousarray(inv["tris"][:, ::-1]))
    bad = I.small_sphere(2, 0.25, 32, seed=5)
    t = bad["tris"].copy()
    t[7, 1] = bad["verts"].shape[0] + 3
    bad = dict(bad, tris=t)
    wl = [good[0], big, good[1], inv, bad, good[2]]
    bc = _run_batch(wl)
    st = bc.ws.front_status()
    assert st[1] & 0x02, st  # outside grid
    assert st[3] & 0x08, st  # orientation
    assert st[4] & 0x10, st  # bad index
    for b in (0, 2, 5):
        assert st[b] == 0, st
    bits = bc.ws.status()
    assert bits & 0x02 and bits & 0x08 and bits & 0x10
    for b, w in ((0, good[0]), (2, good[1]), (5, good[2])):
        single = run_gpu(w)
        _assert_same(bc.results(b), single, _batch_pairs(bc, b), f"front {b}")


def test_autotune_keeps_results():
    wl = _uneven_fronts()
    bc = _run_batch(wl)
    before = [bc.results(b) for b in range(len(wl))]
    t = F.ft_autotune(bc.ws, bc.params, reps=2)
    for k in ("clip_blocks_per_sm", "ppic_blocks_per_sm", "csf_blocks_per_sm", "fill_blocks_per_sm"):
        assert 1 <= t[k] <= 32
    assert t["ppic_min_blocks"] in (4, 6) and t["ppic_dynamic"] in (0, 1)
    assert t["cells_need"] == bc.ws.counts()["M"]
    assert t["step_ms"] > 0
    assert F.ft_get_tuning(bc.ws)["clip_blocks_per_sm"] == t["clip_blocks_per_sm"]
    bc.step()
    torch.cuda.synchronize()
    assert bc.ws.front_status() == [0] * len(wl)
    for b in range(len(wl)):
        after = bc.results(b)
        for f in FIELDS:
            if f in after:
                assert np.array_equal(after[f], before[b][f]), f
    # every shape gives the same results
    F.ft_set_tuning(bc.ws, clip=1, ppic=1, csf=1, fill=1, ppic_min_blocks=6, ppic_dynamic=1 - t["ppic_dynamic"],
                    sort_blocks=7)
    bc.step()
    torch.cuda.synchronize()
    for b in range(len(wl)):
        after = bc.results(b)
        for f in FIELDS:
            if f in after:
                assert np.array_equal(after[f], before[b][f]), f


def test_batch_rejects_one_front_calls():
    wl = _uneven_fronts()[:2]
    bc = _run_batch(wl)
    d = bc.fronts[0]
    with pytest.raises(F.FrontError):
        F.front_bin(bc.ws, d["verts"], d["tris"], bc.params)


# ---------------------------------------------------------------------------
# the 512-front workload (subdivision 3-6, grids 32^3-96^3, radius 3h-20h)
# ---------------------------------------------------------------------------

def _sampled_fronts(fr, k=6):
    """k fronts small enough for the oracle in seconds, spread over the batch."""
    small = [b for b, f in enumerate(fr) if f["tris"].shape[0] <= 20480 and f["grid"].n[0] <= 64]
    idx = np.linspace(0, len(small) - 1, k).round().astype(int)
    return [small[i] for i in idx]


@pytest.mark.parametrize("precision", [F.FT_FP32C, F.FT_FP64], ids=["fp32c", "fp64"])
def test_batch_512(precision):
    fr = I.batch_fronts(5, 512)
    dl = []
    for f in fr:
        d = dict(grid=f["grid"], verts=_dev(f["verts"]), tris=_dev(f["tris"]))
        dl.append(d)
    prm = F.make_params(precision=precision)
    bc = F.BatchCoupling(dl, params=prm, headroom=1.02)
    bc.step(interp=False)
    torch.cuda.synchronize()
    assert bc.ws.status() == 0
    assert bc.ws.front_status() == [0] * len(fr)
    tol = FP32_TOL if precision == F.FT_FP32C else FP64_TOL
    # every front: enclosed volume (sum alpha h^3 = signed mesh volume); each cut
    # cell may carry the alpha tolerance, every other cell is exact
    vols = torch.stack([f["alpha"].sum() for f in bc.fronts]).cpu().numpy()
    off = bc.off.cpu().numpy()
    for b, f in enumerate(fr):
        h = f["grid"].h
        vm = I.signed_volume(f["verts"], f["tris"])
        mb = int(off[b + 1] - off[b])
        assert mb > 0, b
        assert abs(vols[b] * h ** 3 - vm) <= 1e-10 * vm + tol["alpha"] * mb * h ** 3, b
    # sampled fronts against the oracle: bins bit-exact, alpha in full, PPIC on sampled cells
    for b in _sampled_fronts(fr):
        w = fr[b]
        res = bc.results(b)
        pk, pt = _batch_pairs(bc, b)
        keys, tids, st = oracle.bin_pairs(w["verts"], w["tris"], w["grid"], oracle.margin_for(4.0))
        assert st == 0
        assert np.array_equal(pk, keys) and np.array_equal(pt, tids), b
        cells = np.unique(keys)
        assert np.array_equal(res["cell_keys"], cells), b
        a, st2 = oracle.alpha(w["verts"], w["tris"], w["grid"], oracle.margin_for(4.0))
        assert st2 == 0
        inter = np.zeros(a.size, bool)
        inter[cells] = True
        assert np.array_equal(res["alpha"].reshape(-1)[~inter], a.reshape(-1)[~inter]), b
        assert np.max(np.abs(res["alpha"] - a)) <= tol["alpha"], b
        sel = np.sort(I.rng(b).choice(len(cells), size=min(64, len(cells)), replace=False))
        ko, no, co, so = oracle.ppic(w["verts"], w["tris"], w["grid"], cells[sel])
        k = res["kappa"][sel]
        assert np.all(np.abs(k - ko) <= tol["kappa"] * np.maximum(np.abs(ko), 1.0)), b
        assert np.max(np.abs(res["normal"][sel] - no)) <= tol["normal"], b
        assert np.array_equal(res["fit_status"][sel], so), b
