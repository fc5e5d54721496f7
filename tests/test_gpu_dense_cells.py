"""Fronts much finer than the grid: thousands of (cell, triangle) pairs per
cell.  The binning puts each cell's pairs in triangle order with a warp per
cell up to 256 pairs and a block per larger cell (shared-memory sort of chunks
of 4,096 slots, then merges of the sorted runs); the pairs must equal the
oracle's bit for bit on every path, and alpha match it."""
import numpy as np
import pytest

import oracle
from paper_2505_06932_gb300 import _front as F
from paper_2505_06932_gb300 import inputs as I
from gpucase import run_gpu

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("s,expect_max", [(6, 256), (8, 4096)])
def test_dense_cells_pairs_and_alpha(s, expect_max):
    N = 24
    w = I.small_sphere(s, 2.5 / N, N, seed=11)
    g = w["grid"]
    keys, tids, st = oracle.bin_pairs(w["verts"], w["tris"], g)
    assert st == 0
    per_cell = np.unique(keys, return_counts=True)[1]
    assert per_cell.max() > expect_max  # the path under test is taken
    for precision in (F.FT_FP64, F.FT_FP32C):
        gpu = run_gpu(w, precision=precision)
        assert gpu["status"] == 0
        assert np.array_equal(gpu["pair_keys"], keys)
        assert np.array_equal(gpu["pair_tris"], tids)
    # alpha: each cell's terms are summed in another order on either side; with
    # up to n = 22,349 fragment terms of magnitude <= 1 per cell the two sums
    # differ by at most about 2 n 2^-53 per cell, carried down a column of 24
    al, st2 = oracle.alpha(w["verts"], w["tris"], g)
    assert st2 == 0
    gpu = run_gpu(w, precision=F.FT_FP64)
    tol = 2 * 24 * 2.0 * per_cell.max() * 2.0 ** -53
    assert np.max(np.abs(gpu["alpha"] - al)) <= tol
    # the FP32 form sums thousands of float fragment terms per cell with
    # compensated (two-sum) accumulation: it keeps the form's stated 1e-6
    gpu32 = run_gpu(w, precision=F.FT_FP32C)
    assert np.max(np.abs(gpu32["alpha"] - al)) <= 1e-6


def test_cell_capacity_overflow_then_recovery():
    """More interfacial cells than the workspace holds: the binning flags the
    capacity and leaves no cells; the per-key counters are back to zero, so the
    next binning on the same workspace (a front that fits) equals the oracle."""
    import torch
    dev = torch.device("cuda", 0)
    N = 32
    big = I.small_sphere(4, 0.25, N, seed=3)
    small = I.small_sphere(3, 0.12, N, seed=4)
    prm = F.make_params(precision=F.FT_FP64)
    nt = max(big["tris"].shape[0], small["tris"].shape[0])
    M_small = len(np.unique(oracle.bin_pairs(small["verts"], small["tris"], small["grid"])[0]))
    M_big = len(np.unique(oracle.bin_pairs(big["verts"], big["tris"], big["grid"])[0]))
    assert M_small < M_big
    ws = F.Workspace(big["grid"], nt, max_cells=M_small)
    for w, over in ((big, True), (small, False), (big, True), (small, False)):
        v = torch.from_numpy(w["verts"]).to(dev)
        t = torch.from_numpy(w["tris"]).to(dev)
        F.front_bin(ws, v, t, prm)
        c, st = ws.counts(), ws.status()
        if over:
            assert st & 0x01 and c["M"] == 0 and c["P"] == 0
        else:
            assert st == 0
            keys, tids, _ = oracle.bin_pairs(w["verts"], w["tris"], w["grid"])
            P = c["P"]
            k = torch.empty(P, dtype=torch.int32, device=dev)
            tr = torch.empty(P, dtype=torch.int32, device=dev)
            F.ft_bin_pairs(ws, k, tr)
            assert c["M"] == M_small
            assert np.array_equal(k.cpu().numpy().view(np.uint32), keys)
            assert np.array_equal(tr.cpu().numpy(), tids)
    ws.close()
