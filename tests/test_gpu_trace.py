"""The per-kernel trace (ft_trace_start / ft_trace_stop) and the work counts
(ft_work_counts) behind the benchmark's per-kernel rooflines; and the share of
pairs that the FP32 clip leaves to the binary64 canonical clip."""
import numpy as np
import pytest
import torch

from paper_2505_06932_gb300 import _front as F
from paper_2505_06932_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def _coupling(w, precision):
    dev = torch.device("cuda", 0)
    v = torch.from_numpy(w["verts"]).to(dev)
    t = torch.from_numpy(w["tris"]).to(dev)
    fa = [torch.from_numpy(f).to(dev) for f in w["faces"]]
    fc = F.FrontCoupling(w["grid"], t.shape[0], v.shape[0], params=F.make_params(precision=precision))
    return fc, v, t, fa


@pytest.mark.parametrize("precision", [F.FT_FP64, F.FT_FP32C], ids=["fp64", "fp32c"])
def test_trace_counts_every_kernel_of_a_step(precision):
    w = I.laplace_droplet_32(1)
    fc, v, t, fa = _coupling(w, precision)
    fc.step(v, t, fa)  # warm-up
    torch.cuda.synchronize()
    F.trace_start(1024)
    for _ in range(3):
        fc.step(v, t, fa)
    tr = F.trace_stop()
    assert tr[None] == 0
    clip = "k_clip32" if precision == F.FT_FP32C else "k_clip"
    acc = "k_ppic_acc<float>" if precision == F.FT_FP32C else "k_ppic_acc<double>"
    for k in ("k_tri_setup", clip, "k_cnt_down", "k_place", "k_cell_order", "k_alpha_fill", acc,
              "k_ppic_solve", "k_csf_ring_list", "k_csf_force", "k_interp"):
        n, ms = tr[k]
        assert n == 3 and ms > 0.0, k
    # nothing traced once the trace is closed, and a second stop is an error
    fc.step(v, t, fa)
    with pytest.raises(F.FrontError):
        F.trace_stop()
    # a trace does not follow launches into a stream capture
    F.trace_start(1024)
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        fc.step(v, t, fa)
    g.replay()
    torch.cuda.synchronize()
    tr2 = F.trace_stop()
    assert [k for k in tr2 if k is not None] == []
    wc = fc.ws.work_counts()
    c = fc.ws.counts()
    assert wc["T"] == t.shape[0] and wc["M"] == c["M"] and wc["P"] == c["P"] and wc["C"] == c["C"]
    assert wc["fit_pairs"] == c["fit_pairs"] and wc["ring"] > 0
    if precision == F.FT_FP64:
        assert wc["clip_f64"] == 0
    fc.ws.close()


def test_fp32_clip_decides_nearly_every_pair_in_float32():
    """On a generic front the certified float32 clip leaves under 2 % of
    the candidate pairs to the binary64 clip; a box whose faces lie in grid
    planes (fragments in cell faces, edges along cell edges) sends some pairs
    there (its bins are checked bit for bit in test_gpu_parity)."""
    fc, v, t, fa = _coupling(I.ellipsoid_128(3), F.FT_FP32C)
    fc.step(v, t, fa)
    wc = fc.ws.work_counts()
    assert 0 <= wc["clip_f64"] < 0.02 * wc["C"]
    fc.ws.close()
    g = I.unit_grid(48)
    L = 20 * g.h
    bv, bt = I.box_front((0.5 - L / 2,) * 3, (0.5 + L / 2,) * 3, 40)
    dev = torch.device("cuda", 0)
    ws = F.Workspace(g, bt.shape[0])
    F.front_bin(ws, torch.from_numpy(np.ascontiguousarray(bv)).to(dev), torch.from_numpy(bt).to(dev),
                F.make_params(precision=F.FT_FP32C))
    wc = ws.work_counts()
    assert wc["clip_f64"] > 0
    ws.close()
