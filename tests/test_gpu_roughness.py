"""Local roughness detection and smoothing (Sec. 3.4) on the GPU against the
FP64 oracle."""
import numpy as np
import pytest
import torch

import oracle
from paper_2505_06932_gb300 import _front as F
from paper_2505_06932_gb300 import inputs as I

pytestmark = pytest.mark.gpu

DEV = torch.device("cuda", 0)


def _bumpy(s=4, seed=5, n=12):
    v, t = I.sphere_front(s, 0.25, (0.5, 0.5, 0.5), radial_noise=1e-4, gen=I.rng(seed + 1))
    gen = I.rng(seed)
    idx = gen.choice(v.shape[0], n, replace=False)
    v = v.copy()
    v[idx] = 0.5 + (v[idx] - 0.5) * (1.0 + gen.uniform(0.03, 0.06, (n, 1)))
    return v, t


CASES = {
    "rough_sphere": lambda: I.sphere_front(4, 0.25, (0.5, 0.5, 0.5), radial_noise=1e-3, gen=I.rng(2)),
    "bumpy_sphere": lambda: _bumpy(),
    "box": lambda: I.box_front((0.2, 0.25, 0.3), (0.7, 0.65, 0.8), 7),
    "sh_droplet": lambda: I.sh_deformed_front(5, 0.2, np.array([0.5, 0.5, 0.5]), I.rng(9)),
}


@pytest.mark.parametrize("case", list(CASES))
def test_roughness_metrics_match_oracle(case):
    v, t = CASES[case]()
    ref = oracle.roughness(v, t)
    rg = F.Roughness(v.shape[0], t.shape[0])
    got = rg.metrics(torch.from_numpy(v).to(DEV), torch.from_numpy(t).to(DEV))
    assert rg.status() == 0
    scale = np.abs(v).max()
    for k in ("gl",):
        assert np.max(np.abs(got[k].cpu().numpy() - ref[k])) <= 1e-13 * scale, k
    for k in ("G", "V", "rt", "r1", "r2", "rough"):
        r = ref[k]
        assert np.max(np.abs(got[k].cpu().numpy() - r)) <= 1e-12 * max(np.abs(r).max(), 1e-300), k
    rg.close()


@pytest.mark.parametrize("case", ["bumpy_sphere", "sh_droplet"])
def test_roughness_smoothing_matches_oracle(case):
    v, t = CASES[case]()
    if case == "bumpy_sphere":
        r0 = oracle.roughness(*I.sphere_front(4, 0.25, (0.5, 0.5, 0.5)))
        gl_thr = 1.3 * np.linalg.norm(r0["gl"], axis=1).max()
        r_thr = 1.3 * r0["rough"].max()
    else:
        r0 = oracle.roughness(v, t)        # the top of this front's own range
        gl_thr = 0.8 * np.linalg.norm(r0["gl"], axis=1).max()
        r_thr = 0.8 * r0["rough"].max()
    vo, rounds_o, moved_o = oracle.roughness_smooth(v, t, gl_thr, r_thr)
    assert moved_o > 0
    rg = F.Roughness(v.shape[0], t.shape[0])
    x = torch.from_numpy(v.copy()).to(DEV)
    res = rg.smooth(x, torch.from_numpy(t).to(DEV), gl_thr, r_thr)
    assert res["status"] == 0
    assert res["rounds"] == rounds_o and res["moved"] == moved_o
    xg = x.cpu().numpy()
    assert np.max(np.abs(xg - vo)) <= 1e-12 * np.abs(v).max()
    assert abs(oracle.signed_volume(xg, t) / oracle.signed_volume(v, t) - 1.0) <= 1e-13
    rg.close()


def test_roughness_rejects_bad_indices():
    v, t = CASES["rough_sphere"]()
    t = t.copy()
    t[5, 2] = v.shape[0] + 7
    rg = F.Roughness(v.shape[0], t.shape[0])
    with pytest.raises(F.FrontError):
        rg.metrics(torch.from_numpy(v).to(DEV), torch.from_numpy(t).to(DEV))
    rg.close()
