"""Served form on the GPU: continuous batching of requests that arrive over
time.  Each request's result (front positions after its last step, and the
alpha, kappa and force of that step) is the same served alone and served in a
mix with other requests; a request whose front leaves the grid margin fails on
its own; the first step agrees with the oracle."""
import numpy as np
import pytest
import torch

import oracle
from paper_2505_06932_gb300 import _front as F
from paper_2505_06932_gb300 import inputs as I
from paper_2505_06932_gb300 import serve as S

pytestmark = pytest.mark.gpu

FIELDS = ("verts", "alpha", "kappa", "normal", "force")


def _requests(count=8, rate=400.0, seed=3):
    rq = I.served_requests(seed, count, rate, s_choices=(3, 4), n_choices=(32, 48, 64), max_steps=6,
                           pool_per_s=1)
    return [S.Request(r["rid"], r["grid"], r["verts"], r["tris"], r["steps"], r["arrival"], r["dt"],
                      tuple(r["centre"]), tuple(r["omega"])) for r in rq]


def _cap(reqs, budget=None):
    return S.Capacity(budget_bytes=budget or 8 * sum(S.footprint(r) for r in reqs), max_fronts=64,
                      max_grid_cells=sum(r.grid.ncells for r in reqs),
                      max_nt=sum(r.tris.shape[0] for r in reqs),
                      max_cand=sum(S.candidate_estimate(r) for r in reqs))


def _serve(reqs, precision=F.FT_FP32C, budget=None, realtime=False):
    cap = _cap(reqs, budget)
    ex = S.BatchExecutor(cap, F.make_params(precision=precision), keep_results=True)
    try:
        outs, stats = S.serve(reqs, ex, cap, realtime=realtime, keep_results=True)
    finally:
        ex.close()
    return outs, stats


@pytest.mark.parametrize("precision", [F.FT_FP32C, F.FT_FP64], ids=["fp32c", "fp64"])
def test_same_result_alone_and_in_the_mix(precision):
    reqs = _requests()
    # a budget of about three requests forces queueing and joins mid-flight
    budget = 3 * max(S.footprint(r) for r in reqs)
    outs, stats = _serve(reqs, precision, budget=budget)
    assert stats["completed"] == len(reqs) and stats["failed"] == 0
    assert stats["peak_bytes"] <= budget
    overlap = any(outs[a.rid].admitted < outs[b.rid].admitted < outs[a.rid].finished
                  for a in reqs for b in reqs if a.rid != b.rid)
    assert overlap, "no request joined while another was running"
    seq = S.SequentialExecutor(F.make_params(precision=precision), keep_results=True)
    for r in reqs[:4]:
        alone, st = _serve([r], precision)
        a, m = alone[r.rid].result, outs[r.rid].result
        for f in FIELDS:
            assert np.array_equal(a[f], m[f]), (r.rid, f)
        # the plain path: one-front entry points, no batching
        cells, status, res = seq.run(r)
        assert status == 0 and cells == outs[r.rid].cells
        for f in FIELDS:
            assert np.array_equal(res[f], m[f]), (r.rid, f, "sequential")


def test_failing_request_is_isolated():
    reqs = _requests(count=4)
    bad = reqs[1]
    g = bad.grid
    # push the front into the grid margin (its largest x two cells from the face)
    off = np.array([1.0 - 2 * g.h - bad.verts[:, 0].max(), 0.0, 0.0])
    shifted = S.Request(bad.rid, g, bad.verts + off, bad.tris, bad.steps, bad.arrival, bad.dt,
                        tuple(np.asarray(bad.centre) + off), bad.omega)
    mix = [reqs[0], shifted, reqs[2], reqs[3]]
    outs, stats = _serve(mix)
    assert outs[bad.rid].status & 0x02
    assert stats["failed"] == 1
    for r in (reqs[0], reqs[2], reqs[3]):
        alone, _ = _serve([r])
        assert outs[r.rid].status == 0
        for f in FIELDS:
            assert np.array_equal(alone[r.rid].result[f], outs[r.rid].result[f]), (r.rid, f)


def test_first_step_matches_the_oracle():
    """One step of one served request: alpha and kappa at the initial positions
    and the RK4 positions, against the FP64 oracle (FP64 path tolerances)."""
    r = _requests(count=1)[0]
    r.steps = 1
    outs, _ = _serve([r], F.FT_FP64)
    res = outs[r.rid].result
    g = r.grid
    a, st = oracle.alpha(r.verts, r.tris, g)
    assert st == 0
    assert np.max(np.abs(res["alpha"].reshape(a.shape) - a)) <= 1e-12
    cells, _ = oracle.interfacial_cells(r.verts, r.tris, g)
    k, n, _, _ = oracle.ppic(r.verts, r.tris, g, cells)
    assert np.all(np.abs(res["kappa"] - k) <= 1e-9 * np.maximum(np.abs(k), 1.0))
    faces = I.solid_body_faces_exact(g, r.centre, r.omega)
    x1, _ = oracle.advect_rk4(g, faces, r.verts, r.dt)
    assert np.max(np.abs(res["verts"] - x1)) <= 1e-12 * r.dt + 4e-16
