"""Host logic of the serving loop (no GPU): admission by device footprint and
batch capacities in arrival order, continuous batching (requests join while
others run), release of resources, latency accounting."""
import numpy as np

from paper_2505_06932_gb300 import inputs as I
from paper_2505_06932_gb300 import serve as S


class FakeClock:
    def __init__(self):
        self.t = 0.0

    def __call__(self):
        return self.t


class FakeExecutor:
    """Each iteration takes `dt_iter` seconds of the fake clock plus a cost per
    active front; records which requests ran together."""

    def __init__(self, clock, dt_iter=0.01, per_front=0.001):
        self.clock = clock
        self.dt_iter = dt_iter
        self.per_front = per_front
        self.active = []
        self.history = []
        self.fail = set()

    def admit(self, req):
        self.active.append(req.rid)

    def release(self, rid):
        self.active.remove(rid)

    def iterate(self):
        self.clock.t += self.dt_iter + self.per_front * len(self.active)
        self.history.append(list(self.active))
        return ({r: 10 for r in self.active}, {r: (0x02 if r in self.fail else 0) for r in self.active})

    def result(self, rid):
        return {}


def _req(rid, arrival, steps, N=32, s=2):
    g = I.unit_grid(N)
    v, t = I.sphere_front(s, 0.2, (0.5, 0.5, 0.5))
    return S.Request(rid, g, v, t, steps, arrival, 0.25 * g.h)


def _cap(budget, fronts=64):
    return S.Capacity(budget_bytes=budget, max_fronts=fronts, max_grid_cells=10 ** 9, max_nt=10 ** 9,
                      max_cand=10 ** 9)


def test_footprint_counts_fields_and_mesh():
    r = _req(0, 0.0, 1, N=32, s=2)
    n = 32
    faces = 3 * (n + 1) * n * n
    assert S.footprint(r) == 8 * (4 * n ** 3 + faces) + 48 * r.verts.shape[0] + 12 * r.tris.shape[0]


def test_candidate_estimate_bounds_the_box_cells():
    r = _req(0, 0.0, 1, N=32, s=3)
    est = S.candidate_estimate(r, slack=1.0)
    # every triangle touches at least one cell
    assert est >= r.tris.shape[0]
    # and the estimate is a bounding-box count, not a grid-wide one
    assert est < 27 * r.tris.shape[0] + 1024


def test_continuous_batching_and_budget():
    clock = FakeClock()
    ex = FakeExecutor(clock)
    one = S.footprint(_req(0, 0.0, 1))
    cap = _cap(budget=3 * one)          # at most three requests resident at once
    reqs = [_req(i, 0.005 * i, steps=3 + (i % 4)) for i in range(10)]
    outs, stats = S.serve(reqs, ex, cap, realtime=False, clock=clock)
    assert stats["completed"] == 10 and stats["rejected"] == 0
    assert stats["peak_bytes"] <= 3 * one
    assert max(len(h) for h in ex.history) == 3
    # every request ran exactly its steps, and FIFO admission order
    for r in reqs:
        o = outs[r.rid]
        assert o.steps_done == r.steps and o.cells == 10 * r.steps
        assert o.admitted >= r.arrival and o.finished > o.admitted
    adm = [outs[r.rid].admitted for r in reqs]
    assert all(a <= b for a, b in zip(adm, adm[1:]))
    # continuous batching: some request was admitted while another was running,
    # i.e. requests overlap without starting together
    overlap = any(outs[a.rid].admitted < outs[b.rid].admitted < outs[a.rid].finished
                  for a in reqs for b in reqs if a.rid != b.rid)
    assert overlap
    lat = np.array([outs[r.rid].latency for r in reqs])
    assert abs(stats["p50_ms"] - 1e3 * np.percentile(lat, 50)) < 1e-6


def test_too_large_requests_are_rejected_and_failures_isolated():
    clock = FakeClock()
    ex = FakeExecutor(clock)
    small = _req(0, 0.0, 4)
    big = _req(1, 0.0, 4, N=128)
    cap = _cap(budget=2 * S.footprint(small))
    ex.fail.add(2)
    reqs = [small, big, _req(2, 0.0, 4), _req(3, 0.0, 4)]
    outs, stats = S.serve(reqs, ex, cap, realtime=False, clock=clock)
    assert outs[1].rejected.startswith("exceeds")
    assert stats["rejected"] == 1
    assert outs[2].status == 0x02 and outs[2].steps_done == 1     # failed on its first step, released
    assert outs[0].status == 0 and outs[0].steps_done == 4
    assert outs[3].status == 0 and outs[3].steps_done == 4
    assert stats["failed"] == 1


def test_idle_server_waits_for_arrivals():
    clock = FakeClock()
    ex = FakeExecutor(clock)
    reqs = [_req(0, 0.0, 2), _req(1, 5.0, 2)]
    outs, stats = S.serve(reqs, ex, _cap(10 ** 12), realtime=False, clock=clock)
    assert outs[1].admitted >= 5.0
    assert outs[1].latency < 1.0
    assert len(ex.history) == 4


def _head_of_line_stream():
    """A large resident request, then a second large one that cannot fit until
    the first ends, then small requests arriving behind it."""
    big0 = _req(0, 0.0, 20, N=64)
    big1 = _req(1, 0.001, 5, N=64)
    smalls = [_req(2 + i, 0.002 + 0.001 * i, 2) for i in range(4)]
    budget = S.footprint(big0) + 4 * S.footprint(smalls[0])   # big1 fits only once big0 is gone
    return [big0, big1] + smalls, _cap(budget)


def test_fifo_head_of_line_blocks_small_requests():
    clock = FakeClock()
    reqs, cap = _head_of_line_stream()
    outs, _ = S.serve(reqs, FakeExecutor(clock), cap, realtime=False, clock=clock)
    # every small request waits until the second large one is admitted
    for r in reqs[2:]:
        assert outs[r.rid].admitted >= outs[1].admitted


def test_backfill_admits_small_requests_past_a_blocked_head_without_starving_it():
    clock = FakeClock()
    reqs, cap = _head_of_line_stream()
    outs, stats = S.serve(reqs, FakeExecutor(clock), cap, realtime=False, clock=clock, policy="backfill",
                          starve_s=10.0)
    assert stats["completed"] == len(reqs)
    for r in reqs[2:]:
        assert outs[r.rid].admitted < outs[1].admitted      # they passed the blocked head
        assert outs[r.rid].finished < outs[0].finished      # and finished while the first large one ran
    assert outs[1].admitted >= outs[0].finished             # the head still got in
    # with a zero starvation limit nothing passes the head: the FIFO order
    clock2 = FakeClock()
    outs2, _ = S.serve(reqs, FakeExecutor(clock2), cap, realtime=False, clock=clock2, policy="backfill",
                       starve_s=0.0)
    for r in reqs[2:]:
        assert outs2[r.rid].admitted >= outs2[1].admitted
