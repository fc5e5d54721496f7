"""Serving loop for the front/fluid coupling: continuous batching of fronts.

Requests -- a closed front, its grid, a number of time steps -- arrive over
time.  An admitted request keeps its front and its fields (alpha, force, face
velocities, vertex velocities) resident on the device until its last step.
Every iteration runs ONE time step for every active request through one batched
launch sequence of the library: binning, volume fraction, PPIC curvature, CSF
force and the RK4 advection of the vertices (each front with its own time
step), so requests that arrive while others run join the next iteration and
their work overlaps on the device with the others'.  Requests are admitted in
arrival order while their device footprint fits the memory budget and the batch
workspace's capacities (fronts, grid cells, triangles, candidate pairs); a
request that can never fit is rejected.  Latency is arrival -> end of the
iteration that ran its last step.

``Scheduler`` is the host logic alone (no GPU: tested on the CPU with a fake
executor); ``BatchExecutor`` runs the iterations on the GPU; ``serve`` drives
both against the wall clock.  ``SequentialExecutor`` is the plain comparison:
requests one after the other through the one-front entry points.
"""
from __future__ import annotations

import collections
import math
import time
from dataclasses import dataclass, field

import numpy as np


@dataclass
class Request:
    rid: int
    grid: object            # inputs.Grid
    verts: np.ndarray       # (nv, 3) float64, host
    tris: np.ndarray        # (nt, 3) int32, host
    steps: int
    arrival: float          # seconds after the start of the run
    dt: float               # time step of the RK4 advection
    centre: tuple = (0.5, 0.5, 0.5)   # face field: solid-body rotation about centre
    omega: tuple = (0.0, 0.0, 1.0)


@dataclass
class Outcome:
    rid: int
    arrival: float
    admitted: float = math.nan
    finished: float = math.nan
    steps_done: int = 0
    status: int = 0          # FT_ST_* bits seen by this front
    rejected: str = ""
    cells: int = 0           # interfacial cells over all its steps
    result: dict = field(default_factory=dict)

    @property
    def latency(self) -> float:
        return self.finished - self.arrival


def footprint(req: Request) -> int:
    """Device bytes a request holds while active: vertices (positions and
    velocities), triangles, alpha, force and the three face arrays."""
    n0, n1, n2 = (int(x) for x in req.grid.n)
    cells = n0 * n1 * n2
    faces = (n0 + 1) * n1 * n2 + n0 * (n1 + 1) * n2 + n0 * n1 * (n2 + 1)
    nv, nt = req.verts.shape[0], req.tris.shape[0]
    return 8 * (cells + 3 * cells + faces) + 48 * nv + 12 * nt


def candidate_estimate(req: Request, slack: float = 1.5) -> int:
    """Upper estimate of the (triangle, candidate cell) pairs of the front: the
    cells of each triangle's bounding box, with slack for the motion of the
    front during its steps."""
    g = req.grid
    x = req.verts[req.tris]                          # (nt, 3, 3)
    lo = (x.min(axis=1) - np.asarray(g.origin)) / g.h
    hi = (x.max(axis=1) - np.asarray(g.origin)) / g.h
    # cells whose closed extent meets the box: one more below when lo lies on a plane
    ext = np.floor(hi) - np.floor(lo) + 1.0 + (np.floor(lo) == lo)
    return int(slack * np.prod(ext, axis=1).sum()) + 1024


@dataclass
class Capacity:
    budget_bytes: int
    max_fronts: int
    max_grid_cells: int
    max_nt: int
    max_cand: int


class Scheduler:
    """Admission by device footprint and batch capacities (host only).

    policy "fifo": arrived requests are admitted in arrival order and the queue
    head blocks the ones behind it.  policy "backfill": a request behind a head
    that does not fit yet is admitted if it fits, so that small requests do not
    wait behind a large one for memory it cannot use yet; once the head has
    waited `starve_s` seconds nothing passes it any more, so that it is not
    starved."""

    def __init__(self, cap: Capacity, policy: str = "fifo", starve_s: float = 1.0):
        if policy not in ("fifo", "backfill"):
            raise ValueError(f"unknown admission policy {policy!r}")
        self.cap = cap
        self.policy = policy
        self.starve_s = starve_s
        self.pending = collections.deque()
        self.active = []           # requests being served
        self.left = {}             # rid -> steps left
        self.outcomes = {}
        self.used = dict(bytes=0, fronts=0, cells=0, nt=0, cand=0)
        self.peak_bytes = 0
        self._need = {}

    def submit(self, req: Request):
        self.outcomes[req.rid] = Outcome(req.rid, req.arrival)
        need = dict(bytes=footprint(req), fronts=1, cells=int(req.grid.ncells), nt=int(req.tris.shape[0]),
                    cand=candidate_estimate(req))
        c = self.cap
        limits = dict(bytes=c.budget_bytes, fronts=c.max_fronts, cells=c.max_grid_cells, nt=c.max_nt,
                      cand=c.max_cand)
        too_big = [k for k in need if need[k] > limits[k]]
        if too_big:
            self.outcomes[req.rid].rejected = "exceeds " + ",".join(too_big)
            return
        self._need[req.rid] = need
        self.pending.append(req)

    def _fits(self, need) -> bool:
        c = self.cap
        u = self.used
        return (u["bytes"] + need["bytes"] <= c.budget_bytes and u["fronts"] + 1 <= c.max_fronts
                and u["cells"] + need["cells"] <= c.max_grid_cells and u["nt"] + need["nt"] <= c.max_nt
                and u["cand"] + need["cand"] <= c.max_cand)

    def _take(self, req, now):
        need = self._need[req.rid]
        for k in self.used:
            self.used[k] += need[k]
        self.peak_bytes = max(self.peak_bytes, self.used["bytes"])
        self.active.append(req)
        self.left[req.rid] = req.steps
        self.outcomes[req.rid].admitted = now

    def admit(self, now: float):
        """Requests that have arrived by `now` and fit, in arrival order; under
        "fifo" the queue head blocks the ones behind it, under "backfill" the
        ones behind it that fit pass it (until it has waited starve_s)."""
        out = []
        while self.pending and self.pending[0].arrival <= now:
            req = self.pending[0]
            if not self._fits(self._need[req.rid]):
                break
            self.pending.popleft()
            self._take(req, now)
            out.append(req)
        if self.policy == "backfill" and self.pending and self.pending[0].arrival <= now:
            head = self.pending[0]
            if now - head.arrival < self.starve_s:
                keep = collections.deque([head])
                for req in list(self.pending)[1:]:
                    if req.arrival <= now and self._fits(self._need[req.rid]):
                        self._take(req, now)
                        out.append(req)
                    else:
                        keep.append(req)
                self.pending = keep
        return out

    def step_done(self, now: float, cells: dict, status: dict):
        """After an iteration: every active request advanced one step; returns
        the requests that finished (or failed) and releases their resources."""
        done = []
        for req in list(self.active):
            o = self.outcomes[req.rid]
            o.steps_done += 1
            o.cells += int(cells.get(req.rid, 0))
            o.status |= int(status.get(req.rid, 0))
            self.left[req.rid] -= 1
            if self.left[req.rid] <= 0 or o.status:
                o.finished = now
                done.append(req)
        for req in done:
            self.active.remove(req)
            need = self._need.pop(req.rid)
            for k in self.used:
                self.used[k] -= need[k]
            del self.left[req.rid]
        return done

    def next_arrival(self):
        return self.pending[0].arrival if self.pending else None

    def idle(self) -> bool:
        return not self.pending and not self.active


def device_faces(grid, centre, omega, device):
    """Solid-body rotation u = omega x (x - c) at the face centres, on the device."""
    import torch
    out = []
    c = [float(x) for x in centre]
    w = [float(x) for x in omega]
    for ax in range(3):
        n = [int(x) for x in grid.n]
        n[ax] += 1
        xs = [grid.origin[d] + grid.h * (torch.arange(n[d], device=device, dtype=torch.float64)
                                          + (0.0 if d == ax else 0.5)) - c[d] for d in range(3)]
        X, Y, Z = torch.meshgrid(*xs, indexing="ij")
        u = (w[1] * Z - w[2] * Y, w[2] * X - w[0] * Z, w[0] * Y - w[1] * X)[ax]
        out.append(u.contiguous())
    return out


class BatchExecutor:
    """Runs one time step of every active request per iteration through the
    batched entry points.  Each request's front and fields stay on the device
    from admission to its last step."""

    def __init__(self, cap: Capacity, params, device: int = 0, keep_results: bool = False):
        import torch
        from . import _front as F
        self.F = F
        self.torch = torch
        self.dev = torch.device("cuda", device)
        self.params = params
        # interfacial cells are far fewer than candidate pairs (each cell holds several)
        M = cap.max_cand // 2 + 1024
        self.ws = F.BatchWorkspace(cap.max_fronts, cap.max_grid_cells, cap.max_nt, max_cand=cap.max_cand,
                                   max_cells=M, device=device)
        self.cell_keys = torch.empty(M, dtype=torch.int32, device=self.dev)
        self.kappa = torch.empty(M, dtype=torch.float64, device=self.dev)
        self.normal = torch.empty((M, 3), dtype=torch.float64, device=self.dev)
        self.fit_status = torch.empty(M, dtype=torch.int8, device=self.dev)
        self.off = torch.empty(cap.max_fronts + 1, dtype=torch.int64, device=self.dev)
        self.res = {}           # rid -> resident device state
        self.order = []         # rids in table order
        self.dirty = True
        self.keep_results = keep_results
        self.iter_cells = 0

    def admit(self, req: Request):
        torch = self.torch
        g = req.grid
        verts = torch.from_numpy(np.ascontiguousarray(req.verts)).to(self.dev)
        U, V, W = device_faces(g, req.centre, req.omega, self.dev)
        self.res[req.rid] = dict(grid=g, verts=verts, tris=torch.from_numpy(np.ascontiguousarray(req.tris)).to(self.dev),
                                 alpha=torch.empty(g.ncells, dtype=torch.float64, device=self.dev),
                                 force=torch.empty(3 * g.ncells, dtype=torch.float64, device=self.dev),
                                 U=U, V=V, W=W, vel=torch.empty_like(verts), verts_next=verts, dt=req.dt)
        self.order.append(req.rid)
        self.dirty = True

    def release(self, rid):
        self.res.pop(rid)
        self.order.remove(rid)
        self.dirty = True

    def iterate(self):
        """One time step of every active front; returns ({rid: cells}, {rid: status})."""
        F, torch = self.F, self.torch
        if self.dirty:
            self.ws.set_fronts([self.res[r] for r in self.order])
            self.dirty = False
        p, ws = self.params, self.ws
        F.front_bin_batch(ws, p)
        F.front_volume_fraction_batch(ws)
        F.front_curvature_ppic(ws, p, self.cell_keys, self.kappa, self.normal, None, self.fit_status)
        F.front_csf_force_batch(ws, p, self.kappa, self.normal)
        F.ft_batch_cell_ranges(ws, self.off)
        F.front_advect_rk4_batch(ws)
        off = self.off[:len(self.order) + 1].cpu().numpy()      # synchronizes the stream
        st = ws.front_status()
        bits = ws.status()
        if bits & 0x01:
            raise RuntimeError("batch workspace capacity exceeded: the admission estimate was too small")
        cells = {r: int(off[i + 1] - off[i]) for i, r in enumerate(self.order)}
        status = {r: st[i] for i, r in enumerate(self.order)}
        if self.keep_results:
            for i, r in enumerate(self.order):
                s = self.res[r]
                lo, hi = int(off[i]), int(off[i + 1])
                s["last"] = dict(alpha=s["alpha"].clone(), force=s["force"].clone(),
                                 kappa=self.kappa[lo:hi].clone(), normal=self.normal[lo:hi].clone())
        self.iter_cells += sum(cells.values())
        return cells, status

    def result(self, rid) -> dict:
        s = self.res[rid]
        out = dict(verts=s["verts"].cpu().numpy())
        if "last" in s:
            out.update({k: v.cpu().numpy() for k, v in s["last"].items()})
        return out

    def close(self):
        self.ws.close()


def serve(requests, executor, cap: Capacity, realtime: bool = True, keep_results: bool = False,
          clock=time.perf_counter, policy: str = "fifo", starve_s: float = 1.0):
    """Serve the requests (arrival times relative to the start) and return
    (outcomes by rid, stats).  With realtime=False arrivals are taken as
    already due whenever the server is idle (a closed-loop replay).  policy and
    starve_s: the admission rule of Scheduler."""
    sch = Scheduler(cap, policy=policy, starve_s=starve_s)
    for r in sorted(requests, key=lambda r: (r.arrival, r.rid)):
        sch.submit(r)
    t0 = clock()
    iters = 0
    busy = 0.0
    while not sch.idle():
        now = clock() - t0
        for req in sch.admit(now):
            executor.admit(req)
        if not sch.active:
            nxt = sch.next_arrival()
            if nxt is None:
                break
            if realtime:
                time.sleep(max(0.0, nxt - (clock() - t0)))
            else:
                t0 -= max(0.0, nxt - now)   # jump the clock to the next arrival
            continue
        a = clock()
        cells, status = executor.iterate()
        busy += clock() - a
        iters += 1
        now = clock() - t0
        for req in sch.step_done(now, cells, status):
            if keep_results:
                sch.outcomes[req.rid].result = executor.result(req.rid)
            executor.release(req.rid)
    wall = clock() - t0
    done = [o for o in sch.outcomes.values() if not o.rejected and not math.isnan(o.finished)]
    lat = np.array([o.latency for o in done]) if done else np.zeros(1)
    cells = sum(o.cells for o in done)
    stats = dict(requests=len(requests), completed=len(done),
                 rejected=sum(1 for o in sch.outcomes.values() if o.rejected),
                 failed=sum(1 for o in done if o.status), iterations=iters,
                 p50_ms=round(1e3 * float(np.percentile(lat, 50)), 3),
                 p99_ms=round(1e3 * float(np.percentile(lat, 99)), 3),
                 cells=int(cells), wall_s=round(wall, 4), busy_s=round(busy, 4),
                 cells_per_s=round(cells / wall, 1) if wall > 0 else 0.0,
                 peak_bytes=int(sch.peak_bytes))
    return sch.outcomes, stats


class SequentialExecutor:
    """The plain comparison: one request at a time through the one-front entry
    points (no batching), all its steps back to back."""

    def __init__(self, params, device: int = 0, keep_results: bool = False):
        import torch
        from . import _front as F
        self.F, self.torch = F, torch
        self.dev = torch.device("cuda", device)
        self.params = params
        self.device = device
        self.keep_results = keep_results

    def run(self, req: Request) -> tuple:
        """All steps of one request; returns (cells, status, result)."""
        F, torch = self.F, self.torch
        g = req.grid
        verts = torch.from_numpy(np.ascontiguousarray(req.verts)).to(self.dev)
        tris = torch.from_numpy(np.ascontiguousarray(req.tris)).to(self.dev)
        U, V, W = device_faces(g, req.centre, req.omega, self.dev)
        fc = F.FrontCoupling(g, max(1, tris.shape[0]), max(1, verts.shape[0]),
                             max_cand=candidate_estimate(req), params=self.params, device=self.device)
        cells = 0
        status = 0
        for _ in range(req.steps):
            fc.step(verts, tris, (U, V, W))
            F.front_advect_rk4(g, U, V, W, verts, req.dt, verts)
            cells += fc.ws.counts()["M"]
            status |= fc.ws.status()
            if status:
                break
        res = {}
        if self.keep_results:
            M = fc.ws.counts()["M"]
            res = dict(verts=verts.cpu().numpy(), alpha=fc.alpha.cpu().numpy(), force=fc.force.cpu().numpy(),
                       kappa=fc.kappa[:M].cpu().numpy(), normal=fc.normal[:M].cpu().numpy())
        fc.ws.close()
        return cells, status, res


def serve_sequential(requests, executor: SequentialExecutor, realtime: bool = True, clock=time.perf_counter):
    """The same request stream served one request at a time (FIFO)."""
    t0 = clock()
    outcomes = {}
    for req in sorted(requests, key=lambda r: (r.arrival, r.rid)):
        now = clock() - t0
        if now < req.arrival:
            if realtime:
                time.sleep(req.arrival - now)
            else:
                t0 -= req.arrival - now
        o = Outcome(req.rid, req.arrival, admitted=clock() - t0)
        o.cells, o.status, o.result = executor.run(req)
        o.steps_done = req.steps
        o.finished = clock() - t0
        outcomes[req.rid] = o
    wall = clock() - t0
    lat = np.array([o.latency for o in outcomes.values()])
    cells = sum(o.cells for o in outcomes.values())
    return outcomes, dict(requests=len(requests), completed=len(outcomes),
                          p50_ms=round(1e3 * float(np.percentile(lat, 50)), 3),
                          p99_ms=round(1e3 * float(np.percentile(lat, 99)), 3),
                          cells=int(cells), wall_s=round(wall, 4),
                          cells_per_s=round(cells / wall, 1) if wall > 0 else 0.0)
