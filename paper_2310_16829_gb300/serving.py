"""Continuous-batching request loop over the LMA C-ABI (serving the Sec. 4.2.6 use case).

Requests:
  * ``EditRequest``: change one atomic column of the resident specimen (remove it or
    give it another species, every slice), then image the probe region around it. Only
    the exit waves whose windows meet the changed pixels are re-propagated (Sec. 4.2.6).
    Edits accumulate on the resident specimen in arrival order.
  * ``ImageRequest``: a full image of a specimen built from a seeded configuration
    (its own frozen-phonon draw), propagated and read out from scratch.

Scheduling. Each request class maps to a lane; a lane owns instances, and an instance
is a worker thread with its own library context, CUDA stream, specimen and basis (one
context per host thread, as the library requires). Instances of different lanes share
no mutable state, so their kernels overlap on the device. The dispatcher admits
queued requests in arrival order per lane as soon as an instance of that lane is idle,
or, if none is, as soon as a new instance fits the HBM budget (instances reserve their
measured device footprint: exit waves, transmission, tables). A blocked lane does not
hold back the others. Results are bitwise independent of the mix: kernels are
deterministic and lanes share nothing.

Warm pool. A lane may ask for ``min_instances`` instances that the server brings up
and warms (one request's worth of device allocation and work) before it admits any
request. Device allocation can synchronize the whole device, so an instance created
while other lanes' kernels are in flight would stall every lane once; with a warm pool
that only happens when load grows past the pool.

Hardware queues. The device runs CUDA_DEVICE_MAX_CONNECTIONS hardware work queues per
process (8 unless set); streams beyond that share queues, and a kernel queued behind
another stream's kernels in its queue cannot start before them (an edit then waits for a
full image although its stream has priority). The environment variable has to be set
before CUDA initializes; the server warns when it is below the number of instances + 1.

This module holds host logic only; every computation runs in the CUDA library.
"""
from __future__ import annotations

import os
import queue
import threading
import time
import warnings
from dataclasses import dataclass
from typing import Callable, Dict, List, Optional

import numpy as np


@dataclass
class EditRequest:
    cx: float
    cy: float
    op: int               # LMA_EDIT_REMOVE / LMA_EDIT_SET_SPECIES
    species: int = 0
    region_probes: int = 64
    r_site: float = 0.5
    lane: str = "edit"


@dataclass
class ImageRequest:
    lane: str             # e.g. "full_256"
    seed: int


@dataclass
class Result:
    request: object
    image: Optional[np.ndarray]
    error: Optional[BaseException]
    t_arrival: float
    t_start: float
    t_done: float
    instance: int
    n_stale: int = 0

    @property
    def latency(self) -> float:
        return self.t_done - self.t_arrival


class Ticket:
    """Completion handle of one request."""

    def __init__(self):
        self._ev = threading.Event()
        self.result: Optional[Result] = None

    def set(self, r: Result):
        self.result = r
        self._ev.set()

    def wait(self, timeout: Optional[float] = None) -> Result:
        if not self._ev.wait(timeout):
            raise TimeoutError("request did not complete in time")
        return self.result


class Instance:
    """A worker: thread + context + stream + resources of one lane."""

    def __init__(self, lane: "Lane", index: int, reserve_bytes: int, warm: bool = False):
        self.lane = lane
        self.index = index
        self.reserve_bytes = reserve_bytes
        self.busy = False
        self.jobs: "queue.Queue" = queue.Queue()
        self.state = None
        self.warm = warm
        self.ready = threading.Event()
        self.error: Optional[BaseException] = None
        self.thread = threading.Thread(target=self._run, daemon=True)
        self.thread.start()

    def _run(self):
        try:
            self.state = self.lane.make_state()
            if self.warm and self.lane.warm is not None:
                self.lane.warm(self.state)
        except BaseException as e:   # reported by Server.__init__
            self.error = e
        self.ready.set()
        while True:
            job = self.jobs.get()
            if job is None:
                break
            req, ticket, t_arr, done = job
            t0 = time.perf_counter()
            img, err, n_stale = None, None, 0
            try:
                img, n_stale = self.lane.handle(self.state, req)
            except BaseException as e:   # a failing request must not stop the server
                err = e
            ticket.set(Result(req, img, err, t_arr, t0, time.perf_counter(), self.index, n_stale))
            done(self)
        self.lane.close_state(self.state)


class Lane:
    """A request class: how to build an instance's state and how to serve a request."""

    def __init__(self, name: str, make_state: Callable, handle: Callable, close_state: Callable,
                 reserve_bytes: int, max_instances: int = 1 << 30, min_instances: int = 0,
                 warm: Optional[Callable] = None):
        self.name = name
        self.make_state = make_state
        self.handle = handle
        self.close_state = close_state
        self.reserve_bytes = reserve_bytes
        self.max_instances = max_instances
        self.min_instances = min(min_instances, max_instances)
        self.warm = warm
        self.instances: List[Instance] = []


class Server:
    """Continuous batching: admission by idle instance or HBM budget, per-lane FIFO."""

    def __init__(self, lanes: List[Lane], budget_bytes: int, warm_timeout: float = 600.0):
        self.lanes: Dict[str, Lane] = {l.name: l for l in lanes}
        self.budget = budget_bytes
        self.reserved = 0
        self.pending: Dict[str, List] = {l.name: [] for l in lanes}
        self.cv = threading.Condition()
        self.closed = False
        self.admissions: List[tuple] = []          # (time, lane, instance, queued behind)
        # warm pool: brought up before any request is admitted, within the budget
        for lane in lanes:
            while (len(lane.instances) < lane.min_instances and
                   self.reserved + lane.reserve_bytes <= self.budget):
                lane.instances.append(Instance(lane, len(lane.instances), lane.reserve_bytes, warm=True))
                self.reserved += lane.reserve_bytes
        queues = int(os.environ.get("CUDA_DEVICE_MAX_CONNECTIONS", "8"))
        wanted = sum(l.max_instances for l in lanes if l.max_instances < (1 << 20)) + 1
        if queues < wanted:
            warnings.warn(f"CUDA_DEVICE_MAX_CONNECTIONS={queues} is below {wanted} streams: lanes may "
                          "wait for each other's kernels in shared hardware queues")
        for lane in lanes:
            for inst in lane.instances:
                if not inst.ready.wait(warm_timeout):
                    raise TimeoutError(f"lane {lane.name}: instance {inst.index} not ready")
                if inst.error is not None:
                    raise inst.error
        self.dispatcher = threading.Thread(target=self._dispatch, daemon=True)
        self.dispatcher.start()

    # -- public -----------------------------------------------------------------
    def submit(self, req) -> Ticket:
        t = Ticket()
        with self.cv:
            if req.lane not in self.lanes:
                raise KeyError(f"no lane {req.lane!r}")
            self.pending[req.lane].append((req, t, time.perf_counter()))
            self.cv.notify_all()
        return t

    def close(self):
        with self.cv:
            self.closed = True
            self.cv.notify_all()
        self.dispatcher.join()
        for lane in self.lanes.values():
            for inst in lane.instances:
                inst.jobs.put(None)
            for inst in lane.instances:
                inst.thread.join()

    # -- dispatcher -------------------------------------------------------------
    def _done(self, inst: Instance):
        with self.cv:
            inst.busy = False
            self.cv.notify_all()

    def _try_admit(self, lane: Lane) -> bool:
        q = self.pending[lane.name]
        if not q:
            return False
        inst = next((i for i in lane.instances if not i.busy), None)
        if inst is None:
            if (len(lane.instances) < lane.max_instances and
                    self.reserved + lane.reserve_bytes <= self.budget):
                inst = Instance(lane, len(lane.instances), lane.reserve_bytes)
                lane.instances.append(inst)
                self.reserved += lane.reserve_bytes
            else:
                return False
        req, ticket, t_arr = q.pop(0)
        inst.busy = True
        self.admissions.append((time.perf_counter(), lane.name, inst.index, len(q)))
        inst.jobs.put((req, ticket, t_arr, self._done))
        return True

    def _dispatch(self):
        with self.cv:
            while True:
                progressed = True
                while progressed:
                    progressed = False
                    for lane in self.lanes.values():
                        while self._try_admit(lane):
                            progressed = True
                if self.closed and not any(self.pending.values()):
                    return
                self.cv.wait(timeout=0.05)


# ------------------------------------------------------------------------------------
# lanes over the CUDA library
# ------------------------------------------------------------------------------------

def _stream(priority: int = 0):
    """A CUDA stream for one instance; edits use the highest priority so that their
    small launches are scheduled ahead of full-image launches already queued."""
    import torch
    return torch.cuda.Stream(priority=priority)


def edit_lane(workload, device: int = 0, max_instances: int = 1, min_instances: int = 0) -> Lane:
    """Resident specimen: all exit waves propagated once, edits re-propagate locally."""
    from . import lma

    def make():
        ctx = lma.Context(device)
        spec = lma.Specimen(ctx, workload.grid, workload.potential, workload.phonons)
        basis = lma.Basis(ctx, spec, workload.probe, workload.basis)
        import torch
        st = _stream(torch.cuda.Stream.priority_range()[1])
        basis.propagate(0, stream=st)
        basis.image(workload.detectors, workload.region, stream=st)
        return {"ctx": ctx, "spec": spec, "basis": basis, "stream": st, "w": workload}

    def handle(s, req: EditRequest):
        w = s["w"]
        dx = w.grid.lx / w.grid.nx
        sx, sy = w.region.spacing_px
        n = req.region_probes
        px = int(round(req.cx / dx)) // sx * sx
        py = int(round(req.cy / dx)) // sy * sy
        from .workloads import Region
        region = Region(px - (n // 2) * sx, py - (n // 2) * sy, n, n, (sx, sy))
        _, n_stale = s["spec"].edit_column(s["basis"], req.cx, req.cy, req.r_site, req.op, req.species)
        img = s["basis"].image(w.detectors, region, stream=s["stream"])
        return img, n_stale

    def close(s):
        s["basis"].close()
        s["spec"].close()
        s["ctx"].close()

    reserve = _footprint(workload)
    # make() already propagates every exit wave and images the region: no extra warm-up
    return Lane("edit", make, handle, close, reserve, max_instances, min_instances, warm=lambda s: None)


def image_lane(name: str, build: Callable[[int], object], device: int = 0,
               max_instances: int = 4, min_instances: int = 0, max_resident: Optional[int] = None) -> Lane:
    """Fresh specimens of one size: each request uploads its own seeded atoms
    (lma_specimen_set_atoms) and computes the full image from scratch. With max_resident
    the image is computed part by part in a store of that many exit waves (Sec. 4.2.4),
    using the partition strategy with the fewest Multislice runs for the lane's region."""
    from . import lma
    proto = build(0)

    def make():
        ctx = lma.Context(device)
        spec = lma.Specimen(ctx, proto.grid, proto.potential, proto.phonons)
        basis = lma.Basis(ctx, spec, proto.probe, proto.basis)
        state = {"ctx": ctx, "spec": spec, "basis": basis, "stream": _stream(), "strategy": None}
        if max_resident:
            runs = {st: basis.partition(proto.region, st, max_resident)[2]
                    for st in (lma.LMA_PART_ROWS, lma.LMA_PART_RECTANGLES, lma.LMA_PART_GREEDY)}
            state["strategy"] = min(runs, key=runs.get)
        return state

    def handle(s, req: ImageRequest):
        w = build(req.seed)
        s["spec"].set_atoms(w.phonons)
        if max_resident:
            img = s["basis"].image_partitioned(w.detectors, w.region, s["strategy"], max_resident,
                                               stream=s["stream"])
        else:
            img = s["basis"].image(w.detectors, w.region, recompute=True, stream=s["stream"])
        return img, 0

    def close(s):
        s["basis"].close()
        s["spec"].close()
        s["ctx"].close()

    def warm(s):
        handle(s, ImageRequest(name, seed=0))
        s["stream"].synchronize()

    return Lane(name, make, handle, close, _footprint(proto, max_resident), max_instances, min_instances, warm)


def _translates(w) -> int:
    return (w.grid.nx // w.basis.in_spacing_px[0] // w.basis.f) * (w.grid.ny // w.basis.in_spacing_px[1] // w.basis.f)


def _footprint(w, max_resident: Optional[int] = None) -> int:
    """Device bytes an instance holds: exit-wave store (|I_f| waves, or max_resident of a
    partitioned store), padded transmission, tables."""
    W = w.basis.window
    nT = _translates(w)
    waves = min(nT, max_resident) if max_resident else nT
    store = waves * W * W * (4 if getattr(w.basis, "precision", 0) else 8)
    t = w.grid.n_slices * (w.grid.nx + W) * (w.grid.ny + W) * 8
    probes = w.region.npx * w.region.npy
    tables = probes * w.basis.L * 20 + probes * 8 * len(w.detectors) + nT * 4
    return int(store + t + tables + (16 << 20))


def fit_max_resident(w, budget_bytes: int) -> Optional[int]:
    """None when an instance with the full exit-wave store fits budget_bytes; else the
    largest store (in exit waves, a multiple of 256, at least L) whose instance fits, which
    makes the lane compute its images part by part (Sec. 4.2.4). Raises when even an
    L-wave store does not fit."""
    if _footprint(w) <= budget_bytes:
        return None
    lo, hi = w.basis.L, _translates(w)
    if _footprint(w, lo) > budget_bytes:
        raise ValueError("the budget does not hold even L exit waves")
    while hi - lo > 1:
        mid = (lo + hi) // 2
        if _footprint(w, mid) <= budget_bytes:
            lo = mid
        else:
            hi = mid
    return max(w.basis.L, lo // 256 * 256) if lo >= 256 else lo


def poisson_arrivals(n: int, rate: float, seed: int) -> np.ndarray:
    """Seeded arrival times (s) of a Poisson stream."""
    rng = np.random.default_rng(seed)
    return np.cumsum(rng.exponential(1.0 / rate, size=n))


def run_stream(server: Server, requests: List, arrivals: np.ndarray,
               timeout: float = 600.0) -> List[Result]:
    """Submit requests at their arrival times (relative to now); wait for all results."""
    t0 = time.perf_counter()
    tickets = []
    for req, ta in zip(requests, arrivals):
        delay = t0 + ta - time.perf_counter()
        if delay > 0:
            time.sleep(delay)
        tickets.append(server.submit(req))
    return [t.wait(timeout) for t in tickets]


def latency_summary(results: List[Result]) -> dict:
    lat = np.array([r.latency for r in results]) * 1e3
    out = {"requests": len(results), "p50_ms": float(np.percentile(lat, 50)),
           "p99_ms": float(np.percentile(lat, 99)), "mean_ms": float(lat.mean()),
           "errors": sum(r.error is not None for r in results)}
    by = {}
    for r in results:
        by.setdefault(r.request.lane, []).append(r.latency * 1e3)
    out["by_lane"] = {k: {"n": len(v), "p50_ms": float(np.percentile(v, 50)),
                          "p99_ms": float(np.percentile(v, 99))} for k, v in by.items()}
    # where the time went: waiting for an instance, or being served
    for k in out["by_lane"]:
        rs = [r for r in results if r.request.lane == k]
        q = np.array([r.t_start - r.t_arrival for r in rs]) * 1e3
        sv = np.array([r.t_done - r.t_start for r in rs]) * 1e3
        out["by_lane"][k].update({"queue_p99_ms": float(np.percentile(q, 99)),
                                  "service_p50_ms": float(np.percentile(sv, 50)),
                                  "service_p99_ms": float(np.percentile(sv, 99))})
    return out
