"""Host logic of the continuous-batching loop, with fake lanes (no GPU).

Failure detection and admission are exercised on the host: a request that raises,
a budget that admits fewer instances than there are requests, and lanes that must
not block each other.
"""
import threading
import time

import numpy as np
import pytest

from paper_2310_16829_gb300 import serving as S


class Req:
    def __init__(self, lane, k, dur=0.02, fail=False):
        self.lane, self.k, self.dur, self.fail = lane, k, dur, fail


def fake_lane(name, reserve, max_instances=8, log=None):
    lock = threading.Lock()
    active = {"n": 0, "max": 0}

    def make():
        return {"name": name}

    def handle(state, req):
        with lock:
            active["n"] += 1
            active["max"] = max(active["max"], active["n"])
        if log is not None:
            log.append((name, req.k, time.perf_counter()))
        time.sleep(req.dur)
        with lock:
            active["n"] -= 1
        if req.fail:
            raise RuntimeError(f"request {req.k} failed")
        return np.full((1, 2, 2), float(req.k)), 0

    lane = S.Lane(name, make, handle, lambda s: None, reserve, max_instances)
    lane.active = active
    return lane


def test_budget_limits_instances_and_results_complete():
    a = fake_lane("a", reserve=10)
    srv = S.Server([a], budget_bytes=25)          # room for two instances
    tickets = [srv.submit(Req("a", k, dur=0.05)) for k in range(6)]
    res = [t.wait(10) for t in tickets]
    srv.close()
    assert len(a.instances) == 2 and a.active["max"] == 2
    assert [float(r.image[0, 0, 0]) for r in res] == list(range(6))
    assert srv.reserved == 20 <= srv.budget


def test_fifo_per_lane_and_lanes_do_not_block_each_other():
    log = []
    slow = fake_lane("slow", reserve=10, max_instances=1, log=log)
    fast = fake_lane("fast", reserve=10, max_instances=1, log=log)
    srv = S.Server([slow, fast], budget_bytes=100)
    t_slow = [srv.submit(Req("slow", k, dur=0.2)) for k in range(3)]
    t_fast = [srv.submit(Req("fast", k, dur=0.01)) for k in range(5)]
    rf = [t.wait(10) for t in t_fast]
    rs = [t.wait(10) for t in t_slow]
    srv.close()
    assert [e[1] for e in log if e[0] == "slow"] == [0, 1, 2]
    assert [e[1] for e in log if e[0] == "fast"] == [0, 1, 2, 3, 4]
    # every fast request finished before the second slow one started
    assert max(r.t_done for r in rf) < rs[1].t_start


def test_failing_request_reports_error_and_server_continues():
    a = fake_lane("a", reserve=1)
    srv = S.Server([a], budget_bytes=10)
    t_bad = srv.submit(Req("a", 1, fail=True))
    t_ok = srv.submit(Req("a", 2))
    bad, ok = t_bad.wait(10), t_ok.wait(10)
    srv.close()
    assert isinstance(bad.error, RuntimeError) and bad.image is None
    assert ok.error is None and float(ok.image[0, 0, 0]) == 2.0


def test_unknown_lane_is_rejected_and_waiting_times_out():
    a = fake_lane("a", reserve=50)
    srv = S.Server([a], budget_bytes=10)          # no instance ever fits
    with pytest.raises(KeyError):
        srv.submit(Req("b", 0))
    t = srv.submit(Req("a", 0))
    with pytest.raises(TimeoutError):
        t.wait(0.3)
    srv.pending["a"].clear()
    srv.close()


def test_poisson_arrivals_are_seeded():
    a = S.poisson_arrivals(100, 10.0, 4)
    assert np.array_equal(a, S.poisson_arrivals(100, 10.0, 4))
    assert abs(np.mean(np.diff(a)) - 0.1) < 0.03 and np.all(np.diff(a) > 0)


def test_warm_pool_is_ready_before_admission_and_within_budget():
    warmed = []
    a = fake_lane("a", reserve=10, max_instances=4)
    a.min_instances = 3
    a.warm = lambda state: warmed.append(time.perf_counter())
    srv = S.Server([a], budget_bytes=25)            # the budget admits two of the three
    t0 = time.perf_counter()
    assert len(a.instances) == 2 and len(warmed) == 2 and srv.reserved == 20
    assert all(w < t0 for w in warmed)
    res = [srv.submit(Req("a", k, dur=0.01)).wait(10) for k in range(4)]
    srv.close()
    assert [float(r.image[0, 0, 0]) for r in res] == [0.0, 1.0, 2.0, 3.0]
    assert len(a.instances) == 2


def test_warm_failure_is_reported_at_start():
    a = fake_lane("a", reserve=1)
    a.min_instances = 1

    def bad_warm(state):
        raise RuntimeError("warm-up failed")

    a.warm = bad_warm
    with pytest.raises(RuntimeError, match="warm-up failed"):
        S.Server([a], budget_bytes=10)


def test_fit_max_resident_bounds_the_store_to_the_budget():
    from paper_2310_16829_gb300 import workloads as WL
    w = WL.perovskite_workload(cells=20, nx=1024, n_slices=100, n_phonons=1, probes=256)
    full = S._footprint(w)
    assert S.fit_max_resident(w, full) is None
    for frac in (0.9, 0.5, 0.2):
        budget = int(full * frac)
        M = S.fit_max_resident(w, budget)
        assert M is not None and M % 256 == 0 and w.basis.L <= M < S._translates(w)
        assert S._footprint(w, M) <= budget < S._footprint(w, M + 256)
    with pytest.raises(ValueError):
        S.fit_max_resident(w, 1 << 20)
