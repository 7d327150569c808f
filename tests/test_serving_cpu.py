"""Host logic of the continuous-batching server, with the device faked.

The scheduler decides admission (arrival, free slot, free HBM or an idle
pooled context), the number of steps per tick (never past the nearest
completion), the readout of completed requests and the re-use of their
contexts; none of that needs a GPU, so the server's device-facing steps are
replaced by a fake device that counts steps, keeps batch membership and free
memory, and advances a fake clock with the work.
"""
import collections

import numpy as np
import pytest

import paper_2302_04741_gb300 as lbm
from paper_2302_04741_gb300 import serving, workloads as W


class FakeSim:
    def __init__(self, w):
        self.w = w
        self.ctx = self
        self.steps = 0
        self.users = []


class FakeEvent:
    def __init__(self, t):
        self.t = t


class FakeServer(serving.Server):
    """The real scheduler (run) over a fake device."""

    def __init__(self, free_bytes, max_slots, tick_steps, reserve=0, seconds_per_update=1e-10):
        self.precision, self.force_order, self.lattice = W.FP32_SHIFTED, 2, W.D3Q39
        self.max_slots, self.hbm_reserve, self.tick_steps = max_slots, reserve, tick_steps
        self.collect = ("rho", "u", "T", "q")
        self.free = free_bytes
        self.spu = seconds_per_update
        self.t = 0.0
        self.members = []
        self.launches = []
        self._setup()

    def clock(self):
        return self.t

    def _fits(self, req):
        if self.pool[tuple(req.workload["shape"])]:
            return True
        return self.free - serving.request_bytes(req.workload, self.precision) >= self.hbm_reserve

    def _context(self, req):
        idle = self.pool[tuple(req.workload["shape"])]
        if idle:
            sim = idle.pop()
        else:
            sim = FakeSim(req.workload)
            self.contexts.append(sim)
            self.free -= serving.request_bytes(req.workload, self.precision)
        sim.steps = 0  # lbm_init resets the step count
        sim.users.append(req.id)
        return sim

    def _start(self, req):
        assert req.sim not in self.members
        self.members.append(req.sim)

    def _tick(self, n, lups):
        assert self.members, "a tick with no resident grid"
        self.launches.append((n, len(self.members)))
        for m in self.members:
            m.steps += n
        self.t += n * sum(int(np.prod(m.w["shape"])) for m in self.members) * self.spu
        self.ticks.append((n, lups, self.t, None))
        return FakeEvent(self.t)

    def _readout(self, req):
        self.members.remove(req.sim)
        self.pool[tuple(req.workload["shape"])].append(req.sim)
        return serving.Readout(req, None, FakeEvent(self.t))

    def _ready(self, rd):
        return True

    def _wait(self, event):
        pass

    def _collect(self, rd):
        n = rd.req.sites
        return {"rho": np.ones(n), "u": np.zeros((3, n)), "T": np.ones(n), "q": np.zeros((3, n)),
                "steps": rd.req.sim.steps}

    def _busy_seconds(self):
        return self.t


@pytest.fixture(autouse=True)
def fake_step_count(monkeypatch):
    monkeypatch.setattr(lbm, "lbm_step_count", lambda ctx: ctx.steps)


def fake_sleep(srv, monkeypatch):
    monkeypatch.setattr(serving.time, "sleep", lambda s: setattr(srv, "t", srv.t + s))


def trace(n, seed=4, rate=50.0, sides=(32, 48)):
    return W.serving_trace(n_requests=n, rate=rate, seed=seed, sides=sides, steps_range=(50, 400))


@pytest.mark.parametrize("max_slots,tick", [(1, 100), (4, 64), (64, 1000)])
def test_every_request_finishes_with_its_exact_step_count(monkeypatch, max_slots, tick):
    srv = FakeServer(1 << 40, max_slots, tick)
    fake_sleep(srv, monkeypatch)
    reqs = serving.requests_from_trace(trace(30))
    stats = srv.run(reqs, clock=srv.clock)
    assert stats["requests"] == 30
    for r in reqs:
        assert r.sim is None and r.done is not None and r.done >= r.arrival
        assert r.admitted >= r.arrival
        assert {"rho", "u", "T", "q"} <= set(r.result)
        # no overshoot: the grid stopped exactly at its step count
        assert r.result["steps"] == r.steps
    # ticks never exceed the limit, and the resident count never the slots
    assert all(1 <= n <= tick for n, _ in srv.launches)
    assert all(k <= max_slots for _, k in srv.launches)
    assert stats["max_resident"] <= max_slots
    assert stats["lattice_updates"] == sum(r.sites * r.steps for r in reqs)
    assert not srv.members


def test_contexts_are_pooled_per_grid_size(monkeypatch):
    """Finished requests hand their context to the next request of the same
    size: no more contexts exist than requests of a size ever resident at
    once, and every context served requests of one size only."""
    srv = FakeServer(1 << 40, 4, 64)
    fake_sleep(srv, monkeypatch)
    reqs = serving.requests_from_trace(trace(40, rate=500.0))
    srv.run(reqs, clock=srv.clock)
    by_size = collections.Counter(tuple(r.workload["shape"]) for r in reqs)
    assert len(srv.contexts) <= sum(min(4, k) for k in by_size.values())
    assert len(srv.contexts) < len(reqs)
    for sim in srv.contexts:
        sizes = {tuple(next(r for r in reqs if r.id == u).workload["shape"]) for u in sim.users}
        assert len(sizes) == 1


def test_admission_waits_for_device_memory(monkeypatch):
    """With room for one context (all requests of one size) the server never
    holds two, and requests are admitted in arrival order."""
    reqs = serving.requests_from_trace(trace(8, rate=1000.0, sides=(48,)))
    one = max(serving.request_bytes(r.workload, W.FP32_SHIFTED) for r in reqs)
    srv = FakeServer(one + one // 2, 64, 100)
    fake_sleep(srv, monkeypatch)
    stats = srv.run(reqs, clock=srv.clock)
    assert stats["requests"] == 8
    assert stats["max_resident"] == 1
    assert len(srv.contexts) == 1
    order = sorted(reqs, key=lambda r: r.admitted)
    assert [r.id for r in order] == [r.id for r in sorted(reqs, key=lambda r: r.arrival)]


def test_no_request_is_admitted_before_it_arrives(monkeypatch):
    srv = FakeServer(1 << 40, 8, 50, seconds_per_update=1e-12)
    fake_sleep(srv, monkeypatch)
    reqs = serving.requests_from_trace(trace(12, rate=5.0))
    srv.run(reqs, clock=srv.clock)
    assert all(r.admitted >= r.arrival for r in reqs)
    # idle gaps were slept through, not spun with empty launches
    assert all(k >= 1 for _, k in srv.launches)
