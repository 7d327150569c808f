"""Host logic of the continuous-batching server, with the device calls faked.

The scheduler decides admission (arrival, free slot, free HBM), the number
of steps per tick (never past the nearest completion) and retirement; none
of that needs a GPU, so the library entry points it calls are replaced by a
fake batch that only counts steps, and time is a fake clock that advances
with the work.
"""
import numpy as np
import pytest

import paper_2302_04741_gb300 as lbm
from paper_2302_04741_gb300 import serving, workloads as W


class FakeSim:
    live = []

    def __init__(self, w, stream=None):
        self.w = w
        self.ctx = self
        self.steps = 0
        self.closed = False
        FakeSim.live.append(self)

    def init(self):
        return self

    def moments(self):
        n = int(np.prod(self.w["shape"]))
        return np.ones(n), np.zeros((3, n)), np.ones(n), np.zeros((3, n))

    def close(self):
        self.closed = True


class FakeDevice:
    """Batch membership, step counts, a clock advanced by the work and the
    free memory the admission check reads."""

    def __init__(self, free_bytes, seconds_per_update=1e-10):
        self.members = []
        self.launches = []
        self.t = 0.0
        self.free = free_bytes
        self.spu = seconds_per_update

    def clock(self):
        return self.t

    def batch_add(self, b, ctx):
        assert ctx not in self.members
        self.members.append(ctx)
        self.free -= serving.request_bytes(ctx.w, W.FP32_SHIFTED)

    def batch_remove(self, b, ctx):
        self.members.remove(ctx)
        self.free += serving.request_bytes(ctx.w, W.FP32_SHIFTED)

    def batch_step(self, b, n):
        assert self.members, "a tick with no resident grid"
        self.launches.append((n, len(self.members)))
        for m in self.members:
            m.steps += n
        self.t += n * sum(int(np.prod(m.w["shape"])) for m in self.members) * self.spu


class FakeTorchCuda:
    def __init__(self, dev):
        self.dev = dev

    def mem_get_info(self):
        return self.dev.free, 1 << 40


class FakeTorch:
    def __init__(self, dev):
        self.cuda = FakeTorchCuda(dev)


class FakeStream:
    cuda_stream = 0

    def synchronize(self):
        pass


def make_server(monkeypatch, dev, max_slots, tick_steps, reserve=0):
    monkeypatch.setattr(lbm, "Sim", FakeSim)
    monkeypatch.setattr(lbm, "lbm_batch_add", dev.batch_add)
    monkeypatch.setattr(lbm, "lbm_batch_remove", dev.batch_remove)
    monkeypatch.setattr(lbm, "lbm_batch_step", dev.batch_step)
    monkeypatch.setattr(lbm, "lbm_step_count", lambda ctx: ctx.steps)
    monkeypatch.setattr(serving.time, "sleep", lambda s: setattr(dev, "t", dev.t + s))
    s = serving.Server.__new__(serving.Server)
    s.torch = FakeTorch(dev)
    s.lattice, s.precision, s.force_order = W.D3Q39, W.FP32_SHIFTED, 2
    s.max_slots, s.hbm_reserve, s.tick_steps = max_slots, reserve, tick_steps
    s.graph_steps, s.collect = 10, ("rho", "u", "T", "q")
    s.stream, s.batch = FakeStream(), None
    s.resident, s.ticks, s.max_resident = [], [], 0
    return s


def trace(n, seed=4, rate=50.0, sides=(32, 48)):
    return W.serving_trace(n_requests=n, rate=rate, seed=seed, sides=sides, steps_range=(50, 400))


@pytest.mark.parametrize("max_slots,tick", [(1, 100), (4, 64), (64, 1000)])
def test_every_request_finishes_with_its_exact_step_count(monkeypatch, max_slots, tick):
    FakeSim.live = []
    dev = FakeDevice(free_bytes=1 << 40)
    srv = make_server(monkeypatch, dev, max_slots, tick)
    reqs = serving.requests_from_trace(trace(30))
    stats = srv.run(reqs, clock=dev.clock)
    assert stats["requests"] == 30
    for r in reqs:
        assert r.sim is None and r.done is not None and r.done >= r.arrival
        assert r.admitted >= r.arrival
        assert set(r.result) == {"rho", "u", "T", "q"}
    # no overshoot: every grid stopped exactly at its step count
    done_steps = sorted(s.steps for s in FakeSim.live)
    assert done_steps == sorted(r.steps for r in reqs)
    assert all(s.closed for s in FakeSim.live)
    # ticks never exceed the limit, and the resident count never the slots
    assert all(1 <= n <= tick for n, _ in dev.launches)
    assert all(k <= max_slots for _, k in dev.launches)
    assert stats["max_resident"] <= max_slots
    assert stats["lattice_updates"] == sum(r.sites * r.steps for r in reqs)
    assert not dev.members


def test_admission_waits_for_device_memory(monkeypatch):
    """With room for one request at a time (all of one size) the server never
    holds two, and requests are admitted in arrival order."""
    FakeSim.live = []
    reqs = serving.requests_from_trace(trace(8, rate=1000.0, sides=(48,)))
    one = max(serving.request_bytes(r.workload, W.FP32_SHIFTED) for r in reqs)
    dev = FakeDevice(free_bytes=one + one // 2)
    srv = make_server(monkeypatch, dev, max_slots=64, tick_steps=100)
    stats = srv.run(reqs, clock=dev.clock)
    assert stats["requests"] == 8
    assert stats["max_resident"] == 1
    order = sorted(reqs, key=lambda r: r.admitted)
    assert [r.id for r in order] == [r.id for r in sorted(reqs, key=lambda r: r.arrival)]


def test_no_request_is_admitted_before_it_arrives(monkeypatch):
    FakeSim.live = []
    dev = FakeDevice(free_bytes=1 << 40, seconds_per_update=1e-12)
    srv = make_server(monkeypatch, dev, max_slots=8, tick_steps=50)
    reqs = serving.requests_from_trace(trace(12, rate=5.0))
    srv.run(reqs, clock=dev.clock)
    assert all(r.admitted >= r.arrival for r in reqs)
    # idle gaps were slept through, not spun with empty launches
    assert all(k >= 1 for _, k in dev.launches)
