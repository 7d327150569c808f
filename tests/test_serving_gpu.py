"""Continuous batching: requests that arrive while others run join the same
persistent launches; every result must equal the request run alone."""
import numpy as np
import pytest

import paper_2302_04741_gb300 as lbm
from paper_2302_04741_gb300 import serving as S
from paper_2302_04741_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    pytest.importorskip("torch")
    from paper_2302_04741_gb300 import build
    build.build()


class TickClock:
    """Deterministic clock: every call advances time by dt seconds."""

    def __init__(self, dt=0.01):
        self.t = 0.0
        self.dt = dt

    def __call__(self):
        self.t += self.dt
        return self.t


def small_trace():
    rng_sides = [16, 24, 32, 16, 24, 20]
    steps = [60, 150, 90, 40, 110, 75]
    arrivals = [0.0, 0.0, 0.05, 0.3, 0.31, 0.9]
    return [dict(id=k, arrival=a, side=s, g=2e-6 * (k + 1), steps=n, tau=0.7 + 0.05 * k, seed=4)
            for k, (s, n, a) in enumerate(zip(rng_sides, steps, arrivals))]


def run_alone(req, precision):
    sim = lbm.Sim(dict(req.workload, precision=precision)).init()
    sim.step(req.steps)
    out = sim.moments()
    sim.close()
    return out


@pytest.mark.parametrize("precision", [W.FP32_SHIFTED, W.FP16_SCALED])
def test_each_result_same_alone_and_in_the_mix(precision):
    reqs = S.requests_from_trace(small_trace(), precision)
    srv = S.Server(precision=precision, max_slots=4, tick_steps=25, graph_steps=4)
    try:
        stats = srv.run(reqs, clock=TickClock())
    finally:
        srv.close()
    assert stats["requests"] == len(reqs)
    assert stats["max_resident"] >= 3          # requests overlapped on the device
    assert all(r.admitted > r.arrival - 1e-12 for r in reqs)
    for r in reqs:
        alone = run_alone(r, precision)
        for name, a in zip(("rho", "u", "T", "q"), alone):
            np.testing.assert_array_equal(r.result[name], a, err_msg=f"request {r.id} {name}")


def test_slot_limit_and_hbm_admission():
    import torch
    reqs = S.requests_from_trace(small_trace())
    srv = S.Server(max_slots=2, tick_steps=30, graph_steps=0)
    try:
        stats = srv.run(reqs, clock=TickClock())
        assert stats["requests"] == len(reqs) and stats["max_resident"] <= 2
    finally:
        srv.close()
    # equal-size requests and room for exactly one of them at a time
    reqs = S.requests_from_trace([dict(t, side=24) for t in small_trace()])
    need = S.request_bytes(reqs[0].workload, W.FP32_SHIFTED)
    free, _ = torch.cuda.mem_get_info()
    srv = S.Server(max_slots=8, tick_steps=30, graph_steps=0, hbm_reserve=free - int(1.5 * need))
    try:
        stats = srv.run(reqs, clock=TickClock())
        assert stats["requests"] == len(reqs) and stats["max_resident"] == 1
    finally:
        srv.close()


def test_tuned_server_config():
    srv = S.Server(max_slots=4, tick_steps=20, graph_steps=4, tune_sides=(16, 24))
    try:
        bx, spt, gs = srv.config
        assert bx in (64, 128, 256) and spt in (1, 2) and gs == 4
        reqs = S.requests_from_trace(small_trace()[:3])
        stats = srv.run(reqs, clock=TickClock())
        assert stats["requests"] == 3
    finally:
        srv.close()
    for r in reqs:
        alone = run_alone(r, W.FP32_SHIFTED)
        np.testing.assert_array_equal(r.result["u"], alone[1])


def test_served_requests_match_oracle():
    """Requests of the serving trace's smallest side (32^3 D3Q39 boxes), served
    through continuous batching in FP32-shifted storage, agree with the FP64
    oracle run on each request alone: rho, u, T and q within the FP32
    tolerance (q with the floor and the codec bound of the parity tests).
    Each box starts with a resolved shear wave (u ~ 1e-2) so that u is a
    resolved flow rather than a g-driven drift at the storage floor."""
    from helpers import check_fields, oracle_sim
    trace = [dict(id=k, arrival=0.01 * k, side=32, g=3e-6 * (k + 1), steps=30 + 10 * k, tau=0.7 + 0.1 * k,
                  seed=7) for k in range(3)]
    reqs = S.requests_from_trace(trace, W.FP32_SHIFTED)
    for r in reqs:
        s = r.workload["shape"][0]
        z = np.arange(s ** 3) // (s * s)
        u = np.zeros((3, s ** 3))
        u[0] = 1e-2 * np.sin(2 * np.pi * z / s)
        u[1] = 5e-3 * np.cos(2 * np.pi * z / s)
        r.workload["u"] = u
    srv = S.Server(precision=W.FP32_SHIFTED, max_slots=4, tick_steps=10, graph_steps=4)
    try:
        srv.run(reqs, clock=TickClock())
    finally:
        srv.close()
    for r in reqs:
        ref = oracle_sim(r.workload)
        ref.step(r.steps)
        got = (r.result["rho"], r.result["u"], r.result["T"], r.result["q"])
        check_fields(got, ref, r.workload, 1e-6)
