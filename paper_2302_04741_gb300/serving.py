"""Continuous-batching request loop over the C ABI's batches.

Requests (independent simulations of differing sizes and force parameters)
arrive over time.  A request is admitted as soon as a slot is free and the
device has room for its populations (checked against free HBM); its context
joins the running batch, so its steps overlap with every other resident
simulation in the same batch launches.  Each tick advances all resident
grids by min(tick_steps, smallest remaining step count) steps; requests that
reach their step count are read out (physical moments), removed from the batch
and freed, which frees their slot for the next arrival.

Nothing here computes any part of the method: stepping runs in the CUDA
library (lbm_batch_step), this module only schedules.
"""
import math
import time

import numpy as np

import paper_2302_04741_gb300 as lbm
from paper_2302_04741_gb300 import workloads as W


class Request:
    __slots__ = ("id", "arrival", "workload", "steps", "sim", "admitted", "done", "result",
                 "sites")

    def __init__(self, rid, arrival, workload, steps):
        self.id = rid
        self.arrival = arrival
        self.workload = workload
        self.steps = steps
        self.sim = None
        self.admitted = None
        self.done = None
        self.result = None
        self.sites = int(np.prod(workload["shape"]))


def request_bytes(w, precision):
    """Device bytes a request holds: two population buffers plus per-context
    scratch (moment buffer, reductions, force tables)."""
    Q = 37 if w["lattice"] == W.D2Q37 else 39
    D = W.dims(w["lattice"])
    N = int(np.prod(w["shape"]))
    elem = {W.FP64: 8, W.FP32_SHIFTED: 4, W.FP16_SCALED: 2}[precision]
    return 2 * Q * N * elem + (2 + 2 * D) * N * 8 + (1 << 20)


class Server:
    """Continuous batching of lattice-Boltzmann requests on one GPU.

    lattice / precision / force_order: shared by every request of a server
    (one batch kernel instantiation).  max_slots: resident requests at most.
    hbm_reserve: bytes of device memory left free.  tick_steps: steps per
    batch launch sequence between scheduling decisions.  graph_steps: CUDA
    graph length for the batch (even, 0 = plain launches).
    """

    def __init__(self, lattice=W.D3Q39, precision=W.FP32_SHIFTED, force_order=2, max_slots=64,
                 hbm_reserve=4 << 30, tick_steps=100, graph_steps=10, tune_sides=None,
                 collect=("rho", "u", "T", "q")):
        import torch
        self.torch = torch
        self.lattice = lattice
        self.precision = precision
        self.force_order = force_order
        self.max_slots = max_slots
        self.hbm_reserve = hbm_reserve
        self.tick_steps = tick_steps
        self.graph_steps = graph_steps
        self.collect = collect
        self.stream = torch.cuda.Stream()
        self.batch = lbm.lbm_batch_create(lattice, precision, force_order, self.stream.cuda_stream,
                                          max(max_slots, 1))
        bx, spt = 128, 1
        if tune_sides:
            bx, spt = self._tune(tune_sides)
        self.config = (bx, spt, graph_steps)
        lbm.lbm_batch_set_config(self.batch, bx, spt, graph_steps)
        self.resident = []
        self.ticks = []  # (steps, seconds, lattice updates)
        self.max_resident = 0

    def _tune(self, sides):
        """Launch configuration from the autotuner, timed on a warm-up batch of
        periodic boxes with the given sides (tuning steps real grids, so it
        never runs on live requests)."""
        boxes = []
        b = lbm.lbm_batch_create(self.lattice, self.precision, self.force_order,
                                 self.stream.cuda_stream, len(sides))
        try:
            for k, side in enumerate(sides):
                w = W.make_request(dict(id=-1 - k, arrival=0.0, side=side, g=5e-6, steps=0,
                                        tau=0.8, seed=99), self.precision)
                w["force_order"] = self.force_order
                sim = lbm.Sim(w, stream=self.stream.cuda_stream).init()
                boxes.append(sim)
                lbm.lbm_batch_add(b, sim.ctx)
            return lbm.lbm_batch_tune(b, 4)
        finally:
            lbm.lbm_batch_destroy(b)
            for sim in boxes:
                sim.close()

    def close(self):
        for r in self.resident:
            r.sim.close()
        self.resident = []
        if self.batch:
            lbm.lbm_batch_destroy(self.batch)
            self.batch = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ------------------------------------------------------------ admission
    def _fits(self, req):
        free, _ = self.torch.cuda.mem_get_info()
        return free - request_bytes(req.workload, self.precision) >= self.hbm_reserve

    def _admit(self, req, now):
        w = dict(req.workload, precision=self.precision, force_order=self.force_order)
        req.sim = lbm.Sim(w, stream=self.stream.cuda_stream).init()
        lbm.lbm_batch_add(self.batch, req.sim.ctx)
        req.admitted = now
        self.resident.append(req)
        self.max_resident = max(self.max_resident, len(self.resident))

    def _retire(self, req, now):
        out = {}
        m = req.sim.moments()
        for name, v in zip(("rho", "u", "T", "q"), m):
            if name in self.collect:
                out[name] = v
        req.result = out
        lbm.lbm_batch_remove(self.batch, req.sim.ctx)
        req.sim.close()
        req.sim = None
        req.done = now
        self.resident.remove(req)

    # ------------------------------------------------------------- the loop
    def run(self, requests, clock=None):
        """Serve ``requests`` (sorted by arrival, seconds from start).  Returns
        a stats dict with p50 / p99 time-to-result and aggregate MLUPS."""
        clock = clock or time.perf_counter
        pending = sorted(requests, key=lambda r: r.arrival)
        t0 = clock()
        finished = []
        i = 0
        while i < len(pending) or self.resident:
            now = clock() - t0
            # admit every arrived request that fits (continuous batching)
            while (i < len(pending) and pending[i].arrival <= now
                   and len(self.resident) < self.max_slots and self._fits(pending[i])):
                self._admit(pending[i], now)
                i += 1
            if not self.resident:
                # idle until the next arrival
                if i < len(pending):
                    wait = pending[i].arrival - (clock() - t0)
                    if wait > 0:
                        time.sleep(min(wait, 0.05))
                continue
            left = [r.steps - lbm.lbm_step_count(r.sim.ctx) for r in self.resident]
            n = max(1, min(self.tick_steps, min(left)))
            ts = clock()
            lbm.lbm_batch_step(self.batch, n)
            self.stream.synchronize()
            dt = clock() - ts
            self.ticks.append((n, dt, n * sum(r.sites for r in self.resident)))
            now = clock() - t0
            for r in list(self.resident):
                if lbm.lbm_step_count(r.sim.ctx) >= r.steps:
                    self._retire(r, now)
                    finished.append(r)
        wall = clock() - t0
        lat = np.array([r.done - r.arrival for r in finished])
        lups = sum(r.sites * r.steps for r in finished)
        busy = sum(t[1] for t in self.ticks)
        tick_lups = sum(t[2] for t in self.ticks)
        return {
            "requests": len(finished),
            "p50_s": float(np.percentile(lat, 50)) if len(lat) else None,
            "p99_s": float(np.percentile(lat, 99)) if len(lat) else None,
            "mean_s": float(lat.mean()) if len(lat) else None,
            "wall_s": wall,
            "aggregate_mlups": lups / wall / 1e6 if wall > 0 else None,
            "busy_mlups": tick_lups / busy / 1e6 if busy > 0 else None,
            "ticks": len(self.ticks),
            "lattice_updates": lups,
            "max_resident": self.max_resident,
        }


def requests_from_trace(trace, precision=W.FP32_SHIFTED):
    """Request objects for a serving trace (workloads.serving_trace)."""
    out = []
    for t in trace:
        w = W.make_request(t, precision)
        out.append(Request(t["id"], t["arrival"], w, t["steps"]))
    return out


def capacity_rate(mlups, trace):
    """Arrival rate (requests/s) at which the offered lattice updates equal a
    device throughput of ``mlups``."""
    mean_lups = np.mean([t["side"] ** 3 * t["steps"] for t in trace])
    return mlups * 1e6 / mean_lups


def rescale_arrivals(trace, rate):
    """The same trace with Poisson gaps rescaled to mean 1/rate."""
    if not trace:
        return trace
    base_rate = len(trace) / trace[-1]["arrival"] if trace[-1]["arrival"] > 0 else rate
    f = base_rate / rate
    return [dict(t, arrival=t["arrival"] * f) for t in trace]
