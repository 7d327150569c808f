"""Continuous-batching request loop over the C ABI's batches.

Requests (independent simulations of differing sizes and force parameters)
arrive over time.  A request is admitted as soon as a slot is free and the
device has room for its populations (checked against free HBM); its context
joins the running batch, so its steps overlap with every other resident
simulation in the same batch launches.  Each tick advances all resident
grids by min(tick_steps, smallest remaining step count) steps; requests that
reach their step count are read out (physical moments), removed from the
batch, and their context returns to a pool, which frees their slot for the
next arrival.

The loop keeps the GPU busy while the host schedules.  The device work of
one tick -- the initialisation of newly admitted requests (lbm_set_params on
a pooled context of the right grid size, then lbm_init from device copies of
their fields), the batch step, and the readout of the requests it completes
(lbm_moments_async into device memory, then a copy to page-locked host
memory) -- is enqueued on the batch's stream without waiting; the host then
waits only for the PREVIOUS tick, so one tick is always queued behind the
running one, and collects readouts whose event has completed.  In steady
state no device memory is allocated or freed (pooled contexts, torch's
caching allocator), so nothing synchronises the device.

Nothing here computes any part of the method: stepping runs in the CUDA
library (lbm_batch_step), this module only schedules.
"""
import collections
import time

import numpy as np

import paper_2302_04741_gb300 as lbm
from paper_2302_04741_gb300 import workloads as W


class Request:
    __slots__ = ("id", "arrival", "workload", "steps", "sim", "admitted", "done", "result",
                 "sites", "staging")

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
        self.staging = None


def request_bytes(w, precision):
    """Device bytes a request holds: two population buffers plus per-context
    scratch (moment buffer, reductions, force tables)."""
    Q = 37 if w["lattice"] == W.D2Q37 else 39
    D = W.dims(w["lattice"])
    N = int(np.prod(w["shape"]))
    elem = {W.FP64: 8, W.FP32_SHIFTED: 4, W.FP16_SCALED: 2}[precision]
    return 2 * Q * N * elem + (2 + 2 * D) * N * 8 + (1 << 20)


class Readout:
    """A completed request whose moments are on their way to the host."""
    __slots__ = ("req", "host", "event")

    def __init__(self, req, host, event):
        self.req, self.host, self.event = req, host, event


class Server:
    """Continuous batching of lattice-Boltzmann requests on one GPU.

    lattice / precision / force_order: shared by every request of a server
    (one batch kernel instantiation).  max_slots: resident requests at most.
    hbm_reserve: bytes of device memory left free.  tick_steps: steps per
    batch launch sequence between scheduling decisions.  graph_steps: CUDA
    graph length for the batch (even, 0 = plain launches).

    The device-facing steps are the methods _context, _start, _tick,
    _readout, _ready, _wait and _collect; run() holds the scheduling.
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
        self._setup()

    def _setup(self):
        self.resident = []
        self.ticks = []     # (steps, lattice updates, start event, end event)
        self.max_resident = 0
        self.pool = collections.defaultdict(list)  # grid shape -> idle contexts (Sim)
        self.contexts = []                         # every context created
        self.phase = collections.Counter()         # host seconds per phase

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
        if getattr(self, "stream", None) is not None:
            self.stream.synchronize()
        for r in getattr(self, "resident", []):
            lbm.lbm_batch_remove(self.batch, r.sim.ctx)
        for sim in getattr(self, "contexts", []):
            sim.close()
        self.resident, self.contexts, self.pool = [], [], collections.defaultdict(list)
        if getattr(self, "batch", None):
            lbm.lbm_batch_destroy(self.batch)
            self.batch = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ----------------------------------------------------- device-facing steps
    def _fits(self, req):
        if self.pool[tuple(req.workload["shape"])]:
            return True  # an idle context of this size is ready
        free, _ = self.torch.cuda.mem_get_info()
        return free - request_bytes(req.workload, self.precision) >= self.hbm_reserve

    def _context(self, req):
        """An idle pooled context of the request's grid size with its tau and
        force set, or a new one."""
        w = dict(req.workload, precision=self.precision, force_order=self.force_order)
        idle = self.pool[tuple(w["shape"])]
        if idle:
            sim = idle.pop()
            lbm.lbm_set_params(sim.ctx, w["tau"], w.get("g"))
            sim.w = w
            return sim
        sim = lbm.Sim(w, stream=self.stream.cuda_stream)
        self.contexts.append(sim)
        return sim

    def _start(self, req):
        """Fields to the device (page-locked staging, asynchronous on the
        batch's stream), lbm_init from the device copies, join the batch."""
        torch = self.torch
        w = req.workload
        host = [torch.from_numpy(np.ascontiguousarray(w[k], dtype=np.float64)).pin_memory()
                for k in ("rho", "u", "T")]
        with torch.cuda.stream(self.stream):
            dev = [h.to("cuda", non_blocking=True) for h in host]
        lbm.lbm_init(req.sim.ctx, *dev)
        req.staging = (host, dev)  # alive until the copies and the init have run
        lbm.lbm_batch_add(self.batch, req.sim.ctx)

    def _tick(self, n, lups):
        torch = self.torch
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(self.stream)
        lbm.lbm_batch_step(self.batch, n)
        e1.record(self.stream)
        self.ticks.append((n, lups, e0, e1))
        return e1

    def _readout(self, req):
        """Leave the batch and enqueue the moments into page-locked host memory."""
        torch = self.torch
        lbm.lbm_batch_remove(self.batch, req.sim.ctx)
        D = W.dims(req.workload["lattice"])
        N = req.sites
        with torch.cuda.stream(self.stream):
            dev = [torch.empty(n, dtype=torch.float64, device="cuda") for n in (N, D * N, N, D * N)]
            lbm.lbm_moments_async(req.sim.ctx, *dev)
            host = [torch.empty(t.numel(), dtype=torch.float64, pin_memory=True) for t in dev]
            for h, t in zip(host, dev):
                h.copy_(t, non_blocking=True)
        ev = torch.cuda.Event()
        ev.record(self.stream)
        self.pool[tuple(req.workload["shape"])].append(req.sim)  # re-used only after this readout
        return Readout(req, (host, dev), ev)

    def _ready(self, rd):
        return rd.event.query()

    def _wait(self, event):
        event.synchronize()

    def _collect(self, rd):
        host = rd.host[0]
        D = W.dims(rd.req.workload["lattice"])
        names = ("rho", "u", "T", "q")
        vals = [host[0].numpy(), host[1].numpy().reshape(D, -1), host[2].numpy(), host[3].numpy().reshape(D, -1)]
        return {k: v.copy() for k, v in zip(names, vals) if k in self.collect}

    def _busy_seconds(self):
        return sum(e0.elapsed_time(e1) for _, _, e0, e1 in self.ticks) / 1e3

    # ------------------------------------------------------------- the loop
    def _admit(self, req, now):
        req.sim = self._context(req)
        self._start(req)
        req.admitted = now
        self.resident.append(req)
        self.max_resident = max(self.max_resident, len(self.resident))

    def run(self, requests, clock=None):
        """Serve ``requests`` (sorted by arrival, seconds from start).  Returns
        a stats dict with p50 / p99 time-to-result, aggregate MLUPS (lattice
        updates of the finished requests over the wall time), busy MLUPS (the
        same over the device time of the ticks) and the host seconds spent
        per phase of the loop."""
        clock = clock or time.perf_counter
        pending = sorted(requests, key=lambda r: r.arrival)
        t0 = clock()
        finished = []
        readouts = []
        prev_tick = None
        i = 0
        while i < len(pending) or self.resident or readouts:
            now = clock() - t0
            # admit every arrived request that fits (continuous batching)
            ta = clock()
            while (i < len(pending) and pending[i].arrival <= now
                   and len(self.resident) < self.max_slots and self._fits(pending[i])):
                self._admit(pending[i], now)
                i += 1
            tb = clock()
            self.phase["admit"] += tb - ta
            tick = None
            if self.resident:
                # one tick, never past the nearest completion, then the readout
                # of the requests it completes, all enqueued without waiting
                left = [r.steps - lbm.lbm_step_count(r.sim.ctx) for r in self.resident]
                n = max(1, min(self.tick_steps, min(left)))
                tick = self._tick(n, n * sum(r.sites for r in self.resident))
                for r in [r for r in self.resident if lbm.lbm_step_count(r.sim.ctx) >= r.steps]:
                    self.resident.remove(r)
                    readouts.append(self._readout(r))
                    tick = readouts[-1].event  # the tick and its readouts
            tc = clock()
            self.phase["enqueue"] += tc - tb
            # wait for the previous tick only: the one just enqueued keeps the
            # device busy while the host admits and collects
            if prev_tick is not None:
                self._wait(prev_tick)
            prev_tick = tick
            td = clock()
            self.phase["wait"] += td - tc
            for rd in list(readouts):
                if self._ready(rd):
                    rd.req.result = self._collect(rd)
                    rd.req.done = clock() - t0
                    rd.req.sim = None
                    rd.req.staging = None
                    finished.append(rd.req)
                    readouts.remove(rd)
            self.phase["collect"] += clock() - td
            if not self.resident and readouts and tick is None:
                self._wait(readouts[-1].event)  # drain the last readouts
            elif not self.resident and not readouts and i < len(pending):
                # idle until the next arrival
                wait = pending[i].arrival - (clock() - t0)
                if wait > 0:
                    time.sleep(min(wait, 0.05))
                prev_tick = None
        wall = clock() - t0
        lat = np.array([r.done - r.arrival for r in finished])
        lups = sum(r.sites * r.steps for r in finished)
        busy = self._busy_seconds()
        tick_lups = sum(t[1] for t in self.ticks)
        return {
            "requests": len(finished),
            "p50_s": float(np.percentile(lat, 50)) if len(lat) else None,
            "p99_s": float(np.percentile(lat, 99)) if len(lat) else None,
            "mean_s": float(lat.mean()) if len(lat) else None,
            "wall_s": wall,
            "aggregate_mlups": lups / wall / 1e6 if wall > 0 else None,
            "busy_mlups": tick_lups / busy / 1e6 if busy > 0 else None,
            "busy_fraction": busy / wall if wall > 0 else None,
            "ticks": len(self.ticks),
            "lattice_updates": lups,
            "max_resident": self.max_resident,
            "contexts_created": len(self.contexts),
            "host_seconds": {k: float(v) for k, v in self.phase.items()},
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
