#!/usr/bin/env python
"""Throughput benchmark of the fused stream-collide step (one JSON line).

Workload: thermal Rayleigh-Benard cell on D2Q37, 1024 x 512 sites, walls at
y = -1/2 (T = 1.05) and y = 511.5 (T = 0.95), periodic in x, uniform gravity
g_y = -1e-5, tau-hat = 0.6, populations stored as FP32 deviations f_i - w_i,
seeded 1e-4 temperature perturbation (workloads.rayleigh_benard).

One benchmark step = lbm_step(ctx, INNER) (INNER fused stream-collide
launches) followed by lbm_conserved (the FP64 conservation / stability
diagnostic), i.e. one pass over every row of the hot path.  L2 is flushed
(256 MiB write) before every timed step, outside the timed interval.

Multi-GPU (torchrun): every rank runs its own independent grid (weak scaling,
no data-path collective); the timing is the max over ranks.

--impl reference times the FP64 CPU oracle on the host cores instead (one
oracle LBM step over the same grid per benchmark step).
"""
import argparse
import ctypes
import hashlib
import json
import math
import os
import re
import subprocess
import sys
import tempfile
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "MLUPS & % HBM roofline, FP32-shifted vs FP64 at stated L2 error; serving p50/p99"
FALLBACK_HBM_GBS = 6800.0
KERNEL_SOURCES = ["lbm_device.cuh", "lbm_kernels.cuh", "lbm_tma.cuh", "lbm_async.cuh",
                  "lbm_wave.cuh", "lbm_batch.cuh", "lbm_launch.cuh", "lbm_df.cuh", "lattice_tables.cuh"]


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--inner", type=int, default=50, help="LBM steps per benchmark step")
    ap.add_argument("--graph-steps", type=int, default=10,
                    help="lbm_step replays CUDA graphs of this many steps (0 = plain launches)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--nx", type=int, default=1024)
    ap.add_argument("--ny", type=int, default=512)
    ap.add_argument("--kernel", default="auto", choices=["auto", "plain", "tma", "prefetch"],
                    help="step kernel of the FP32 context")
    ap.add_argument("--tma-stages", type=int, default=0)
    ap.add_argument("--block-x", type=int, default=0, help="threads per block (0 = library default)")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the other configurations (Kolmogorov, ragged batch, serving, 3-D FP16)")
    ap.add_argument("--serve-requests", type=int, default=120)
    ap.add_argument("--no-accuracy", action="store_true",
                    help="skip the full-length FP32 accuracy runs (three 20k-step FP64 runs)")
    return ap.parse_args()


def code_tokens(text):
    """C++/CUDA source without comments and with whitespace runs collapsed:
    edits to comments leave a kernel's identity unchanged."""
    text = re.sub(r"/\*.*?\*/", " ", text, flags=re.S)
    text = re.sub(r"//[^\n]*", " ", text)
    return " ".join(text.split())


def kernel_source_sha():
    """Identity of the kernel sources the committed ncu summaries were taken
    on (their code, not their comments)."""
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        with open(os.path.join(ROOT, "paper_2302_04741_gb300", "csrc", f)) as fh:
            h.update(code_tokens(fh.read()).encode())
    return h.hexdigest()[:16]


def measured_peak():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as fh:
            return float(json.load(fh)["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


def profiled_value(name, key):
    """A number recorded in a committed ncu summary (``key: value``), if the
    summary was taken on the current kernel source; else None."""
    path = os.path.join(ROOT, "profiles", name)
    try:
        with open(path) as fh:
            text = fh.read()
    except OSError:
        return None
    m = re.search(re.escape(key) + r":\s*([0-9.eE+]+)", text)
    s = re.search(r"kernel_source_sha:\s*([0-9a-f]+)", text)
    if not m or not s or s.group(1) != kernel_source_sha():
        return None
    return float(m.group(1))


def profiled_traffic(name):
    """DRAM bytes per launch from a committed ncu summary (current source only)."""
    return profiled_value(name, "traffic_bytes_per_launch")


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled every 200 ms."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.file = None

    def start(self):
        try:
            self.file = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=self.file, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if not self.proc:
            return None
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.file.flush()
        self.file.seek(0)
        rows = [r.split(",") for r in self.file.read().strip().splitlines() if r.strip()]
        os.unlink(self.file.name)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            try:
                sm.append(float(r[1]))
                mx.append(float(r[2]))
            except (ValueError, IndexError):
                continue
            for k, n in enumerate(names):
                if len(r) > 5 + k and r[5 + k].strip().lower() == "active":
                    reasons.add(n)
        if not sm:
            return None
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


class NvmlSampler:
    """SM clock and clock-event reasons read through NVML (libnvidia-ml,
    read-only queries) from a thread every few milliseconds: a timed region
    of a few tens of milliseconds is shorter than nvidia-smi's sampling
    period.  start() returns False when NVML cannot be used."""

    REASONS = {0x4: "sw_power_cap", 0x8: "hw_slowdown", 0x20: "sw_thermal_slowdown",
               0x40: "hw_thermal_slowdown"}

    def __init__(self, index, period=0.005):
        self.index = index
        self.period = period
        self.lib = None
        self.handle = None
        self.max_mhz = None
        self.thread = None
        self.running = False
        self.samples = []

    def start(self):
        try:
            lib = ctypes.CDLL("libnvidia-ml.so.1")
            lib.nvmlInit_v2.restype = ctypes.c_int
            if lib.nvmlInit_v2() != 0:
                return False
            h = ctypes.c_void_p()
            if lib.nvmlDeviceGetHandleByIndex_v2(ctypes.c_uint(self.index), ctypes.byref(h)) != 0:
                return False
            self.reason_fn = getattr(lib, "nvmlDeviceGetCurrentClocksEventReasons", None) or \
                lib.nvmlDeviceGetCurrentClocksThrottleReasons
            mx = ctypes.c_uint()
            if lib.nvmlDeviceGetMaxClockInfo(h, ctypes.c_int(1), ctypes.byref(mx)) != 0:
                return False
        except (OSError, AttributeError):
            return False
        self.lib, self.handle, self.max_mhz = lib, h, mx.value
        self.running = True
        self.thread = threading.Thread(target=self._loop, daemon=True)
        self.thread.start()
        return True

    def _loop(self):
        clk, rs = ctypes.c_uint(), ctypes.c_ulonglong()
        while self.running:
            if (self.lib.nvmlDeviceGetClockInfo(self.handle, ctypes.c_int(1), ctypes.byref(clk)) == 0
                    and self.reason_fn(self.handle, ctypes.byref(rs)) == 0):
                self.samples.append((clk.value, rs.value))
            time.sleep(self.period)

    def stop(self):
        if not self.thread:
            return None
        self.running = False
        self.thread.join(timeout=2)
        try:
            self.lib.nvmlShutdown()
        except Exception:
            pass
        if not self.samples:
            return None
        reasons = sorted({n for _, r in self.samples for bit, n in self.REASONS.items() if r & bit})
        return {"sm_mhz": float(np.median([c for c, _ in self.samples])), "sm_max_mhz": self.max_mhz,
                "reasons": reasons, "samples": len(self.samples), "source": "nvml, 5 ms"}


def aggregate_ranks(elapsed_ms, units_per_rank, world, device=None):
    """Whole-job throughput over `world` ranks that each processed
    `units_per_rank` lattice updates in `elapsed_ms`: the slowest rank's time
    (max all-reduce; the only collective, on the host-side timing, never on
    the data path) divides the units of all ranks.  Returns (MLUPS, max ms)."""
    t_max = elapsed_ms
    if world > 1:
        import torch
        import torch.distributed as dist
        t = torch.tensor([elapsed_ms], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        t_max = float(t.item())
    return world * units_per_rank / (t_max / 1e3) / 1e6, t_max


def dist_info():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


# --------------------------------------------------------------- the oracle arm
def cpu_model():
    """The host CPU's model name (or architecture) for the baseline record."""
    try:
        with open("/proc/cpuinfo") as fh:
            for line in fh:
                if line.lower().startswith(("model name", "cpu model")):
                    return line.split(":", 1)[1].strip()
    except OSError:
        pass
    import platform
    return platform.machine()


def oracle_rate(w, steps, warmup, budget_s=None, threads=None):
    """MLUPS of the FP64 CPU oracle on workload w (host cores; threads=None:
    all of them)."""
    import oracle
    from paper_2302_04741_gb300 import workloads as W

    oracle.set_threads(threads or os.cpu_count() or 1)
    g = W.g_field_array(w["lattice"], w["shape"], w["g"])
    s = oracle.OracleSim(w["lattice"], *w["shape"], w["tau"], g, force_order=w["force_order"],
                         bc=w["bc"], T_lo=w["T_lo"], T_hi=w["T_hi"])
    s.init(w["rho"], w["u"], w["T"])
    N = int(np.prod(w["shape"]))
    s.step(warmup)
    if budget_s is not None:
        t0 = time.perf_counter()
        s.step(1)
        t1 = time.perf_counter() - t0
        steps = int(max(1, min(steps, budget_s / max(t1, 1e-6))))
    t0 = time.perf_counter()
    s.step(steps)
    dt = time.perf_counter() - t0
    return N * steps / dt / 1e6, steps, dt, oracle.get_threads()


def run_reference(args):
    rank, world, _ = dist_info()
    if rank != 0:
        return
    from paper_2302_04741_gb300 import workloads as W

    w = W.rayleigh_benard(nx=args.nx, ny=args.ny, precision=W.FP64)
    mlups, steps, dt, cores = oracle_rate(w, args.steps, args.warmup)
    sample = f"FP64 oracle, full {args.nx}x{args.ny} D2Q37 Rayleigh-Benard grid, {steps} LBM steps"
    line = {
        "impl": "reference", "metric": METRIC, "value": mlups, "unit": "MLUPS", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / steps * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": f"rayleigh_benard_d2q37_{args.nx}x{args.ny}", "lattice": "D2Q37",
                   "grid": [args.nx, args.ny], "precision": "fp64 (oracle)", "bc": "thermal walls y, periodic x",
                   "step": "one oracle LBM step over the full grid"},
        "cpu_baseline": {"value": mlups, "unit": "MLUPS", "cores": cores, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": mlups, "unit": "MLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ------------------------------------------------------ other configurations
def event_time(torch, stream, fn, reps):
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(reps):
        fn()
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / 1e3


def extra_kolmogorov(lbm, torch, W, peak):
    """64x64 D2Q37 FP64 Kolmogorov flow, 2000 steps (L2-resident correctness case)."""
    stream = torch.cuda.Stream()
    w = W.kolmogorov()
    sim = lbm.Sim(w, stream=stream.cuda_stream).init()
    sim.step(10)
    t = event_time(torch, stream, lambda: sim.step(2000), 1)
    sim.close()
    return {"workload": "kolmogorov_d2q37_64x64_fp64", "steps": 2000,
            "mlups": 4096 * 2000 / t / 1e6, "note": "2.4 MB working set, L2-resident"}


def extra_ragged(lbm, torch, W, peak, single_mlups, K=5, inner=10):
    """64 periodic D2Q37 Kolmogorov grids of ragged sizes, FP32-shifted, one
    persistent launch per step, graph replay, autotuned block / sites per thread."""
    stream = torch.cuda.Stream()
    ws = W.ragged_batch()
    sims = [lbm.Sim(w, stream=stream.cuda_stream).init() for w in ws]
    b = lbm.lbm_batch_create(W.D2Q37, W.FP32_SHIFTED, 2, stream.cuda_stream, len(ws))
    try:
        for s_ in sims:
            lbm.lbm_batch_add(b, s_.ctx)
        bx, spt = lbm.lbm_batch_tune(b, 4)
        staged = lbm.lbm_batch_get_staging(b)
        lbm.lbm_batch_set_config(b, bx, spt, inner)
        lbm.lbm_batch_step(b, 2 * inner)
        t = event_time(torch, stream, lambda: lbm.lbm_batch_step(b, inner), K)
    finally:
        lbm.lbm_batch_destroy(b)
        for s_ in sims:
            s_.close()
    sites = sum(int(np.prod(w["shape"])) for w in ws)
    mlups = sites * inner * K / t / 1e6
    return {"workload": "ragged_batch_64_d2q37_fp32", "grids": len(ws), "sites": sites,
            "mlups": mlups, "roofline_frac": mlups * 1e6 * 296 / (peak * 1e9),
            "tuned": {"block_x": bx, "sites_per_thread": spt, "halo_staged": staged, "graph_steps": inner},
            "vs_single_grid_mlups": mlups / single_mlups}


def extra_serving(lbm, torch, W, peak, n_req):
    """Poisson arrivals of D3Q39 periodic boxes (sides 32..96), FP32-shifted,
    continuous batching; overloaded at the configured 200/s, and at 0.5x and
    0.9x the measured capacity."""
    from paper_2302_04741_gb300 import serving as S
    # single-box reference rate (96^3, plain step kernel)
    stream = torch.cuda.Stream()
    w = W.make_request(dict(id=0, arrival=0.0, side=96, g=5e-6, steps=0, tau=0.8, seed=4))
    sim = lbm.Sim(w, stream=stream.cuda_stream).init()
    sim.step(10)
    t = event_time(torch, stream, lambda: sim.step(50), 1)
    sim.close()
    single = 96 ** 3 * 50 / t / 1e6
    out = {"workload": "serving_d3q39_fp32_poisson", "single_box_96_mlups": single}
    trace = W.serving_trace(n_requests=n_req, rate=200.0)
    srv = S.Server(max_slots=64, tick_steps=100, graph_steps=10, tune_sides=(32, 48, 64, 96))
    try:
        st = srv.run(S.requests_from_trace(trace))
    finally:
        srv.close()
    st["offered_rate_per_s"] = 200.0
    st["busy_vs_single_box"] = st["busy_mlups"] / single
    out["at_200_per_s"] = st
    cap = S.capacity_rate(st["busy_mlups"], trace)
    n_low = max(8, n_req // 3)
    for key, frac, seed in (("at_half_capacity", 0.5, 5), ("at_0.9_capacity", 0.9, 6)):
        low = S.rescale_arrivals(W.serving_trace(n_requests=n_low, rate=200.0, seed=seed), frac * cap)
        srv = S.Server(max_slots=64, tick_steps=100, graph_steps=10, tune_sides=(32, 48, 64, 96))
        try:
            st2 = srv.run(S.requests_from_trace(low))
        finally:
            srv.close()
        st2["offered_rate_per_s"] = frac * cap
        st2["busy_vs_single_box"] = st2["busy_mlups"] / single
        out[key] = st2
    return out


def extra_rb3d(lbm, torch, W, peak, K=20, err_steps=100):
    """D3Q39 Rayleigh-Benard 512x512x256, FP16-scaled, z walls 1.02 / 0.98,
    g_z = -5e-6, tau 0.55; error against the same run in FP64 on the GPU."""
    stream = torch.cuda.Stream()
    w16 = W.rayleigh_benard(nx=512, ny=512, nz=256, lattice=W.D3Q39, tau=0.55, g=-5e-6,
                            T_bottom=1.02, T_top=0.98, seed=5, precision=W.FP16_SCALED)
    N = 512 * 512 * 256
    a = lbm.Sim(w16, stream=stream.cuda_stream).init()
    a.step(2)
    t = event_time(torch, stream, lambda: a.step(1), K)
    mlups = N * K / t / 1e6
    a.close()
    from paper_2302_04741_gb300 import accuracy as A
    acc = A.codec_accuracy(w16, W.FP16_SCALED, [err_steps], stream=stream.cuda_stream,
                           runs=("codec", "floor"))[err_steps]
    return {"workload": "rayleigh_benard_d3q39_512x512x256_fp16", "sites": N, "mlups": mlups,
            "roofline_frac": mlups * 1e6 * 156 / (peak * 1e9),
            "l2_vs_fp64_gpu": dict(steps=err_steps, **acc["codec"], storage_floor=acc["floor"])}


# --------------------------------------------------------------- our arm
def time_context(lbm, torch, sim, stream, flush, K, W_, inner):
    """Times K benchmark steps (after W_ warm-up ones).  Returns total device
    ms, summed ms of the step launches, and the launches counted."""
    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(K)]
    for _ in range(W_):
        sim.step(inner)
        sim.conserved()
    torch.cuda.synchronize()
    for k in range(K):
        with torch.cuda.stream(stream):
            flush.zero_()
        ev[k][0].record(stream)
        sim.step(inner)
        ev[k][1].record(stream)
        sim.conserved()
        ev[k][2].record(stream)
    torch.cuda.synchronize()
    total = sum(e[0].elapsed_time(e[2]) for e in ev)
    kern = sum(e[0].elapsed_time(e[1]) for e in ev)
    return total, kern, K * (inner + 2)


def run_ours(args):
    import torch

    rank, world, local = dist_info()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    import paper_2302_04741_gb300 as lbm
    from paper_2302_04741_gb300 import build as lbm_build
    from paper_2302_04741_gb300 import workloads as W

    if rank == 0 or world == 1:
        lbm_build.build()
    if world > 1:
        torch.distributed.barrier()
    lbm.lib()

    nx, ny, inner, K, Wm = args.nx, args.ny, args.inner, args.steps, args.warmup
    N = nx * ny
    Q = 37
    stream = torch.cuda.Stream()
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")  # 256 MiB
    w32 = W.rayleigh_benard(nx=nx, ny=ny, precision=W.FP32_SHIFTED, seed=2 + rank)
    kern = {"auto": lbm.LBM_KERNEL_AUTO, "plain": lbm.LBM_KERNEL_PLAIN, "tma": lbm.LBM_KERNEL_TMA,
            "prefetch": lbm.LBM_KERNEL_PREFETCH}
    sim = lbm.Sim(w32, stream=stream.cuda_stream, kernel=kern[args.kernel],
                  tma_stages=args.tma_stages, graph_steps=args.graph_steps,
                  block_x=args.block_x).init()

    def barrier():
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()

    barrier()
    clocks = NvmlSampler(local)
    if not clocks.start():
        clocks = ClockSampler(local)
        clocks.start()
    total_ms, kern_ms, launches = time_context(lbm, torch, sim, stream, flush, K, Wm, inner)
    barrier()
    clk = clocks.stop()
    value, t_max = aggregate_ranks(total_ms, N * inner * K, world, device="cuda")

    bytes_per_launch = 2 * Q * 4 * N
    t_launch = kern_ms / 1e3 / (K * inner)
    achieved = bytes_per_launch / t_launch / 1e9
    peak, peak_kind = measured_peak()
    traffic = profiled_traffic("k_step_fp32_rayleigh_benard_1024x512.md")
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak, "traffic": traffic,
                "peak_source": f"{peak_kind} (MEASURED_PEAKS.json hbm_gbs)" if peak_kind == "measured" else "fallback 6.8 TB/s",
                "kernel": {lbm.LBM_KERNEL_TMA: "k_step_tma", lbm.LBM_KERNEL_PREFETCH: "k_step_async"}.get(
                    lbm.lbm_step_kernel(sim.ctx), "k_step") + "<D2Q37, FP32_SHIFTED, order 2>",
                "bytes_per_launch": bytes_per_launch, "avg_launch_us": t_launch * 1e6}

    extra = {}
    # FP64 storage, same workload (the FP32/FP64 ratio of the target), with
    # the float-float step (the FP64 headline) and the IEEE double step
    if not args.no_fp64:
        from paper_2302_04741_gb300 import peaks as PK
        rates = PK.rates(reps=3)
        w64 = W.rayleigh_benard(nx=nx, ny=ny, precision=W.FP64, seed=2 + rank)
        K64 = max(2, min(K, 5))
        runs = {}
        for arith in (lbm.LBM_ARITH_FLOAT_PAIR, lbm.LBM_ARITH_DOUBLE):
            sim64 = lbm.Sim(w64, stream=stream.cuda_stream, graph_steps=args.graph_steps,
                            fp64_arith=arith).init()
            t64, k64, _ = time_context(lbm, torch, sim64, stream, flush, K64, 1, inner)
            sim64.close()
            t_launch64 = k64 / 1e3 / (K64 * inner)
            runs[arith] = (N * inner * K64 / (t64 / 1e3) / 1e6, 2 * Q * 8 * N / t_launch64 / 1e9, t_launch64)
        prof = "k_step_fp64_rayleigh_benard_1024x512.md"
        v_df, a_df, tl_df = runs[lbm.LBM_ARITH_FLOAT_PAIR]
        v_ie, a_ie, tl_ie = runs[lbm.LBM_ARITH_DOUBLE]
        # ALU roofline of the IEEE double step: its FP64 instructions per site
        # (ncu count) at the measured DFMA / DADD rate
        f64_ops = profiled_value(prof, "ieee_fp64_ops_per_site")
        alu_ie = None
        if f64_ops:
            ach = f64_ops * N / tl_ie
            alu_ie = {"bound": "fp64_alu", "achieved_ops": ach, "peak_ops": rates["dfma"],
                      "frac": ach / rates["dfma"], "fp64_ops_per_site": f64_ops,
                      "peak_source": "measured DFMA rate (peaks.py, this run)"}
        # the float-float step is bound by instruction issue: thread
        # instructions per site (ncu count) against 128 per SM per clock
        inst = profiled_value(prof, "float_pair_inst_per_site")
        alu_df = None
        nsm = torch.cuda.get_device_properties(local).multi_processor_count
        clk_hz = float((clk or {}).get("sm_mhz") or 2070.0) * 1e6
        if inst:
            ach = inst * N / tl_df
            pk = 128.0 * nsm * clk_hz
            alu_df = {"bound": "issue", "achieved_inst": ach, "peak_inst": pk, "frac": ach / pk,
                      "inst_per_site": inst, "peak_source": "4 warp instructions per SM per clock x median SM clock"}
        extra["fp64"] = {"value": v_df, "unit": "MLUPS", "arith": "float_pair (lbm_options.fp64_arith)",
                         "roofline_frac_hbm": a_df / peak, "achieved_gbs": a_df, "roofline_alu": alu_df,
                         "ratio_fp32_over_fp64": value / world / v_df,
                         "ieee_double": {"value": v_ie, "unit": "MLUPS", "roofline_frac_hbm": a_ie / peak,
                                         "achieved_gbs": a_ie, "roofline_alu": alu_ie},
                         "measured_rates_tops": {k: v / 1e12 for k, v in rates.items()}}
        # accuracy of the FP32-shifted run against the FP64 run over the
        # configuration's full 20k steps, with the FP64 butterfly floor and the
        # FP32 storage floor (paper_2302_04741_gb300.accuracy)
        from paper_2302_04741_gb300 import accuracy as A
        if not args.no_accuracy:
            acc = A.codec_accuracy(w32, W.FP32_SHIFTED, [1000, 20000], stream=stream.cuda_stream,
                                   graph_steps=args.graph_steps)
            extra["l2_fp32_vs_fp64_gpu"] = {
                "steps": 20000, **acc[20000]["codec"], "at_1000_steps": acc[1000]["codec"],
                "butterfly_floor": acc[20000]["butterfly"], "storage_floor": acc[20000]["floor"],
                "note": "relative L2 against the FP64 GPU run of the same grid (itself oracle-checked); "
                        "butterfly = FP64 with a 1e-15 initial perturbation; storage floor = FP64 "
                        "arithmetic with FP32 storage rounding"}

    # end to end: host arrays in, moments out, through the C ABI
    pin = lambda a: torch.from_numpy(np.ascontiguousarray(a)).pin_memory()
    h_in = [pin(w32["rho"]), pin(w32["u"]), pin(w32["T"])]
    h_out = [torch.empty(N, dtype=torch.float64).pin_memory(),
             torch.empty(2 * N, dtype=torch.float64).pin_memory(),
             torch.empty(N, dtype=torch.float64).pin_memory(),
             torch.empty(2 * N, dtype=torch.float64).pin_memory()]
    e2e_sim = lbm.Sim(w32, stream=stream.cuda_stream)
    Ke = max(3, K // 4)
    lbm.lbm_init(e2e_sim.ctx, *h_in)
    e2e_sim.step(inner)
    lbm.lbm_moments(e2e_sim.ctx, *h_out)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(Ke):
        lbm.lbm_init(e2e_sim.ctx, *h_in)
        e2e_sim.step(inner)
        lbm.lbm_moments(e2e_sim.ctx, *h_out)
    e1.record(stream)
    torch.cuda.synchronize()
    e2e_ms = e0.elapsed_time(e1)
    e2e = {"value": world * N * inner * Ke / (e2e_ms / 1e3) / 1e6, "unit": "MLUPS",
           "h2d_bytes_per_step": 4 * N * 8, "d2h_bytes_per_step": 6 * N * 8,
           "step": f"lbm_init(pinned host rho,u,T) + lbm_step({inner}) + lbm_moments(pinned host)"}
    # the read-out kernel alone, into device memory (k_moments: Q float
    # populations in, rho, u, T, q as doubles out)
    d_out = [torch.empty(n, dtype=torch.float64, device="cuda") for n in (N, 2 * N, N, 2 * N)]
    lbm.lbm_moments_async(e2e_sim.ctx, *d_out)
    Km = 20
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(Km):
        lbm.lbm_moments_async(e2e_sim.ctx, *d_out)
    e1.record(stream)
    torch.cuda.synchronize()
    mom_us = e0.elapsed_time(e1) * 1e3 / Km
    mom_bytes = N * (37 * 4 + 6 * 8)
    e2e["k_moments_device"] = {"us": mom_us, "bytes": mom_bytes,
                               "hbm_frac": mom_bytes / (mom_us * 1e-6) / (peak * 1e9),
                               "note": "lbm_moments_async into device memory, 20 launches, CUDA events"}
    e2e_sim.close()

    configs = {}
    if not args.no_extras:
        configs["kolmogorov"] = extra_kolmogorov(lbm, torch, W, peak)
        configs["ragged_batch"] = extra_ragged(lbm, torch, W, peak, value / world)
        configs["serving"] = extra_serving(lbm, torch, W, peak, args.serve_requests)
        configs["rb3d_fp16"] = extra_rb3d(lbm, torch, W, peak)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        mlups, steps, dt, cores = oracle_rate(W.rayleigh_benard(nx=nx, ny=ny, precision=W.FP64),
                                              40, 0, budget_s=12.0)
        m1, s1, d1, _ = oracle_rate(W.rayleigh_benard(nx=256, ny=128, precision=W.FP64),
                                    40, 0, budget_s=4.0, threads=1)
        cpu = {"value": mlups, "unit": "MLUPS", "cores": cores, "kind": "oracle",
               "sample": f"FP64 oracle, full {nx}x{ny} grid, {steps} LBM steps ({dt:.1f} s)",
               "single_thread": {"value": m1, "unit": "MLUPS",
                                 "sample": f"256x128 grid of the same workload, {s1} steps ({d1:.1f} s)"},
               "cpu_model": cpu_model()}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "MLUPS", "n_gpus": world, "steps": K,
            "warmup": Wm, "ms_per_step": t_max / K, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": f"rayleigh_benard_d2q37_{nx}x{ny}", "lattice": "D2Q37",
                       "grid": [nx, ny], "precision": "fp32_shifted", "tau_hat": 0.6,
                       "g": [0.0, -1e-5], "walls": "thermal y (1.05 / 0.95), periodic x",
                       "force_order": 2, "inner_lbm_steps_per_step": inner,
                       "step": f"lbm_step({inner}) + lbm_conserved",
                       "graph_steps": args.graph_steps,
                       "l2": "256 MiB flush before every timed step (outside the timed interval); "
                             "working set 2 x 77.6 MB",
                       "parallelism": f"{world} independent grids" if world > 1 else "1 grid"},
            "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches,
            "clocks": clk,
        }
        line.update(extra)
        if configs:
            line["configs"] = configs
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


def main():
    args = parse_args()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
