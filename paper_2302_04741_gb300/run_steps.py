"""Runs a few plain steps of one configuration (for profilers: a fixed,
small launch sequence of the step kernel).

    python -m paper_2302_04741_gb300.run_steps --config rb2d --precision fp64 --steps 3
    python -m paper_2302_04741_gb300.run_steps --config rb2d --precision fp32 --steps 3 --moments 20
    python -m paper_2302_04741_gb300.run_steps --config rb3d --precision fp32 --steps 3 --time 20
"""
import argparse

from paper_2302_04741_gb300 import workloads as W

PRECISIONS = {"fp64": W.FP64, "fp32": W.FP32_SHIFTED, "fp16": W.FP16_SCALED}


def workload(config, precision, nx=None, ny=None, nz=None):
    if config == "rb2d":
        return W.rayleigh_benard(nx=nx or 1024, ny=ny or 512, precision=precision)
    if config == "rb3d":
        return W.rayleigh_benard(nx=nx or 512, ny=ny or 512, nz=nz or 256, lattice=W.D3Q39, tau=0.55,
                                 g=-5e-6, T_bottom=1.02, T_top=0.98, seed=5, precision=precision)
    raise ValueError(config)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--config", default="rb2d", choices=["rb2d", "rb3d"])
    ap.add_argument("--precision", default="fp32", choices=sorted(PRECISIONS))
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--nx", type=int, default=None)
    ap.add_argument("--ny", type=int, default=None)
    ap.add_argument("--nz", type=int, default=None)
    ap.add_argument("--arith", type=int, default=None, help="lbm_options.fp64_arith (FP64 storage)")
    ap.add_argument("--time", type=int, default=0,
                    help="then K more steps timed with CUDA events (MLUPS and algorithmic GB/s)")
    ap.add_argument("--moments", type=int, default=0,
                    help="then K read-outs into device memory (lbm_moments_async), timed with CUDA events")
    args = ap.parse_args()
    import torch
    import paper_2302_04741_gb300 as lbm
    from paper_2302_04741_gb300 import build
    build.build()
    w = workload(args.config, PRECISIONS[args.precision], args.nx, args.ny, args.nz)
    kw = {} if args.arith is None else {"fp64_arith": args.arith}
    sim = lbm.Sim(w, overlap_steps=0, **kw).init()
    sim.step(args.steps)
    torch.cuda.synchronize()
    st = sim.conserved()
    print("ok", args.config, args.precision, args.steps, "mass", st[1])
    elem = {W.FP64: 8, W.FP32_SHIFTED: 4, W.FP16_SCALED: 2}[PRECISIONS[args.precision]]
    if args.time > 0:
        stream = torch.cuda.current_stream()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        sim.step(args.time)
        e1.record(stream)
        torch.cuda.synchronize()
        us = e0.elapsed_time(e1) * 1e3 / args.time
        print(f"time {args.time} x {us:.2f} us per step, {sim.N / us:.1f} MLUPS, "
              f"{sim.N * 2 * sim.Q * elem / us / 1e3:.1f} GB/s algorithmic")
    if args.moments > 0:
        D, N = sim.D, sim.N
        rho = torch.empty(N, dtype=torch.float64, device="cuda")
        u = torch.empty(D * N, dtype=torch.float64, device="cuda")
        T = torch.empty(N, dtype=torch.float64, device="cuda")
        q = torch.empty(D * N, dtype=torch.float64, device="cuda")
        out = (rho, u, T, q)
        stream = torch.cuda.current_stream()
        lbm.lbm_moments_async(sim.ctx, *out)  # warm-up (the context's stream)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.moments):
            lbm.lbm_moments_async(sim.ctx, *out)
        e1.record(stream)
        torch.cuda.synchronize()
        us = e0.elapsed_time(e1) * 1e3 / args.moments
        nbytes = N * (sim.Q * elem + (2 + 2 * D) * 8)
        print(f"moments {args.moments} x {us:.2f} us per read-out, {nbytes / us / 1e3:.1f} GB/s algorithmic")
    sim.close()


if __name__ == "__main__":
    main()
