"""Accuracy of a reduced-precision population codec against FP64, with the two
floors that separate its error from other causes.

For a workload and a codec (LBM_FP32_SHIFTED or LBM_FP16_SCALED), four runs
of the same initial state are stepped side by side on the GPU:

  codec       the workload in the codec (its own storage and arithmetic);
  fp64        the workload in FP64 (the reference);
  butterfly   FP64 with the initial temperature perturbed by a relative
              1e-15: its distance from fp64 is the physical sensitivity of
              the flow to a perturbation at the FP64 rounding level (a
              chaotic flow amplifies it; a stable one keeps it near 1e-15);
  floor       FP64 arithmetic whose stored deviations are rounded to the
              codec's format after every step (lbm_options.storage_probe):
              its distance from fp64 is what the codec's storage alone
              costs, the codec's storage floor.

The reported errors are relative L2 norms over all sites and components of
rho, u, T and q, with q normalised by max(||q_fp64||, 1e-3 Ma sqrt(D N)) (a
nearly zero reference flux compared at the scale of the flow).

Command line (one configuration at a time):
    python -m paper_2302_04741_gb300.accuracy rb2d --steps 20000
    python -m paper_2302_04741_gb300.accuracy rb3d --steps 10000
"""
import argparse
import json
import math
import time

import numpy as np


def rel_errors(a, b):
    """Relative L2 of (rho, u, T, q) tuples a against b; q normalised by
    max(||q_b||, 1e-3 max(|u_b|, 1e-3) sqrt(size))."""
    qf = 1e-3 * max(float(np.abs(b[1]).max()), 1e-3) * math.sqrt(b[1].size)
    out = {}
    for nm, x, y in zip(("rho", "u", "T", "q"), a, b):
        fl = qf if nm == "q" else 0.0
        out[nm] = float(np.linalg.norm(x - y) / max(np.linalg.norm(y), fl))
    return out


def codec_accuracy(w, precision, checkpoints, stream=None, graph_steps=10, butterfly=1e-15,
                   runs=("codec", "butterfly", "floor"), ref_arith=0):
    """Errors against FP64 of the runs named in ``runs`` at each step count of
    ``checkpoints`` (increasing).  ``w`` is a workload dict (its precision
    field is ignored).  ref_arith: lbm_options.fp64_arith of the FP64
    reference and butterfly runs (the float-float step agrees with IEEE
    double to ~1e-12 and runs about twice as fast on GB300); the floor run
    uses IEEE double (the storage probe).  Returns {steps: {run: {rho, u, T,
    q}}} plus "seconds"."""
    import paper_2302_04741_gb300 as lbm
    from paper_2302_04741_gb300 import workloads as W

    sims = {}
    t0 = time.time()
    try:
        mk = lambda ww, **kw: lbm.Sim(ww, stream=stream, graph_steps=graph_steps, **kw).init()
        sims["fp64"] = mk(dict(w, precision=W.FP64, fp64_arith=ref_arith))
        if "codec" in runs:
            sims["codec"] = mk(dict(w, precision=precision))
        if "butterfly" in runs:
            sims["butterfly"] = mk(dict(w, precision=W.FP64, fp64_arith=ref_arith,
                                        T=np.asarray(w["T"]) * (1.0 + butterfly)))
        if "floor" in runs:
            sims["floor"] = mk(dict(w, precision=W.FP64), storage_probe=precision)
        out = {}
        done = 0
        for n in checkpoints:
            for s in sims.values():
                s.step(n - done)
            done = n
            ref = sims["fp64"].moments()
            out[n] = {k: rel_errors(s.moments(), ref) for k, s in sims.items() if k != "fp64"}
            out[n]["max_abs_u"] = float(np.abs(ref[1]).max())
        out["seconds"] = time.time() - t0
        return out
    finally:
        for s in sims.values():
            s.close()


def workload(name, seed=None):
    """The configurations whose full-length accuracy is reported: rb2d, the
    D2Q37 Rayleigh-Benard cell 1024 x 512 (FP32-shifted, 20k steps), and
    rb3d, the D3Q39 Rayleigh-Benard cell 512 x 512 x 256 (FP16-scaled, 10k
    steps)."""
    from paper_2302_04741_gb300 import workloads as W
    if name == "rb2d":
        return W.rayleigh_benard(precision=W.FP32_SHIFTED, seed=2 if seed is None else seed), W.FP32_SHIFTED
    if name == "rb3d":
        return (W.rayleigh_benard(nx=512, ny=512, nz=256, lattice=W.D3Q39, tau=0.55, g=-5e-6, T_bottom=1.02,
                                  T_top=0.98, seed=5 if seed is None else seed, precision=W.FP16_SCALED),
                W.FP16_SCALED)
    raise ValueError(f"unknown configuration {name!r}")


def main():
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("config", choices=["rb2d", "rb3d"])
    ap.add_argument("--steps", type=int, required=True)
    ap.add_argument("--checkpoints", type=int, nargs="*", default=None)
    ap.add_argument("--runs", default="codec,butterfly,floor")
    ap.add_argument("--ref-arith", type=int, default=0, help="fp64_arith of the FP64 reference")
    ap.add_argument("--out", default=None, help="write the result as JSON here")
    args = ap.parse_args()
    import torch
    from paper_2302_04741_gb300 import build
    build.build()
    w, prec = workload(args.config)
    cps = sorted(set((args.checkpoints or []) + [args.steps]))
    s = torch.cuda.Stream()
    res = codec_accuracy(w, prec, cps, stream=s.cuda_stream, runs=tuple(args.runs.split(",")),
                         ref_arith=args.ref_arith)
    res = {"config": args.config, "precision": prec, "steps": args.steps, "ref_arith": args.ref_arith,
           **{str(k): v for k, v in res.items()}}
    text = json.dumps(res, indent=1)
    print(text)
    if args.out:
        with open(args.out, "w") as fh:
            fh.write(text + "\n")


if __name__ == "__main__":
    main()
