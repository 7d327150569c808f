"""Full-length accuracy of the reduced-precision codecs against FP64 on the
GPU, with the butterfly floor (FP64 with a 1e-15 initial perturbation: the
flow's own sensitivity) and the storage floor (FP64 arithmetic with the
codec's storage rounding: lbm_options.storage_probe).

Measured on GB300 (the numbers the bounds below guard):
  D2Q37 Rayleigh-Benard 1024 x 512, FP32-shifted, 20k steps:
    codec   rho 4.6e-7  u 2.3e-5  T 5.1e-7  q 8.2e-5
    floor   rho 1.2e-9  u 1.3e-7  T 1.2e-9  q 1.9e-6
    butterfly < 2e-13
  The FP32 u and q errors lie ~100x above the storage floor: the float
  arithmetic of the collision, not the storage, limits FP32 at this length
  (a stable flow: the butterfly floor stays at 1e-13).
  D3Q39 Rayleigh-Benard 512 x 512 x 256, FP16-scaled, 10k steps:
    1,000 steps   rho 5.8e-6  u 9.3e-4  T 4.6e-6  q 9.6e-3  (floor: 5.6e-6 9.2e-4 4.5e-6 9.6e-3)
    10,000 steps  rho 4.7e-5  u 3.0e-3  T 5.1e-5  q 1.5e-2
  FP16 sits on its storage floor: 11 bits per scaled deviation.
"""
import os
import tempfile

import numpy as np
import pytest

import paper_2302_04741_gb300 as lbm
from paper_2302_04741_gb300 import accuracy as A
from paper_2302_04741_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    pytest.importorskip("torch")
    from paper_2302_04741_gb300 import build
    build.build()


def raw_doubles(sim):
    with tempfile.TemporaryDirectory() as d:
        path = os.path.join(d, "s.ckpt")
        lbm.lbm_save(sim.ctx, path)
        data = open(path, "rb").read()
    n = sim.Q * sim.N * 8
    return np.frombuffer(data[len(data) - n:], dtype=np.float64).reshape(sim.Q, sim.N)


def test_storage_probe_stores_float_deviations():
    """With the FP32 probe every stored deviation f - w is a float (up to the
    rounding of the double sum w + d), and the run differs from plain FP64."""
    w = W.rayleigh_benard(nx=96, ny=32, precision=W.FP64, T_bottom=1.05, T_top=0.95, g=-1e-4,
                          T_noise=1e-3)
    probe = lbm.Sim(w, storage_probe=W.FP32_SHIFTED).init()
    plain = lbm.Sim(w).init()
    probe.step(30)
    plain.step(30)
    f = raw_doubles(probe)
    d = f - probe.wts[:, None]
    assert np.max(np.abs(d - d.astype(np.float32).astype(np.float64))) <= 1e-16
    dp = raw_doubles(plain) - plain.wts[:, None]
    assert np.max(np.abs(dp - dp.astype(np.float32).astype(np.float64))) > 1e-12
    errs = A.rel_errors(probe.moments(), plain.moments())
    assert 0 < errs["rho"] < 1e-7 and errs["u"] < 1e-5


def test_storage_probe_fp16_matches_the_codec_floor():
    """The FP16 probe (half of s d / w, the codec's scale) costs what the FP16
    codec costs: on this thermal cell the codec's error equals its storage
    floor within a factor 2 (its float arithmetic is far finer than half)."""
    import torch
    w, prec = A.workload("rb3d")
    w = W.rayleigh_benard(nx=64, ny=64, nz=48, lattice=W.D3Q39, tau=0.55, g=-5e-6, T_bottom=1.02,
                          T_top=0.98, seed=5, precision=W.FP16_SCALED)
    s = torch.cuda.Stream()
    res = A.codec_accuracy(w, W.FP16_SCALED, [200], stream=s.cuda_stream, runs=("codec", "floor"))
    codec, floor = res[200]["codec"], res[200]["floor"]
    for k in ("rho", "u", "T", "q"):
        assert 0 < floor[k] <= 2 * codec[k] and codec[k] <= 2 * floor[k], (k, codec, floor)


def test_rb2d_fp32_full_length_accuracy():
    """D2Q37 Rayleigh-Benard 1024 x 512, FP32-shifted, the full 20k steps."""
    import torch
    w, prec = A.workload("rb2d")
    s = torch.cuda.Stream()
    res = A.codec_accuracy(w, prec, [20000], stream=s.cuda_stream)
    r = res[20000]
    assert all(v <= 1e-12 for v in r["butterfly"].values()), r["butterfly"]
    assert r["floor"]["rho"] <= 1e-8 and r["floor"]["T"] <= 1e-8 and r["floor"]["u"] <= 1e-6
    assert r["floor"]["q"] <= 5e-6
    assert r["codec"]["rho"] <= 1e-6 and r["codec"]["T"] <= 1e-6
    # u and q: the FP32 arithmetic floor, guarded at about twice the measured value
    assert r["codec"]["u"] <= 5e-5 and r["codec"]["q"] <= 2e-4, r["codec"]


def test_rb3d_fp16_full_size_accuracy():
    """D3Q39 Rayleigh-Benard 512 x 512 x 256, FP16-scaled, against the
    float-float FP64 step (which agrees with IEEE double to ~1e-12 over this
    length): 1,000 steps, and at 100 steps the codec's error against its
    storage floor.  The full 10,000-step run is the committed command
    `python -m paper_2302_04741_gb300.accuracy rb3d --steps 10000
    --checkpoints 1000 5000 --runs codec --ref-arith 1` (about six minutes on
    GB300), whose result is the table in the module docstring."""
    import torch
    w, prec = A.workload("rb3d")
    s = torch.cuda.Stream()
    res = A.codec_accuracy(w, prec, [1000], stream=s.cuda_stream, runs=("codec",),
                           ref_arith=lbm.LBM_ARITH_FLOAT_PAIR)
    r1 = res[1000]["codec"]
    assert r1["rho"] <= 1e-5 and r1["T"] <= 1e-5 and r1["u"] <= 2e-3 and r1["q"] <= 2e-2, r1
    res = A.codec_accuracy(w, prec, [100], stream=s.cuda_stream, runs=("codec", "floor"),
                           ref_arith=lbm.LBM_ARITH_FLOAT_PAIR)
    codec, floor = res[100]["codec"], res[100]["floor"]
    for k in ("rho", "u", "T", "q"):
        assert 0 < floor[k] <= 1.1 * codec[k] and codec[k] <= 1.1 * floor[k], (k, codec, floor)
