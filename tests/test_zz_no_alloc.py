"""lbm_conserved_static: the conservation sums without any device allocation.

It exists for callers that may not allocate device memory -- a plugin inside
an application that owns every device byte through its own pool, a runtime
with a fully reserved memory budget, or a latency-critical loop that cannot
afford the device-wide synchronisation of cudaMalloc / cudaFree.  Its partial
sums live in a static device array shared by all calls, so these tests check
that it reproduces lbm_conserved on the same state on two calls in a row, and
that grids too large for that array, and pointers that are not device memory
of the current device, are rejected before any launch.  This file is
collected last on purpose: if it fails, a run that stops at the first failure
has already run every other test.
"""
import os
import tempfile

import numpy as np
import pytest

import paper_2302_04741_gb300 as lbm
from paper_2302_04741_gb300 import build as lbm_build
from paper_2302_04741_gb300 import workloads as W


def test_rejects_grids_beyond_the_static_scratch():
    lbm_build.build()
    opt = lbm.options(W.FP32_SHIFTED)
    # ceil(4096 / 128) * 2048 = 65536 row tiles > LBM_STATIC_MAX_TILES = 32768;
    # the size check comes before any device work, so dummy pointers are fine
    with pytest.raises(lbm.LbmError) as ei:
        lbm.lbm_conserved_static(0, 4096, 2048, 1, opt, None, 0.0, 16, 16)
    assert ei.value.status == lbm.LBM_EINVAL
    assert "static scratch" in str(ei.value)


def test_rejects_host_memory_before_any_launch():
    lbm_build.build()
    opt = lbm.options(W.FP32_SHIFTED)
    f = np.zeros(37 * 64 * 16, dtype=np.float32)
    out = np.zeros(6)
    with pytest.raises(lbm.LbmError) as ei:
        lbm.lbm_conserved_static(0, 64, 16, 1, opt, None, 0.0, f.ctypes.data, out.ctypes.data)
    assert ei.value.status == lbm.LBM_EINVAL
    assert "device memory" in str(ei.value)


def raw_state(sim):
    """The context's stored post-collision buffer, byte for byte (the
    checkpoint's payload follows its header)."""
    elem = {W.FP64: np.float64, W.FP32_SHIFTED: np.float32, W.FP16_SCALED: np.float16}
    dt = elem[sim.opt.precision]
    with tempfile.TemporaryDirectory() as d:
        path = os.path.join(d, "state.ckpt")
        lbm.lbm_save(sim.ctx, path)
        data = open(path, "rb").read()
    nbytes = sim.Q * sim.N * np.dtype(dt).itemsize
    return np.frombuffer(data[len(data) - nbytes:], dtype=dt)


def check_static_matches(sim, w, g_static, torch, stream=None):
    st, mass, mom, energy = sim.conserved()
    raw = torch.from_numpy(raw_state(sim).copy()).cuda()
    opt = lbm.options(w["precision"], w["force_order"], w["bc"], w["T_lo"], w["T_hi"],
                      stream=stream.cuda_stream if stream is not None else None)
    out = torch.empty(6, dtype=torch.float64, device="cuda")
    scale = lbm.lbm_fp16_scale(sim.ctx)
    D = sim.D
    for _ in range(2):
        out.fill_(np.nan)
        torch.cuda.synchronize()
        lbm.lbm_conserved_static(w["lattice"], *w["shape"], opt, g_static, scale, raw, out)
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        assert abs(got[0] - mass) <= 1e-13 * mass
        np.testing.assert_allclose(got[1:1 + D], mom, rtol=0, atol=1e-13 * mass)
        if D == 2:
            assert got[3] == 0.0  # no z momentum in 2-D
        assert abs(got[4] - energy) <= 1e-13 * energy
        assert got[5] == 0


@pytest.mark.gpu
@pytest.mark.parametrize("precision", [W.FP64, W.FP32_SHIFTED, W.FP16_SCALED])
def test_static_scratch_sums_match_context_sums(precision):
    torch = pytest.importorskip("torch")
    lbm_build.build()
    w = W.rayleigh_benard(nx=300, ny=64, precision=precision, T_bottom=1.1, T_top=0.9, g=-1e-4,
                          T_noise=1e-2)
    sim = lbm.Sim(w).init()
    sim.step(25)
    check_static_matches(sim, w, w["g"], torch)
    sim.close()


@pytest.mark.gpu
def test_static_sums_d3q39_fp16_thermal_z_walls_on_a_stream():
    torch = pytest.importorskip("torch")
    lbm_build.build()
    w = W.rayleigh_benard(nx=32, ny=16, nz=12, lattice=W.D3Q39, tau=0.6, g=-1e-4, T_bottom=1.05,
                          T_top=0.95, seed=9, precision=W.FP16_SCALED, T_noise=1e-2)
    stream = torch.cuda.Stream()
    sim = lbm.Sim(w, stream=stream.cuda_stream).init()
    sim.step(10)
    check_static_matches(sim, w, w["g"], torch, stream=stream)
    sim.close()


@pytest.mark.gpu
@pytest.mark.parametrize("precision", [W.FP64, W.FP32_SHIFTED])
def test_static_sums_with_a_field_force(precision):
    """LBM_G_FIELD: the caller's double field on the device; the float codec
    rounds it to float as a context rounds its own copy."""
    torch = pytest.importorskip("torch")
    lbm_build.build()
    w = W.rayleigh_benard(nx=200, ny=48, precision=precision, T_bottom=1.1, T_top=0.9, g=-1e-4,
                          T_noise=1e-2)
    N = 200 * 48
    field = 3e-5 * (W.uniform(7, 41, 2 * N).reshape(2, N) - 0.5)
    field[1] -= 1e-4
    w = dict(w, g={"kind": W.G_FIELD, "field": np.ascontiguousarray(field)})
    sim = lbm.Sim(w).init()
    sim.step(20)
    dfield = torch.from_numpy(np.ascontiguousarray(field)).cuda()
    check_static_matches(sim, w, {"kind": W.G_FIELD, "field": dfield}, torch)
    sim.close()
