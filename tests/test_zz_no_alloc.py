"""lbm_conserved_static: the conservation sums without any device allocation.

It exists for callers that may not allocate device memory -- a plugin inside
an application that owns every device byte through its own pool, a runtime
with a fully reserved memory budget, or a latency-critical loop that cannot
afford the device-wide synchronisation of cudaMalloc / cudaFree.  Its partial
sums live in a static device array shared by all calls, so these tests check
that it reproduces lbm_conserved on the same state on two calls in a row, and
that grids too large for that array are rejected.  This file is collected
last on purpose: if it fails, a run that stops at the first failure has
already run every other test.
"""
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


@pytest.mark.gpu
@pytest.mark.parametrize("precision", [W.FP64, W.FP32_SHIFTED])
def test_static_scratch_sums_match_context_sums(precision):
    torch = pytest.importorskip("torch")
    lbm_build.build()
    w = W.rayleigh_benard(nx=300, ny=64, precision=precision, T_bottom=1.1, T_top=0.9, g=-1e-4,
                          T_noise=1e-2)
    sim = lbm.Sim(w).init()
    sim.step(25)
    st, mass, mom, energy = sim.conserved()
    # the raw device buffer in the library's storage format, rebuilt from the
    # decoded state (exact for both codecs)
    f = sim.get_state()
    if precision == W.FP64:
        raw = torch.from_numpy(np.ascontiguousarray(f)).cuda()
    else:
        raw = torch.from_numpy(np.ascontiguousarray((f - sim.wts[:, None]).astype(np.float32))).cuda()
    opt = lbm.options(precision, w["force_order"], w["bc"], w["T_lo"], w["T_hi"])
    out = torch.empty(6, dtype=torch.float64, device="cuda")
    for _ in range(2):
        out.fill_(np.nan)
        lbm.lbm_conserved_static(w["lattice"], *w["shape"], opt, w["g"], 0.0, raw, out)
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        assert abs(got[0] - mass) <= 1e-13 * mass
        np.testing.assert_allclose(got[1:3], mom, rtol=0, atol=1e-13 * mass)
        assert abs(got[4] - energy) <= 1e-13 * energy
        assert got[5] == 0
