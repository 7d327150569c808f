"""Slab decomposition of one grid along its last axis: every slab steps its
own layers with the plain step kernel and a halo exchange per cut supplies
the three layers each slab pulls from its neighbours (Eq. lbm is local).
The slabs must reproduce the undivided grid bit for bit; their conservation
sums, added, must equal the grid's to rounding."""
import numpy as np
import pytest

import paper_2302_04741_gb300 as lbm
from paper_2302_04741_gb300 import slabs as SL
from paper_2302_04741_gb300 import workloads as W
from helpers import workload

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    pytest.importorskip("torch")
    from paper_2302_04741_gb300 import build
    build.build()


def field_g(lat, shape, seed=5, amp=3e-5):
    D = W.dims(lat)
    N = shape[0] * shape[1] * shape[2]
    return {"kind": W.G_FIELD, "field": amp * (W.uniform(seed, 30, D * N).reshape(D, N) - 0.5)}


SINE_LAST = {2: {"kind": W.G_SINE, "g0": (3e-5, 0.0, 0.0), "wave_axis": 1},
             3: {"kind": W.G_SINE, "g0": (3e-5, 1e-5, 0.0), "wave_axis": 2}}

CASES = [
    # (id, lattice, shape, bc, precision, force, cuts)
    ("d2-periodic-2", 0, (40, 24, 1), (0, 0, 0), 0, None, 2),
    ("d2-periodic-3-sine", 0, (33, 30, 1), (0, 0, 0), 0, "sine", 3),
    ("d2-periodic-1", 0, (20, 12, 1), (0, 0, 0), 0, None, 1),
    ("d2-thermal-3", 0, (50, 27, 1), (0, 2, 0), 0, None, 3),
    ("d2-bounce-2-field", 0, (37, 20, 1), (0, 1, 0), 0, "field", 2),
    ("d2-thermal-uneven-fp32", 0, (64, 40, 1), (0, 2, 0), 1, None, [(0, 3), (3, 31), (31, 40)]),
    ("d3-thermal-2", 1, (12, 10, 16), (0, 0, 2), 0, None, 2),
    ("d3-periodic-3-sine-fp32", 1, (10, 9, 18), (0, 0, 0), 1, "sine", 3),
    ("d3-periodic-2-fp16", 1, (16, 12, 14), (0, 0, 0), 2, None, 2),
]


def make(case):
    _, lat, shape, bc, prec, force, cuts = case
    D = W.dims(lat)
    g = None
    if force == "sine":
        g = SINE_LAST[D]
    elif force == "field":
        g = field_g(lat, shape)
    return workload(lat, shape, tau=0.7, g=g, seed=21, precision=prec, bc=bc,
                    T_lo=(1.0, 1.06, 1.06), T_hi=(1.0, 0.95, 0.95)), cuts


@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
def test_slabs_reproduce_the_grid_bitwise(case):
    import torch
    w, cuts = make(case)
    stream = torch.cuda.Stream()
    whole = lbm.Sim(w, stream=stream.cuda_stream).init()
    grid = SL.SlabGrid(w, cuts, stream=stream.cuda_stream).init()
    for n in (1, 4, 7):
        whole.step(n)
        grid.step(n)
        a, b = whole.moments(), grid.moments()
        for name, x, y in zip(("rho", "u", "T", "q"), a, b):
            np.testing.assert_array_equal(x, y, err_msg=f"{case[0]} {name}")
    st, mass, mom, energy = whole.conserved()
    m2, p2, e2 = grid.conserved()
    tol = 1e-13 if w["precision"] == W.FP64 else 1e-12
    assert abs(m2 - mass) <= tol * mass and abs(e2 - energy) <= tol * energy
    np.testing.assert_allclose(p2, mom, rtol=0, atol=tol * mass)
    grid.close()
    whole.close()


def test_pack_unpack_equals_direct_exchange():
    """The exchange through messages (the path between devices or processes:
    pack, move the bytes, unpack) gives the same state as the direct
    same-device exchange."""
    import torch
    w, _ = make(CASES[3])
    stream = torch.cuda.Stream()
    direct = SL.SlabGrid(w, 3, stream=stream.cuda_stream).init()
    msg = SL.SlabGrid(w, 3, stream=stream.cuda_stream).init()
    nbytes = lbm.lbm_slab_halo_bytes(msg.ctx[0])
    assert nbytes == lbm.lbm_slab_halo_bytes(msg.ctx[1]) > 0
    bufs = {k: torch.empty(nbytes, dtype=torch.uint8, device="cuda") for k in ("up", "down")}
    for _ in range(6):
        direct.step(1)
        for c in msg.ctx:
            lbm.lbm_step(c, 1)
        for lo, hi in msg.cuts:
            lbm.lbm_slab_halo_pack(msg.ctx[lo], 1, bufs["up"])
            lbm.lbm_slab_halo_pack(msg.ctx[hi], 0, bufs["down"])
            lbm.lbm_slab_halo_unpack(msg.ctx[hi], 0, bufs["up"])
            lbm.lbm_slab_halo_unpack(msg.ctx[lo], 1, bufs["down"])
    for x, y in zip(direct.moments(), msg.moments()):
        np.testing.assert_array_equal(x, y)
    direct.close()
    msg.close()


def test_slab_rejections():
    w, _ = make(CASES[3])  # thermal walls on y
    lat, shape = w["lattice"], w["shape"]
    opt = lbm.options(0, 2, w["bc"], w["T_lo"], w["T_hi"])
    lo = lbm.lbm_create_slab(lat, *shape, 0, 10, 0.7, None, opt)
    hi = lbm.lbm_create_slab(lat, *shape, 12, 27, 0.7, None, opt)
    try:
        assert lbm.lbm_slab_info(lo) == (0, 10, 0, 3)
        assert lbm.lbm_slab_info(hi) == (12, 27, 3, 0)
        rho, u, T = w["rho"], w["u"], w["T"]
        S = shape[0]
        lbm.lbm_init(lo, rho[:10 * S].copy(), np.ascontiguousarray(u[:, :10 * S]), T[:10 * S].copy())
        lbm.lbm_init(hi, rho[12 * S:].copy(), np.ascontiguousarray(u[:, 12 * S:]), T[12 * S:].copy())
        with pytest.raises(lbm.LbmError) as ei:   # not adjacent
            lbm.lbm_slab_exchange(lo, hi)
        assert ei.value.status == lbm.LBM_EINVAL
        import torch
        buf = torch.empty(lbm.lbm_slab_halo_bytes(lo), dtype=torch.uint8, device="cuda")
        with pytest.raises(lbm.LbmError) as ei:   # the bottom slab has a wall below
            lbm.lbm_slab_halo_pack(lo, 0, buf)
        assert ei.value.status == lbm.LBM_EINVAL
    finally:
        lbm.lbm_destroy(lo)
        lbm.lbm_destroy(hi)
