"""Parity of the CUDA path (through the C ABI) with the FP64 CPU oracle.

Tolerances (relative L2 over all sites and components of rho, u, T, q):
FP64 1e-12, FP32-shifted 1e-6, FP16-scaled 1e-3.  The heat flux q is
normalised by max(||q_ref||, 1e-3 * Ma * sqrt(D N)) so that a nearly zero
reference flux is compared in absolute terms at the scale of the flow, and
its check adds the forward-error bound of its defining FP64 sum,
8 eps_64 sum_i |f~_i| |xi_i - u|^3 per site: q is a strongly cancelling sum
(terms ~ w |xi|^3, result ~ 1e-5 in the Kolmogorov run), so its round-off
floor lies above 1e-12 * ||q|| even when the state agrees to 1e-13.  For
the float codecs the q bound also adds the error the codec's rounding of the
stored deviations can cause in that sum (helpers.q_codec_bound): twice the
rms of one half-precision rounding for FP16 (storage-dominated), the
first-order worst case of one float rounding for FP32 (arithmetic-dominated).
"""
import os
import tempfile

import numpy as np
import pytest

import oracle
import paper_2302_04741_gb300 as lbm
from paper_2302_04741_gb300 import workloads as W
from helpers import (check_fields, compare_fields, oracle_sim, perm_to_oracle, q_floor,
                     q_roundoff, rel_l2, workload)

pytestmark = pytest.mark.gpu

TOL = {0: 1e-12, 1: 1e-6, 2: 1e-3}


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2302_04741_gb300 import build
    build.build()
    oracle.set_threads(os.cpu_count() or 1)


def run_both(w, steps, **simkw):
    sim = lbm.Sim(w, **simkw).init()
    ref = oracle_sim(w)
    sim.step(steps)
    ref.step(steps)
    return sim, ref


SINE_Y = {"kind": W.G_SINE, "g0": (3e-5, 0.0, 0.0), "wave_axis": 1}


def field_g(lat, shape, seed=5, amp=3e-5):
    D = W.dims(lat)
    N = shape[0] * shape[1] * shape[2]
    return {"kind": W.G_FIELD, "field": amp * (W.uniform(seed, 30, D * N).reshape(D, N) - 0.5)}


CASES = [
    # (id, lattice, shape, bc, force order, g)
    ("d2-periodic-o2", 0, (37, 23, 1), (0, 0, 0), 2, None),
    ("d2-periodic-o1-sine", 0, (150, 9, 1), (0, 0, 0), 1, SINE_Y),
    ("d2-periodic-o0", 0, (33, 7, 1), (0, 0, 0), 0, None),
    ("d2-bounce-o2", 0, (41, 16, 1), (0, 1, 0), 2, None),
    ("d2-thermal-o2-field", 0, (130, 12, 1), (0, 2, 0), 2, "field"),
    ("d3-periodic-o2", 1, (9, 7, 5), (0, 0, 0), 2, None),
    ("d3-thermal-o2", 1, (11, 6, 10), (0, 0, 2), 2, None),
    ("d3-bounce-o1-field", 1, (7, 9, 8), (0, 0, 1), 1, "field"),
]


def make_case(case, precision):
    _, lat, shape, bc, fo, g = case
    if g == "field":
        g = field_g(lat, shape)
    wall_T = dict(T_lo=(1.0, 1.08, 1.08), T_hi=(1.0, 0.93, 0.93))
    return workload(lat, shape, tau=0.7, g=g, seed=11, precision=precision, force_order=fo, bc=bc,
                    **wall_T)


@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
def test_fp64_step_parity(case):
    w = make_case(case, 0)
    sim, ref = run_both(w, 12)
    check_fields(sim, ref, w, TOL[0])
    perm = perm_to_oracle(w["lattice"])
    fg = sim.populations()
    fo = ref.pulled()[perm]
    assert np.max(np.abs(fg - fo)) < 1e-14


@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
def test_fp64_float_pair_step_parity(case):
    """FP64 storage with the float-float step (lbm_options.fp64_arith): the
    FP64 field tolerance against the oracle, and per population within
    1e-12 of the oracle (the float-float arithmetic carries ~48 bits)."""
    w = make_case(case, 0)
    w["fp64_arith"] = lbm.LBM_ARITH_FLOAT_PAIR
    sim, ref = run_both(w, 12)
    check_fields(sim, ref, w, TOL[0])
    perm = perm_to_oracle(w["lattice"])
    assert np.max(np.abs(sim.populations() - ref.pulled()[perm])) < 1e-12


@pytest.mark.parametrize("precision", [1, 2])
@pytest.mark.parametrize("case", CASES[:1] + CASES[3:6] + CASES[6:7], ids=lambda c: str(c[0]) if isinstance(c, tuple) else str(c))
def test_reduced_precision_parity(case, precision):
    w = make_case(case, precision)
    sim, ref = run_both(w, 12)
    check_fields(sim, ref, w, TOL[precision])


@pytest.mark.parametrize("precision", [1, 2])
@pytest.mark.parametrize("case", CASES[:1] + CASES[3:6] + CASES[6:7], ids=lambda c: str(c[0]) if isinstance(c, tuple) else str(c))
def test_reduced_precision_white_noise(case, precision):
    """Grid-scale white noise (u ~ 0.02, T ~ 0.03 per site): after 12 steps |u|
    has decayed to ~1e-3 while the non-equilibrium parts stay ~|f - w|, so the
    relative error of u reaches the float floor eps_32 |f - w| / |u|; the bound
    here is 10x the resolved-flow tolerance for FP32; FP16 keeps its 1e-3."""
    _, lat, shape, bc, fo, g = case
    if g == "field":
        g = field_g(lat, shape)
    w = workload(lat, shape, tau=0.7, g=g, seed=11, precision=precision, force_order=fo, bc=bc,
                 T_lo=(1.0, 1.08, 1.08), T_hi=(1.0, 0.93, 0.93), white_noise=True)
    sim, ref = run_both(w, 12)
    check_fields(sim, ref, w, 1e-5 if precision == 1 else TOL[2])


MU_CASES = [CASES[0], CASES[4], CASES[5], CASES[6]]


@pytest.mark.parametrize("precision", [0, 1, 2])
@pytest.mark.parametrize("case", MU_CASES, ids=[c[0] for c in MU_CASES])
def test_constant_mu_parity(case, precision):
    """Constant dynamic viscosity: tau-hat = mu / (rho theta) + 1/2 per site
    from the mid-point state, in the update and the heat-flux diagnostic."""
    w = make_case(case, precision)
    w["mu"] = 0.25
    w["tau"] = 5.0  # unused with mu > 0: a wrong path would show
    sim, ref = run_both(w, 12)
    check_fields(sim, ref, w, TOL[precision])
    if precision == 0:
        fg = sim.populations()
        fo = ref.pulled()[perm_to_oracle(w["lattice"])]
        assert np.max(np.abs(fg - fo)) < 1e-14


def test_constant_mu_rejects_negative():
    w = workload(0, (16, 8, 1))
    w["mu"] = -1.0
    with pytest.raises(lbm.LbmError) as ei:
        lbm.Sim(w)
    assert ei.value.status == lbm.LBM_EINVAL


SIGMA_CASES = [c for c in CASES if c[4] == 2]


@pytest.mark.parametrize("precision", [0, 1, 2])
@pytest.mark.parametrize("case", SIGMA_CASES, ids=[c[0] for c in SIGMA_CASES])
def test_sigma_bar_parity(case, precision):
    """Force order 2 with the sigma-bar terms (a^(2) = a^(2)_0 - sigma-bar in
    the n = 3 force term).  |g| ~ 5e-4 with the sheared smooth state makes the
    terms change the populations by far more than the FP64 tolerance."""
    w = make_case(case, precision)
    D = W.dims(w["lattice"])
    w["g"] = {"kind": W.G_UNIFORM, "g0": (4e-4, -3e-4, 2e-4)[:D] + (0.0,) * (3 - D)}
    w["include_sigma"] = True
    sim, ref = run_both(w, 12)
    check_fields(sim, ref, w, TOL[precision])
    if precision == 0:
        perm = perm_to_oracle(w["lattice"])
        fo = ref.pulled()[perm]
        assert np.max(np.abs(sim.populations() - fo)) < 1e-14
        plain = oracle_sim(dict(w, include_sigma=False))
        plain.step(12)
        assert np.max(np.abs(plain.pulled()[perm] - fo)) > 1e-11


@pytest.mark.parametrize("case", MU_CASES, ids=[c[0] for c in MU_CASES])
def test_float_pair_sigma_and_constant_mu(case):
    """The float-float step with the sigma-bar terms and with constant mu."""
    for extra in (dict(mu=0.25, tau=5.0), dict(include_sigma=True)):
        w = make_case(case, 0)
        if extra.get("include_sigma"):
            if case[4] != 2:
                continue
            D = W.dims(w["lattice"])
            w["g"] = {"kind": W.G_UNIFORM, "g0": (4e-4, -3e-4, 2e-4)[:D] + (0.0,) * (3 - D)}
        w.update(extra)
        w["fp64_arith"] = lbm.LBM_ARITH_FLOAT_PAIR
        sim, ref = run_both(w, 12)
        check_fields(sim, ref, w, TOL[0])
        fo = ref.pulled()[perm_to_oracle(w["lattice"])]
        assert np.max(np.abs(sim.populations() - fo)) < 1e-12


def test_sigma_bar_with_constant_mu():
    w = make_case(CASES[4], 0)
    w["g"] = {"kind": W.G_UNIFORM, "g0": (3e-4, -5e-4, 0.0)}
    w["include_sigma"] = True
    w["mu"] = 0.2
    sim, ref = run_both(w, 12)
    check_fields(sim, ref, w, TOL[0])
    fo = ref.pulled()[perm_to_oracle(w["lattice"])]
    assert np.max(np.abs(sim.populations() - fo)) < 1e-14


def test_sigma_bar_needs_plain_kernel():
    w = workload(0, (64, 12, 1), precision=1)
    w["include_sigma"] = True
    for kern in (lbm.LBM_KERNEL_TMA, lbm.LBM_KERNEL_PREFETCH):
        with pytest.raises(lbm.LbmError) as ei:
            lbm.Sim(w, kernel=kern)
        assert ei.value.status == lbm.LBM_EINVAL
    torch = pytest.importorskip("torch")
    stream = torch.cuda.Stream()
    sim = lbm.Sim(w, stream=stream.cuda_stream).init()
    b = lbm.lbm_batch_create(0, 1, 2, stream.cuda_stream, 2)
    try:
        with pytest.raises(lbm.LbmError) as ei:
            lbm.lbm_batch_add(b, sim.ctx)
        assert ei.value.status == lbm.LBM_EINVAL and "force order" in str(ei.value)
    finally:
        lbm.lbm_batch_destroy(b)
        sim.close()


@pytest.mark.parametrize("lat,shape,bc", [(0, (21, 13, 1), (0, 0, 0)), (0, (19, 10, 1), (0, 1, 0)),
                                          (1, (6, 5, 7), (0, 0, 1))])
@pytest.mark.parametrize("precision", [0, 1, 2])
def test_init_roundtrip(lat, shape, bc, precision):
    """lbm_moments right after lbm_init returns the given fields."""
    w = workload(lat, shape, seed=4, precision=precision, bc=bc)
    sim = lbm.Sim(w).init()
    rho, u, T, q = sim.moments()
    tol = TOL[precision] * (10 if precision else 1)
    assert rel_l2(rho, w["rho"]) < tol
    assert rel_l2(u, w["u"]) < tol
    assert rel_l2(T, w["T"]) < tol


@pytest.mark.parametrize("fo", [2, 1])
@pytest.mark.parametrize("arith", [0, 1])
def test_kolmogorov_64_fp64_2000_steps(fo, arith):
    """The 64x64 FP64 Kolmogorov configuration (third-moment term on/off), full
    run, with IEEE double and with float-float step arithmetic."""
    w = W.kolmogorov(force_order=fo)
    w["fp64_arith"] = arith
    sim, ref = run_both(w, 2000)
    err = check_fields(sim, ref, w, TOL[0])
    print("kolmogorov fo", fo, err)


@pytest.mark.parametrize("precision", [0, 1])
def test_conserved_sums(precision):
    w = make_case(CASES[4], precision)
    sim, ref = run_both(w, 7)
    st, m, p, e = sim.conserved()
    rho, u, T, _ = ref.moments()
    D = 2
    mr = np.sum(rho)
    pr = (rho * u).sum(axis=1)
    er = np.sum(0.5 * rho * (np.sum(u * u, axis=0) + D * T))
    tol = 1e-13 if precision == 0 else 1e-7
    assert abs(m - mr) < tol * mr
    assert np.all(np.abs(p - pr) < tol * mr)
    assert abs(e - er) < tol * er


def test_conserved_flags_unstable():
    w = workload(0, (16, 8, 1), seed=3)
    sim = lbm.Sim(w).init()
    f = sim.get_state()
    f[:, 5] = -1.0  # negative density at one site (host-side corruption)
    sim.set_state(f)
    st, m, p, e = sim.conserved(raise_unstable=False)
    assert st == lbm.LBM_EUNSTABLE


@pytest.mark.parametrize("precision", [0, 1])
def test_sampled_one_step_full_size(precision):
    """Rayleigh-Benard 1024x512 (walls, FP32-shifted / FP64) in the launch
    configuration the benchmark uses (10-step graphs, programmatic dependent
    launches, L2 evict-first loads at this size): one step from the GPU's own
    state, checked at sampled sites against the oracle evaluating those
    sites, and the mass over a graph replay."""
    w = W.rayleigh_benard(precision=precision)
    sim = lbm.Sim(w, graph_steps=10).init()   # 10-step graphs, as timed
    sim.step(40)
    m0 = sim.conserved()[1]
    sim.step(10)                               # one replay of the graph
    state = sim.get_state()
    sim.step(1)
    after = sim.get_state()
    # the diffuse walls conserve mass per column: over the replayed steps the
    # total moves only by rounding
    assert abs(sim.conserved()[1] / m0 - 1) < (1e-13 if precision == 0 else 1e-6)
    ref = oracle_sim(w)
    perm = perm_to_oracle(0)
    inv = np.argsort(perm)
    N = w["shape"][0] * w["shape"][1]
    rng = np.random.default_rng(0)
    rows = np.concatenate([np.arange(0, 3), np.arange(509, 512), rng.integers(3, 509, 6)])
    cols = rng.integers(0, 1024, 64)
    sites = (rows[:, None] * 1024 + cols[None, :]).ravel()
    sites = np.unique(np.concatenate([sites, rng.integers(0, N, 1000)]))
    st_oracle = np.empty_like(state)
    st_oracle[perm] = state
    out = ref.step_sites(st_oracle, sites)[:, perm]          # library order
    got = after[:, sites].T
    wts = lbm.lbm_lattice_info(0)[4]
    err = np.max(np.abs(got - out) / wts)
    # FP64: the oracle's rank-4 tensor contractions cancel terms ~ |xi|^4 ~ 200
    # down to results ~ 0.3, leaving ~1e-14 relative round-off of its own
    assert err < (1e-13 if precision == 0 else 3e-7), err


def test_graph_replay_is_bitwise_plain():
    w = make_case(CASES[3], 1)
    a = lbm.Sim(w).init()
    b = lbm.Sim(w, graph_steps=4).init()
    a.step(11)
    b.step(11)
    np.testing.assert_array_equal(a.get_state(), b.get_state())


@pytest.mark.parametrize("precision", [0, 1, 2])
def test_checkpoint_continuation_is_bitwise(precision):
    w = make_case(CASES[4], precision)
    a = lbm.Sim(w).init()
    a.step(5)
    with tempfile.TemporaryDirectory() as d:
        path = os.path.join(d, "ck.bin")
        lbm.lbm_save(a.ctx, path)
        b = lbm.Sim(w)
        lbm.lbm_load(b.ctx, path)
        assert lbm.lbm_step_count(b.ctx) == 5
    a.step(6)
    b.step(6)
    np.testing.assert_array_equal(a.get_state(), b.get_state())


@pytest.mark.parametrize("block_x", [32, 64, 256])
def test_block_shape_does_not_change_result(block_x):
    w = make_case(CASES[1], 1)
    a = lbm.Sim(w).init()
    b = lbm.Sim(w, block_x=block_x).init()
    a.step(5)
    b.step(5)
    np.testing.assert_array_equal(a.get_state(), b.get_state())


def test_translation_invariance_bitwise():
    lat, shape = 0, (40, 24, 1)
    w = workload(lat, shape, seed=8, precision=1)
    a = lbm.Sim(w).init()
    a.step(6)

    def roll(v):
        v = np.asarray(v)
        return np.ascontiguousarray(
            np.roll(v.reshape(v.shape[:-1] + (24, 40)), (5, 7), axis=(-2, -1)).reshape(v.shape))

    w2 = dict(w, rho=roll(w["rho"]), u=roll(w["u"]), T=roll(w["T"]))
    b = lbm.Sim(w2).init()
    b.step(6)
    np.testing.assert_array_equal(roll(a.get_state()), b.get_state())


@pytest.mark.parametrize("graph_steps", [0, 10])
@pytest.mark.parametrize("precision", [0, 1])
def test_overlapped_launches_are_bitwise_plain(precision, graph_steps):
    """Programmatic dependent launch of successive steps changes nothing."""
    w = workload(0, (200, 40, 1), seed=8, precision=precision, bc=(0, 2, 0),
                 T_lo=(1.0, 1.05, 1.0), T_hi=(1.0, 0.95, 1.0))
    a = lbm.Sim(w, overlap_steps=1, graph_steps=graph_steps).init()
    b = lbm.Sim(w, overlap_steps=0, graph_steps=graph_steps).init()
    a.step(30)
    b.step(30)
    np.testing.assert_array_equal(a.populations(), b.populations())


@pytest.mark.parametrize("precision", [0, 1, 2])
def test_pinned_host_buffers_are_read_and_written_in_place(precision):
    """Page-locked host arrays go to the kernels through their mapped device
    address (no staging copy); results equal the pageable-array path and a
    re-init keeps the captured graphs valid."""
    torch = pytest.importorskip("torch")
    w = workload(0, (96, 24, 1), seed=12, precision=precision, bc=(0, 2, 0),
                 T_lo=(1.0, 1.04, 1.0), T_hi=(1.0, 0.97, 1.0))
    ref = lbm.Sim(w, graph_steps=4).init()
    ref.step(8)
    want = ref.moments()
    sim = lbm.Sim(w, graph_steps=4)
    pin = lambda a: torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).pin_memory()
    h_in = [pin(w["rho"]), pin(w["u"]), pin(w["T"])]
    N = sim.N
    h_out = [torch.zeros(n, dtype=torch.float64).pin_memory() for n in (N, 2 * N, N, 2 * N)]
    for _ in range(2):  # the second pass re-initialises with the graphs in place
        lbm.lbm_init(sim.ctx, *h_in)
        sim.step(8)
        lbm.lbm_moments(sim.ctx, *h_out)
        for got, exp in zip(h_out, want):
            np.testing.assert_array_equal(got.numpy(), np.asarray(exp).ravel())


def test_errors_are_reported():
    w = workload(0, (16, 8, 1))
    s = lbm.Sim(w)
    with pytest.raises(lbm.LbmError) as ei:
        s.step(1)
    assert ei.value.status == lbm.LBM_ESTATE
    with pytest.raises(lbm.LbmError) as ei:
        lbm.lbm_step(s.ctx, -1)
    assert ei.value.status == lbm.LBM_EINVAL
    with pytest.raises(lbm.LbmError) as ei:
        lbm.lbm_load(s.ctx, "/nonexistent/ck.bin")
    assert ei.value.status == lbm.LBM_EIO


def test_device_pointers_and_stream():
    torch = pytest.importorskip("torch")
    w = workload(0, (64, 20, 1), seed=6, precision=1)
    stream = torch.cuda.Stream()
    sim = lbm.Sim(w, stream=stream.cuda_stream)
    dev = [torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in (w["rho"], w["u"], w["T"])]
    lbm.lbm_init(sim.ctx, *dev)
    lbm.lbm_step(sim.ctx, 3)
    out = [torch.zeros_like(dev[0]), torch.zeros_like(dev[1]), torch.zeros_like(dev[0]),
           torch.zeros_like(dev[1])]
    lbm.lbm_moments(sim.ctx, *out)
    host = lbm.Sim(w, stream=stream.cuda_stream).init()
    host.step(3)
    hr = host.moments()
    for a, b in zip(out, hr):
        np.testing.assert_array_equal(a.cpu().numpy(), b)


# ------------------------------------------- TMA-staged step kernel vs plain
TMA_CASES = [
    ("d2-periodic-tiles", 0, (256, 20, 1), (0, 0, 0)),
    ("d2-periodic-ragged", 0, (200, 13, 1), (0, 0, 0)),
    ("d2-narrow", 0, (64, 9, 1), (0, 0, 0)),
    ("d2-bounce", 0, (136, 12, 1), (0, 1, 0)),
    ("d2-thermal", 0, (1024, 16, 1), (0, 2, 0)),
    ("d3-thermal", 1, (40, 8, 10), (0, 0, 2)),
    ("d3-periodic", 1, (16, 12, 9), (0, 0, 0)),
]


@pytest.mark.parametrize("fo", [1, 2])
@pytest.mark.parametrize("precision", [1, 2])
@pytest.mark.parametrize("case", TMA_CASES, ids=[c[0] for c in TMA_CASES])
def test_tma_kernel_bitwise_equals_plain(case, precision, fo):
    _, lat, shape, bc = case
    w = workload(lat, shape, tau=0.7, seed=13, precision=precision, force_order=fo, bc=bc,
                 T_lo=(1.0, 1.08, 1.08), T_hi=(1.0, 0.93, 0.93))
    a = lbm.Sim(w, kernel=lbm.LBM_KERNEL_PLAIN).init()
    b = lbm.Sim(w, kernel=lbm.LBM_KERNEL_TMA).init()
    assert lbm.lbm_step_kernel(a.ctx) == lbm.LBM_KERNEL_PLAIN
    assert lbm.lbm_step_kernel(b.ctx) == lbm.LBM_KERNEL_TMA
    a.step(7)
    b.step(7)
    np.testing.assert_array_equal(a.get_state(), b.get_state())
    assert b.conserved()[0] == lbm.LBM_OK  # no bounded wait ran out


@pytest.mark.parametrize("stages", [2, 4, 6])
def test_tma_stage_count_does_not_change_result(stages):
    w = workload(0, (384, 24, 1), tau=0.8, seed=14, precision=1, bc=(0, 2, 0),
                 T_lo=(1.0, 1.05, 1.0), T_hi=(1.0, 0.95, 1.0))
    a = lbm.Sim(w, kernel=lbm.LBM_KERNEL_PLAIN).init()
    b = lbm.Sim(w, kernel=lbm.LBM_KERNEL_TMA, tma_stages=stages).init()
    a.step(9)
    b.step(9)
    np.testing.assert_array_equal(a.get_state(), b.get_state())


def test_kernel_selection():
    # AUTO runs the plain kernel; the TMA kernel needs FP32/FP16 rows of 16-byte multiples
    assert lbm.lbm_step_kernel(lbm.Sim(workload(0, (64, 8, 1), precision=0)).ctx) == lbm.LBM_KERNEL_PLAIN
    assert lbm.lbm_step_kernel(lbm.Sim(workload(0, (68, 8, 1), precision=1)).ctx) == lbm.LBM_KERNEL_PLAIN
    tma = lbm.Sim(workload(0, (68, 8, 1), precision=1), kernel=lbm.LBM_KERNEL_TMA)
    assert lbm.lbm_step_kernel(tma.ctx) == lbm.LBM_KERNEL_TMA
    with pytest.raises(lbm.LbmError) as ei:
        lbm.Sim(workload(0, (64, 8, 1), precision=0), kernel=lbm.LBM_KERNEL_TMA)
    with pytest.raises(lbm.LbmError) as ei:
        lbm.Sim(workload(0, (66, 8, 1), precision=1), kernel=lbm.LBM_KERNEL_TMA)
    assert ei.value.status == lbm.LBM_EINVAL


@pytest.mark.parametrize("block_x", [64, 128])
@pytest.mark.parametrize("case", TMA_CASES, ids=[c[0] for c in TMA_CASES])
def test_prefetch_kernel_bitwise_equals_plain(case, block_x):
    _, lat, shape, bc = case
    w = workload(lat, shape, tau=0.7, seed=15, precision=1, force_order=2, bc=bc,
                 T_lo=(1.0, 1.08, 1.08), T_hi=(1.0, 0.93, 0.93))
    a = lbm.Sim(w, kernel=lbm.LBM_KERNEL_PLAIN).init()
    b = lbm.Sim(w, kernel=lbm.LBM_KERNEL_PREFETCH, block_x=block_x).init()
    assert lbm.lbm_step_kernel(b.ctx) == lbm.LBM_KERNEL_PREFETCH
    a.step(7)
    b.step(7)
    np.testing.assert_array_equal(a.get_state(), b.get_state())


WAVE_CASES = TMA_CASES + [("d2-periodic-y-short", 0, (96, 7, 1), (0, 0, 0))]


@pytest.mark.parametrize("steps,graph", [(7, 0), (12, 4)])
@pytest.mark.parametrize("precision", [1, 2])
@pytest.mark.parametrize("case", WAVE_CASES, ids=[c[0] for c in WAVE_CASES])
def test_wave_kernel_bitwise_equals_plain(case, precision, steps, graph):
    """Several steps per launch (wavefront order) give exactly the plain
    kernel's state, with walls or periodic wrap on the last axis, odd step
    counts and graph replay."""
    _, lat, shape, bc = case
    w = workload(lat, shape, seed=21, precision=precision, bc=bc, force_order=2,
                 T_lo=(1.0, 1.05, 1.05), T_hi=(1.0, 0.96, 0.96))
    a = lbm.Sim(w, kernel=lbm.LBM_KERNEL_WAVE, graph_steps=graph).init()
    assert lbm.lbm_step_kernel(a.ctx) == lbm.LBM_KERNEL_WAVE
    b = lbm.Sim(w, kernel=lbm.LBM_KERNEL_PLAIN).init()
    a.step(steps)
    b.step(steps)
    np.testing.assert_array_equal(a.populations(), b.populations())
    assert a.conserved()[0] == lbm.LBM_OK  # no bounded wait ran out
    a.step(3)
    b.step(3)
    np.testing.assert_array_equal(a.populations(), b.populations())


def test_wave_kernel_rejections():
    w = workload(0, (64, 12, 1), precision=0)
    with pytest.raises(lbm.LbmError):
        lbm.Sim(w, kernel=lbm.LBM_KERNEL_WAVE)
    w = workload(0, (64, 12, 1), precision=1)
    w["include_sigma"] = True
    with pytest.raises(lbm.LbmError):
        lbm.Sim(w, kernel=lbm.LBM_KERNEL_WAVE)


@pytest.mark.parametrize("lat,shape,fo", [(0, (96, 24, 1), 2), (0, (80, 20, 1), 1), (1, (24, 20, 16), 2)])
def test_float_storage_moments_match_fp64_sums(lat, shape, fo):
    """For float storage the diagnostic sums the deviations as compensated
    float pairs and combines them in float-float arithmetic (~48 bits); an
    all-fluid solid mask sends the same state through the FP64 summation and
    combination instead.  rho, u and T agree to 1e-13 relative; q, the small
    remainder of a cancelling combination, agrees to 2^-40 of the size of
    its terms, sum_i |f~_i - w_i| |xi_i - u|^3 (both far below the 6e-8 of the
    float storage itself)."""
    w = workload(lat, shape, seed=17, precision=1, force_order=fo)
    a = lbm.Sim(w).init()
    b = lbm.Sim(w)
    lbm.lbm_set_solid(b.ctx, np.zeros(a.N, np.uint8), np.ones(a.N))
    b.init()
    a.step(9)
    b.step(9)
    np.testing.assert_array_equal(a.populations(), b.populations())
    ma, mb = a.moments(), b.moments()
    for name, x, y in zip(("rho", "u", "T"), ma, mb):
        np.testing.assert_allclose(x, y, rtol=1e-13, atol=1e-16, err_msg=name)
    f = b.populations()
    D = a.D
    xi = a.c * a.e[:, :D].astype(float)
    cc = xi[:, :, None] - mb[1][None, :, :]
    scale = (np.abs(f - a.wts[:, None]) * np.sqrt((cc * cc).sum(axis=1)) ** 3).sum(axis=0)
    dq = np.abs(ma[3] - mb[3]).max(axis=0)
    assert np.all(dq <= 2.0 ** -40 * scale), float(np.max(dq / scale))


def _create(lat=0, nx=32, ny=16, nz=1, tau=0.8, **opt):
    o = lbm.options(**{k: v for k, v in opt.items() if k in (
        "precision", "force_order", "bc", "block_x", "graph_steps", "kernel", "tma_stages", "mu",
        "include_sigma", "overlap_steps")})
    return lbm.lbm_create(lat, nx, ny, nz, tau, None, o)


@pytest.mark.parametrize("kw,why", [
    (dict(nx=0), "empty grid"),
    (dict(nz=2), "D2Q37 with nz > 1"),
    (dict(lat=1, nx=2048, ny=2048, nz=1024), "N >= 2^31"),
    (dict(tau=0.5), "tau-hat <= 1/2"),
    (dict(tau=float("nan")), "tau-hat not finite"),
    (dict(precision=3), "unknown precision"),
    (dict(force_order=3), "force order > 2"),
    (dict(bc=(0, 1, 0), ny=5), "walled axis below 6 sites"),
    (dict(bc=(1, 0, 0)), "walls off the last axis"),
    (dict(nx=2), "periodic axis below 3 sites"),
    (dict(block_x=48), "block width not a multiple of 32"),
    (dict(graph_steps=3), "odd graph length"),
    (dict(kernel=9), "unknown kernel"),
    (dict(mu=-1.0), "negative viscosity"),
    (dict(overlap_steps=2), "bad overlap switch"),
    (dict(tma_stages=1), "TMA ring depth"),
])
def test_create_rejects_invalid_arguments(kw, why):
    """Every invalid argument is caught before any device memory is taken:
    LBM_EINVAL with a message, and no context."""
    with pytest.raises(lbm.LbmError) as ei:
        _create(**kw)
    assert ei.value.status == lbm.LBM_EINVAL, why
    assert str(ei.value), why


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("lat,shape", [(W.D2Q37, (128, 4, 1)), (W.D3Q39, (96, 4, 4))])
def test_adiabatic_sound_speed_on_gpu(lat, shape, precision):
    """The CUDA path carries sound at the adiabatic speed sqrt((D + 2) / D)
    (the oracle's pin of the same run): a 1e-4 density wave in a fluid at
    rest, the velocity's projection on sin(kx) timed between zero crossings."""
    D = W.dims(lat)
    nx, ny, nz = shape
    N = nx * ny * nz
    x = np.arange(N) % nx
    k = 2 * np.pi / nx
    w = dict(lattice=lat, shape=shape, tau=0.6, g={"kind": W.G_UNIFORM, "g0": (0.0, 0.0, 0.0)},
             precision=precision, force_order=2, bc=(0, 0, 0), T_lo=(1.0,) * 3, T_hi=(1.0,) * 3,
             rho=1.0 + 1e-4 * np.cos(k * x), u=np.zeros((D, N)), T=np.ones(N), name="sound")
    sim = lbm.Sim(w).init()
    s = np.sin(k * x)
    a = []
    for _ in range(260):
        a.append(sim.moments()[1][0] @ s / (s @ s))
        sim.step(1)
    a = np.array(a)
    z = [t + a[t] / (a[t] - a[t + 1]) for t in range(1, len(a) - 1) if a[t] * a[t + 1] < 0]
    cs = nx * sim.c / (z[2] - z[0])
    assert abs(cs / np.sqrt((D + 2) / D) - 1) < 1e-3, cs


@pytest.mark.parametrize("precision,tol", [(0, 1e-4), (1, 1e-3)])
def test_galilean_invariance_on_gpu(precision, tol):
    """A shear wave u_y = A sin(kx) on a stream U0 = 0.2 (D2Q37): the CUDA
    path carries it at U0 and damps it as at rest (the oracle's pin of the
    same run), in FP64 and in FP32-shifted storage."""
    lat, shape = W.D2Q37, (64, 4, 1)
    D, N = 2, 256
    x = np.arange(N) % 64
    A, T = 1e-4, 150
    amp = {}
    for U0 in (0.0, 0.2):
        u = np.zeros((D, N))
        u[0] = U0
        u[1] = A * np.sin(2 * np.pi * x / 64)
        w = dict(lattice=lat, shape=shape, tau=0.8, g={"kind": W.G_UNIFORM, "g0": (0.0, 0.0, 0.0)},
                 precision=precision, force_order=2, bc=(0, 0, 0), T_lo=(1.0,) * 3,
                 T_hi=(1.0,) * 3, rho=np.ones(N), u=u, T=np.ones(N), name="shear")
        sim = lbm.Sim(w).init()
        k = 2 * np.pi / (64 * sim.c)
        sim.step(T)
        z = sim.moments()[1][1] @ np.exp(-1j * 2 * np.pi * x / 64) / (N / 2) / (-1j * A)
        amp[U0] = abs(z)
        assert abs(np.angle(z * np.exp(1j * k * U0 * T))) < tol, (U0, np.angle(z))
        sim.close()
    assert abs(amp[0.2] / amp[0.0] - 1) < tol, amp
