"""Batches: one persistent launch steps many grids; each result must be
bit-identical to the same grid stepped alone (same device code per site)."""
import numpy as np
import pytest

import paper_2302_04741_gb300 as lbm
from paper_2302_04741_gb300 import workloads as W
from helpers import workload

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    t = pytest.importorskip("torch")
    from paper_2302_04741_gb300 import build
    build.build()
    return t


def mixed_grids(precision, lat=0):
    if lat == 0:
        specs = [((128, 64, 1), (0, 0, 0)), ((200, 37, 1), (0, 0, 0)), ((64, 96, 1), (0, 2, 0)),
                 ((384, 12, 1), (0, 1, 0)), ((36, 40, 1), (0, 0, 0))]
    else:
        specs = [((16, 16, 16), (0, 0, 0)), ((24, 12, 10), (0, 0, 2)), ((32, 8, 9), (0, 0, 0))]
    ws = []
    for k, (shape, bc) in enumerate(specs):
        ws.append(workload(lat, shape, tau=0.55 + 0.1 * k, seed=40 + k, precision=precision, bc=bc,
                           T_lo=(1.0, 1.06, 1.06), T_hi=(1.0, 0.95, 0.95),
                           g={"kind": W.G_UNIFORM, "g0": (1e-5 * (k + 1), -2e-5, 1e-5)}))
    return ws


def states(sims):
    return [s.get_state() for s in sims]


@pytest.mark.parametrize("lat,precision", [(0, 1), (0, 2), (1, 1)])
@pytest.mark.parametrize("cfg", [(128, 1, 0), (64, 2, 0), (256, 1, 4), (128, 2, 6)])
def test_batch_bitwise_equals_single(torch, lat, precision, cfg):
    stream = torch.cuda.Stream()
    ws = mixed_grids(precision, lat)
    members = [lbm.Sim(w, stream=stream.cuda_stream).init() for w in ws]
    alone = [lbm.Sim(w).init() for w in ws]
    b = lbm.lbm_batch_create(lat, precision, 2, stream.cuda_stream, 16)
    try:
        for m in members:
            lbm.lbm_batch_add(b, m.ctx)
        lbm.lbm_batch_set_config(b, *cfg)
        lbm.lbm_batch_step(b, 9)   # odd: parities flip, table re-uploaded
        lbm.lbm_batch_step(b, 14)  # graph replays (when configured) + remainder
        for a in alone:
            a.step(23)
        for m, a in zip(members, alone):
            assert lbm.lbm_step_count(m.ctx) == 23
            np.testing.assert_array_equal(m.get_state(), a.get_state())
    finally:
        lbm.lbm_batch_destroy(b)


@pytest.mark.parametrize("lat", [0, 1])
@pytest.mark.parametrize("bx,fo,graph", [(64, 2, 0), (128, 0, 4), (256, 2, 0), (128, 1, 0)])
def test_staged_batch_bitwise_equals_single(torch, lat, bx, fo, graph):
    """The halo-staged batch kernel (cp.async prefetch of the next tile)
    against each grid stepped alone by the plain step kernel."""
    stream = torch.cuda.Stream()
    ws = mixed_grids(1, lat)
    if fo != 2:
        ws = [dict(w, force_order=fo) for w in ws]
    members = [lbm.Sim(w, stream=stream.cuda_stream).init() for w in ws]
    alone = [lbm.Sim(w).init() for w in ws]
    b = lbm.lbm_batch_create(lat, 1, fo, stream.cuda_stream, 16)
    try:
        for m in members:
            lbm.lbm_batch_add(b, m.ctx)
        lbm.lbm_batch_set_config(b, bx, 1, graph)
        lbm.lbm_batch_set_staging(b, 1)
        assert lbm.lbm_batch_get_staging(b) == 1
        lbm.lbm_batch_step(b, 7)
        lbm.lbm_batch_step(b, 10)
        for a in alone:
            a.step(17)
        for m, a in zip(members, alone):
            np.testing.assert_array_equal(m.get_state(), a.get_state())
    finally:
        lbm.lbm_batch_destroy(b)


def test_staging_rules(torch):
    stream = torch.cuda.Stream()
    b16 = lbm.lbm_batch_create(0, 2, 2, stream.cuda_stream, 2)
    b32 = lbm.lbm_batch_create(0, 1, 2, stream.cuda_stream, 2)
    try:
        with pytest.raises(lbm.LbmError) as ei:   # FP16-scaled: 2-byte populations
            lbm.lbm_batch_set_staging(b16, 1)
        assert ei.value.status == lbm.LBM_EINVAL
        lbm.lbm_batch_set_config(b32, 128, 2, 0)
        with pytest.raises(lbm.LbmError):         # two sites per thread
            lbm.lbm_batch_set_staging(b32, 1)
        lbm.lbm_batch_set_config(b32, 128, 1, 0)
        lbm.lbm_batch_set_staging(b32, 1)
        with pytest.raises(lbm.LbmError):
            lbm.lbm_batch_set_config(b32, 128, 2, 0)
        assert lbm.lbm_batch_get_config(b32)[:2] == (128, 1)
        with pytest.raises(lbm.LbmError):
            lbm.lbm_batch_set_staging(b32, 2)
        lbm.lbm_batch_set_staging(b32, 0)
        assert lbm.lbm_batch_get_staging(b32) == 0
    finally:
        lbm.lbm_batch_destroy(b16)
        lbm.lbm_batch_destroy(b32)


def test_batch_membership_rules(torch):
    stream = torch.cuda.Stream()
    ws = mixed_grids(1)
    b = lbm.lbm_batch_create(0, 1, 2, stream.cuda_stream, 2)
    try:
        m = [lbm.Sim(w, stream=stream.cuda_stream).init() for w in ws[:3]]
        lbm.lbm_batch_add(b, m[0].ctx)
        with pytest.raises(lbm.LbmError) as ei:   # already a member
            lbm.lbm_batch_add(b, m[0].ctx)
        assert ei.value.status == lbm.LBM_ESTATE
        with pytest.raises(lbm.LbmError) as ei:   # members are stepped by their batch
            m[0].step(1)
        assert ei.value.status == lbm.LBM_ESTATE
        other = lbm.Sim(ws[1]).init()              # another stream
        with pytest.raises(lbm.LbmError) as ei:
            lbm.lbm_batch_add(b, other.ctx)
        assert ei.value.status == lbm.LBM_EINVAL
        f64 = lbm.Sim(dict(ws[1], precision=0), stream=stream.cuda_stream).init()
        with pytest.raises(lbm.LbmError):
            lbm.lbm_batch_add(b, f64.ctx)
        lbm.lbm_batch_add(b, m[1].ctx)
        with pytest.raises(lbm.LbmError) as ei:   # capacity 2
            lbm.lbm_batch_add(b, m[2].ctx)
        assert ei.value.status == lbm.LBM_ENOMEM
        lbm.lbm_batch_remove(b, m[0].ctx)
        m[0].step(1)                               # free again
        m[1].close()                               # destroying a member detaches it
        assert lbm.lbm_batch_size(b) == 0
        with pytest.raises(lbm.LbmError):
            lbm.lbm_batch_create(0, 0, 2, None, 4)  # FP64 batches are not offered
    finally:
        lbm.lbm_batch_destroy(b)


def test_batch_tune_then_continue(torch):
    stream = torch.cuda.Stream()
    ws = mixed_grids(1)
    members = [lbm.Sim(w, stream=stream.cuda_stream).init() for w in ws]
    alone = [lbm.Sim(w).init() for w in ws]
    b = lbm.lbm_batch_create(0, 1, 2, stream.cuda_stream, 8)
    try:
        for m in members:
            lbm.lbm_batch_add(b, m.ctx)
        bx, spt = lbm.lbm_batch_tune(b, 4)
        assert bx in (64, 128, 256) and spt in (1, 2)
        assert lbm.lbm_batch_get_config(b)[:2] == (bx, spt)
        n_tuned = lbm.lbm_step_count(members[0].ctx)
        assert n_tuned == 9 * (4 + 2)  # 6 plain candidates + 3 halo-staged ones
        assert lbm.lbm_batch_get_staging(b) in (0, 1)
        lbm.lbm_batch_step(b, 5)
        for a in alone:
            a.step(n_tuned + 5)
        for m, a in zip(members, alone):
            np.testing.assert_array_equal(m.get_state(), a.get_state())
        # a second tune of the same mix hits the cache: no steps taken
        lbm.lbm_batch_tune(b, 4)
        assert lbm.lbm_step_count(members[0].ctx) == n_tuned + 5
    finally:
        lbm.lbm_batch_destroy(b)


def test_reinit_member_inside_batch(torch):
    stream = torch.cuda.Stream()
    ws = mixed_grids(1)[:2]
    members = [lbm.Sim(w, stream=stream.cuda_stream).init() for w in ws]
    b = lbm.lbm_batch_create(0, 1, 2, stream.cuda_stream, 4)
    try:
        for m in members:
            lbm.lbm_batch_add(b, m.ctx)
        lbm.lbm_batch_step(b, 3)
        members[0].init()          # back to t = 0, buffer parity reset
        lbm.lbm_batch_step(b, 4)
        ref = lbm.Sim(ws[0]).init()
        ref.step(4)
        np.testing.assert_array_equal(members[0].get_state(), ref.get_state())
    finally:
        lbm.lbm_batch_destroy(b)


def test_ragged_subset_matches_oracle(torch):
    """Four grids of the ragged-batch configuration (periodic Kolmogorov, own
    tau and force amplitude each; sides from its set, one of them 256 wide so
    that a row spans several tiles of every launch shape) stepped together in
    one batch agree with the FP64 oracle run grid by grid: rho, u, T and q
    within the FP32 tolerance (q with the floor and the codec bound of the
    parity tests, helpers.check_fields)."""
    from helpers import check_fields, oracle_sim
    ws = W.ragged_batch(count=3, seed=3, sides=(128, 192))
    ws.append(W.kolmogorov(nx=256, ny=128, tau=0.65, g0=4e-5, seed=77, precision=W.FP32_SHIFTED))
    ws[-1]["name"] = "ragged_extra_256x128"
    for w in ws:  # a resolved perturbation so that u is not identically zero
        N = w["shape"][0] * w["shape"][1]
        k = np.arange(N)
        w["u"] = 1e-2 * np.stack([np.sin(2 * np.pi * k / N), np.cos(4 * np.pi * k / N)])
    stream = torch.cuda.Stream()
    members = [lbm.Sim(w, stream=stream.cuda_stream).init() for w in ws]
    b = lbm.lbm_batch_create(0, W.FP32_SHIFTED, 2, stream.cuda_stream, 8)
    try:
        for m in members:
            lbm.lbm_batch_add(b, m.ctx)
        lbm.lbm_batch_step(b, 20)
        for m, w in zip(members, ws):
            lbm.lbm_batch_remove(b, m.ctx)
            ref = oracle_sim(w)
            ref.step(20)
            check_fields(m, ref, w, 1e-6)
    finally:
        lbm.lbm_batch_destroy(b)
