"""CPU-only checks of the C ABI: the library builds and loads, exports every
function include/lbm.h declares, validates arguments before touching a GPU,
and its compile-time velocity sets agree with the oracle's (two independent
solvers of the same moment conditions)."""
import ctypes
import itertools
import os
import re

import numpy as np
import pytest

import oracle
import paper_2302_04741_gb300 as lbm
from paper_2302_04741_gb300 import build as lbm_build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def libpath():
    return lbm_build.build()


def declared_functions():
    with open(os.path.join(ROOT, "include", "lbm.h")) as fh:
        text = fh.read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(lbm_[a-z0-9_]+)\s*\(", text)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("lbm_create", "lbm_init", "lbm_step", "lbm_moments", "lbm_destroy",
                     "lbm_conserved", "lbm_last_error"):
        assert required in names


def test_library_exports_every_declared_symbol(libpath):
    L = ctypes.CDLL(libpath)
    missing = [n for n in declared_functions() if not hasattr(L, n)]
    assert not missing, missing


def test_default_options_and_validation(libpath):
    o = lbm.lbm_default_options()
    assert o.precision == lbm.LBM_FP64 and o.force_order == 2 and o.include_sigma == 0
    assert list(o.bc) == [0, 0, 0] and o.graph_steps == 0
    bad = [
        dict(lat=7, nx=8, ny=8, nz=1, tau=0.8),
        dict(lat=0, nx=8, ny=8, nz=2, tau=0.8),     # D2Q37 with nz != 1
        dict(lat=0, nx=8, ny=8, nz=1, tau=0.5),     # tau-hat must exceed 1/2
        dict(lat=0, nx=2, ny=8, nz=1, tau=0.8),     # periodic axis shorter than 3
    ]
    for b in bad:
        with pytest.raises(lbm.LbmError) as ei:
            lbm.lbm_create(b["lat"], b["nx"], b["ny"], b["nz"], b["tau"])
        assert ei.value.status == lbm.LBM_EINVAL
    for kw in (dict(bc=(1, 0, 0)), dict(bc=(0, 2, 0), ny=5), dict(force_order=3),
               dict(block_x=48), dict(graph_steps=3)):
        ny = kw.pop("ny", 8)
        o = lbm.options(**kw)
        with pytest.raises(lbm.LbmError) as ei:
            lbm.lbm_create(0, 8, ny, 1, 0.8, None, o)
        assert ei.value.status == lbm.LBM_EINVAL
    o = lbm.lbm_default_options()
    o.include_sigma = 1
    with pytest.raises(lbm.LbmError):
        lbm.lbm_create(0, 8, 8, 1, 0.8, None, o)
    # float-float step arithmetic: FP64 storage, plain kernel, no storage probe
    for kw in (dict(precision=1, fp64_arith=1), dict(fp64_arith=2), dict(fp64_arith=1, storage_probe=1),
               dict(fp64_arith=1, kernel=lbm.LBM_KERNEL_TMA)):
        o = lbm.options(**kw)
        with pytest.raises(lbm.LbmError) as ei:
            lbm.lbm_create(0, 8, 8, 1, 0.8, None, o)
        assert ei.value.status == lbm.LBM_EINVAL
    # the storage probe: FP64 storage, a float codec's format, the plain kernel
    for kw in (dict(precision=1, storage_probe=1), dict(storage_probe=3), dict(storage_probe=-1),
               dict(storage_probe=2, kernel=lbm.LBM_KERNEL_TMA)):
        o = lbm.options(**kw)
        with pytest.raises(lbm.LbmError) as ei:
            lbm.lbm_create(0, 8, 8, 1, 0.8, None, o)
        assert ei.value.status == lbm.LBM_EINVAL


@pytest.mark.parametrize("lat", [0, 1])
def test_tables_agree_with_oracle(libpath, lat):
    D, Q, c, e, w = lbm.lbm_lattice_info(lat)
    Do, Qo, co, eo, wo, _ = oracle.lattice_info(lat)
    assert (D, Q) == (Do, Qo)
    assert c == co  # bit-identical: both rounded once from high precision
    idx = {tuple(v): k for k, v in enumerate(eo)}
    perm = np.array([idx[tuple(v)] for v in e])
    assert sorted(perm) == list(range(Q))
    np.testing.assert_array_equal(w, wo[perm])


@pytest.mark.parametrize("lat,deg", [(0, 9), (1, 7)])
def test_library_tables_are_gauss_hermite(libpath, lat, deg):
    D, Q, c, e, w = lbm.lbm_lattice_info(lat)
    xi = c * e[:, :D].astype(float)
    # direction order: rest first, then opposite pairs
    assert np.all(e[0] == 0)
    for k in range(1, Q, 2):
        assert np.all(e[k] == -e[k + 1])
    for alpha in itertools.product(range(deg + 1), repeat=D):
        if sum(alpha) > deg:
            continue
        s = np.sum(w * np.prod(xi ** np.array(alpha), axis=1))
        exact = 1
        for a in alpha:
            exact = 0 if a % 2 else exact * int(np.prod(np.arange(a - 1, 0, -2)) if a else 1)
        assert abs(s - exact) < 2e-14 * max(1, exact)


def test_batch_entry_points_reject_a_null_batch(libpath):
    """Argument checks that precede any CUDA call (no GPU needed)."""
    calls = [lambda: lbm.lbm_batch_set_staging(None, 1), lambda: lbm.lbm_batch_get_staging(None),
             lambda: lbm.lbm_batch_set_config(None, 128, 1, 0), lambda: lbm.lbm_batch_get_config(None),
             lambda: lbm.lbm_batch_step(None, 1), lambda: lbm.lbm_batch_tune(None, 4)]
    for call in calls:
        with pytest.raises(lbm.LbmError) as ei:
            call()
        assert ei.value.status == lbm.LBM_EINVAL
