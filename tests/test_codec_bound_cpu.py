"""Pin of the q bound the float codecs' comparisons use (helpers.q_codec_bound)
on the CPU oracle: the stored deviations of an oracle state are rounded as
each codec stores them (FP32: d to float; FP16: s d / w_i to half with the
power-of-two scale the library picks, max |d/w| s in [2^12, 2^13)), and the
oracle's q of the rounded state must differ from its q of the exact state by
no more than the bound -- and by not much less, so that the bound is not
vacuous (a dropped |xi - u|^3 weight or a lost factor makes it fail one side).
"""
import numpy as np
import pytest

import oracle
import helpers as H
from paper_2302_04741_gb300 import workloads as W


def rounded_state(f, wt, precision):
    d = f - wt[:, None]
    if precision == W.FP32_SHIFTED:
        return wt[:, None] + d.astype(np.float32).astype(np.float64)
    r = d / wt[:, None]
    k = 12 - int(np.floor(np.log2(np.abs(r).max())))
    s = 2.0 ** k
    h = (np.float32(s) * r.astype(np.float32)).astype(np.float16)
    return wt[:, None] + h.astype(np.float64) / s * wt[:, None]


# observed / bound: FP32's bound is the first-order worst case (all roundings
# aligned), FP16's twice the rms of independent roundings
RATIO = {W.FP32_SHIFTED: (0.01, 1.0), W.FP16_SCALED: (0.1, 1.0)}


@pytest.mark.parametrize("lat,shape", [(W.D2Q37, (24, 16, 1)), (W.D3Q39, (10, 8, 6))])
@pytest.mark.parametrize("precision", [W.FP32_SHIFTED, W.FP16_SCALED])
def test_codec_rounding_moves_q_within_the_bound(lat, shape, precision):
    w = H.workload(lat, shape, tau=0.7, seed=3, precision=precision)
    ref = H.oracle_sim(w)
    ref.step(5)
    wt = oracle.lattice_info(lat)[4]
    alt = H.oracle_sim(w)
    alt.set_state(rounded_state(ref.get_state(), wt, precision))
    dq = float(np.linalg.norm((alt.moments()[3] - ref.moments()[3]).ravel()))
    bound = H.q_codec_bound(ref, w)
    lo, hi = RATIO[precision]
    assert lo * bound <= dq <= hi * bound, (dq, bound)


def test_fp64_has_no_codec_term():
    w = H.workload(W.D2Q37, (12, 10, 1), precision=W.FP64)
    ref = H.oracle_sim(w)
    assert H.q_codec_bound(ref, w) == 0.0
