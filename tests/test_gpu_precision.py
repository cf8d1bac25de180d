"""Precision of the ln g tables (the precision study of the L = 64 workload).

With ln f = 2^-k every ln g is a dyadic rational: double and the compensated
float pair hold it exactly, so both follow the oracle's trajectory bit for bit
(see test_gpu_parity.py).  A single float cannot: once ln f is below half an
ulp of ln g, every increment rounds away -- the reason the compensated pair
exists.  This test shows that failure directly."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1508_02748_gb300 as P
    from paper_1508_02748_gb300 import build
    build.build()
    return P


@pytest.mark.parametrize("sampler", [0, 1])
@pytest.mark.parametrize("prec", ["fp64", "f32x2", "f32"])
def test_lnf_increments_below_half_ulp(P, prec, sampler):
    code = {"fp64": P.FP64, "f32x2": P.F32X2, "f32": P.F32}[prec]
    lnf = 2.0 ** -20                       # half an ulp of 40.0 in float is 2^-19
    run = P.REWL(P.Config(L=8, n_win_E=3, n_win_M=3, walkers_per_window=4, precision=code,
                          lnf_init=lnf, seed=17, sampler=sampler))
    lng, H = run.tables()
    lng[:] = 40.0
    H[:] = 0
    run.set_tables(lng, H)
    run.sweep(10000)
    lng2, H2 = run.tables()
    gain = lng2 - 40.0
    assert H2.sum() == 36 * 10000
    if prec == "f32":
        assert np.all(gain == 0.0)         # every increment lost
    else:
        np.testing.assert_array_equal(gain, H2 * lnf)   # every increment kept, exactly
