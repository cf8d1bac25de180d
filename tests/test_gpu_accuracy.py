"""Accuracy of a whole run against the exact density of states.

The 2D REWL workload at L = 8 (3 x 3 windows at 75% overlap, 4 walkers per
window, exchange every 10^4 trials, ln f from 1 halved down to <= 1e-6, 80%
flatness) is run to its final ln f on the GPU in both exact table formats.
The joined E marginal (Eq. 3) must lie within a mean relative error of 5e-3
of the exact g(E) of the 8 x 8 torus (Beale's closed form, stored under
tests/golden/ by make_golden.py from the oracle), over every E with g(E) > 1
(the error metric of Fig. 5: |ln g_sim - ln g_exact| / ln g_exact, both
normalised to sum g = 2^N).  Both formats follow the same chain, so their
tables must also be identical.
"""
import os

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

GOLD = os.path.join(os.path.dirname(__file__), "golden")
GATE = 5e-3


@pytest.fixture(scope="module")
def P():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1508_02748_gb300 as P
    from paper_1508_02748_gb300 import build
    build.build()
    return P


def _run_to_done(P, precision):
    from paper_1508_02748_gb300.workloads import REWL_L8
    run = P.REWL(P.Config.from_workload(REWL_L8, replicate=0, drive_budget=10**8, precision=precision))
    st = run.status()
    while not st["done"]:
        st = run.run_cycles(1024)
        assert st["cycles"] < 200_000, "run did not reach its final ln f"
    return run, st


def test_rewl_L8_final_lnf_meets_error_gate_in_both_formats(P):
    ex = np.loadtxt(os.path.join(GOLD, "lngE_L8.txt"))
    ok = np.isfinite(ex) & (ex > 0)                    # g(E) > 1
    runs = {}
    for prec in (P.FP64, P.F32X2):
        run, st = _run_to_done(P, prec)
        assert st["iteration"] == 21 and st["lnf"] == 2.0 ** -20
        mE = run.lng(P.LNG_MARGINAL_E)
        assert np.array_equal(np.isfinite(mE), np.isfinite(ex))
        eps = np.abs(mE[ok] - ex[ok]) / ex[ok]
        assert eps.mean() <= GATE, f"mean relative error {eps.mean():.3e} above {GATE}"
        runs[prec] = (run, st, mE)
    (r64, s64, m64), (r32, s32, m32) = runs[P.FP64], runs[P.F32X2]
    assert s64["cycles"] == s32["cycles"]
    l64, H64 = r64.tables()
    l32, H32 = r32.tables()
    np.testing.assert_array_equal(H32, H64)
    np.testing.assert_array_equal(l32, l64)
    np.testing.assert_array_equal(m32, m64)
