"""The measurement entry points: rewl_measure_peaks (the roofline's
denominators) and rewl_tables_digest (comparison of table sets too large to
copy to the host)."""
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


def test_measured_peaks_are_consistent(P):
    pk = P.measure_peaks()
    import torch
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    assert pk["sms"] == sms
    for k in ("lop3_ops_per_s", "iadd_ops_per_s", "imad_ops_per_s", "ffma_ops_per_s", "smem_bytes_per_s",
              "l2_bytes_per_s"):
        assert pk[k] > 0
    # no rate can exceed one warp instruction per cycle per SM sub-partition at 3 GHz
    ceiling = sms * 4 * 32 * 3.0e9
    for k in ("lop3_ops_per_s", "iadd_ops_per_s", "imad_ops_per_s", "ffma_ops_per_s"):
        assert pk[k] < ceiling
    assert pk["lop3_ops_per_s"] <= pk["iadd_ops_per_s"] * 1.05
    assert pk["smem_bytes_per_s"] > pk["l2_bytes_per_s"]
    assert 1.0 <= pk["dep_iadd_cycles"] < 20.0


def test_table_digest_follows_the_tables(P):
    kw = dict(L=8, n_win_E=3, n_win_M=3, walkers_per_window=4, exchange_interval=5000, seed=20152899)
    a = P.REWL(P.Config(precision=P.FP64, **kw))
    b = P.REWL(P.Config(precision=P.F32X2, **kw))
    assert a.digest() == b.digest()                 # same (empty) tables in both formats
    a.run_cycles(30)
    b.run_cycles(30)
    la, Ha = a.tables()
    lb, Hb = b.tables()
    assert np.array_equal(la, lb) and np.array_equal(Ha, Hb)
    assert a.digest() == b.digest()                 # same chain, same values, different formats
    d0 = a.digest()
    Ha2 = Ha.copy()
    k = int(np.flatnonzero(Ha2 > 0)[0])
    Ha2[k] += 1
    a.set_tables(la, Ha2)
    assert a.digest() != d0                         # one visit more in one bin
    la2 = la.copy()
    la2[k] += 2.0 ** -20
    a.set_tables(la2, Ha)
    assert a.digest() != d0                         # one ln g value moved by 2^-20
    a.set_tables(la, Ha)
    assert a.digest() == d0


def test_autotuned_tiling_keeps_the_trajectory(P):
    """The autotuner times every tiling and placement on the actual
    configuration; whichever it returns runs the same chain as the default
    tiling (same table digest and walker states after whole cycles)."""
    from paper_1508_02748_gb300.autotune import autotune
    cfg = P.Config(L=8, n_win_E=2, n_win_M=2, walkers_per_window=3, exchange_interval=2000, seed=20152901)
    tuned = autotune(cfg, cache_path=None, cycles=2)
    assert tuned.sampler in (P.SAMPLER_WARP, P.SAMPLER_THREAD)
    assert tuned.table_mode in (P.TABLES_AUTO, P.TABLES_GLOBAL)
    assert tuned.lattice_mode in (P.LATTICE_AUTO, P.LATTICE_SHARED)
    a, b = P.REWL(cfg), P.REWL(tuned)
    a.run_cycles(40)
    b.run_cycles(40)
    assert a.digest() == b.digest()
    sa, pa = a.walkers()
    sb, pb = b.walkers()
    assert np.array_equal(sa, sb) and np.array_equal(pa, pb)
    a.close()
    b.close()
