"""Batched runs (rewl_batch_*): several REWL runs of different L, geometry
and precision advanced together by one CUDA graph must each follow exactly
the trajectory they follow alone -- and the oracle's."""
import numpy as np
import pytest

import oracle

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


CFGS = [dict(L=4, exchange_interval=3000, check_every=1, seed=101),
        dict(L=6, n_win_E=2, n_win_M=2, walkers_per_window=3, exchange_interval=2000, check_every=2, seed=102,
             precision=1),
        dict(L=8, n_win_E=3, n_win_M=3, walkers_per_window=4, exchange_interval=5000, check_every=4, seed=103),
        dict(L=12, n_win_E=4, n_win_M=2, walkers_per_window=2, exchange_interval=1000, check_every=1, seed=104,
             precision=1, lanes_per_walker=16)]


def _state(r):
    st, sp = r.walkers()
    lng, H = r.tables()
    return st[:, :3].copy(), sp, lng, H, r.status()


def test_batch_equals_solo_runs(P):
    batched = [P.REWL(P.Config(**c)) for c in CFGS]
    solo = [P.REWL(P.Config(**c)) for c in CFGS]
    b = P.Batch(batched)
    assert b.k == 4                       # lcm of check_every = 1, 2, 4, 1
    b.run_cycles(3 * b.k)
    b.enqueue()
    b.stream.synchronize()
    for r in solo:
        r.run_cycles(4 * b.k)
    for rb, rs in zip(batched, solo):
        sb, ss = _state(rb), _state(rs)
        for x, y in zip(sb[:4], ss[:4]):
            np.testing.assert_array_equal(x, y)
        assert sb[4]["cycles"] == ss[4]["cycles"] == 16
        assert sb[4]["exch_attempts"] == ss[4]["exch_attempts"]
    b.close()


def test_batch_member_matches_oracle(P):
    c = CFGS[2]
    o = oracle.OracleREWL(oracle.OracleConfig(**{k: v for k, v in c.items()
                                                 if k in oracle.OracleConfig.__dataclass_fields__}))
    runs = [P.REWL(P.Config(**cc)) for cc in CFGS]
    b = P.Batch(runs)
    b.run_cycles(2 * b.k)
    o.run_cycles(2 * b.k)
    so, spo = o.walkers()
    sg, spg = runs[2].walkers()
    np.testing.assert_array_equal(sg[:, :3], so[:, :3])
    np.testing.assert_array_equal(spg, spo)
    lo, Ho, _ = o.tables()
    lg, Hg = runs[2].tables()
    np.testing.assert_array_equal(Hg, Ho)
    np.testing.assert_array_equal(lg, lo)
    b.close()
