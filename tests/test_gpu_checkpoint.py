"""Checkpoint / resume (rewl_save, rewl_load): every random draw is a Philox
counter of the trial or exchange index, so a run restored from a checkpoint
continues exactly as the saved run does -- spins, bins, tables, counters."""
import os

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


@pytest.mark.parametrize("prec", [0, 1])
def test_resume_is_exact(P, tmp_path, prec):
    cfg = P.Config(L=8, n_win_E=3, n_win_M=3, walkers_per_window=4, exchange_interval=3000, check_every=2,
                   seed=777, precision=prec)
    a = P.REWL(cfg)
    a.run_cycles(41)                     # odd: the resumed run is mid check block
    path = os.path.join(tmp_path, "run.ckpt")
    a.save(path)
    a.run_cycles(90)
    b = P.REWL.load(path)
    assert b.cfg == a.cfg
    b.run_cycles(90)
    sa, spa = a.walkers()
    sb, spb = b.walkers()
    np.testing.assert_array_equal(sa, sb)
    np.testing.assert_array_equal(spa, spb)
    la, Ha = a.tables()
    lb, Hb = b.tables()
    np.testing.assert_array_equal(Ha, Hb)
    np.testing.assert_array_equal(la, lb)
    assert a.status() == b.status()
    np.testing.assert_array_equal(a.lng(), b.lng())


def test_load_rejects_other_files(P, tmp_path):
    path = os.path.join(tmp_path, "junk.ckpt")
    with open(path, "wb") as f:
        f.write(b"not a checkpoint" * 4)
    with pytest.raises(P.REWLError):
        P.REWL.load(path)
