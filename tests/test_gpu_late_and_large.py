"""Parity with the oracle in the states and at the sizes the benchmarks meet.

- Late-run states: tables shaped like a converged run (the exact ln g of the
  8 x 8 torus inside each window, an offset near 8192 and dyadic noise), ln f
  from 2^-15 down, a first check that ends the iteration at once (H near
  1000 everywhere), then ordinary iterations: the float screen's near-ties,
  the exact re-decision and the fold of large visit counts at a late ln f
  all run, and the trajectory must stay the oracle's bit for bit.
- The geometry of the L = 64 precision study: 32 x 8 windows at 75% overlap
  (12 of them empty), tables in global memory, both exact formats, from
  creation and from a late state at ln f = 2^-27.
- The sizes of the uneven batch: L = 48 (16 x 4 windows, 8 walkers each) and
  L = 16 (4 x 2 windows, 32 walkers each) advanced together by one graph.
"""
import os

import numpy as np
import pytest

import oracle
from oracle import OracleConfig, OracleREWL

pytestmark = pytest.mark.gpu

GOLD = os.path.join(os.path.dirname(__file__), "golden")


@pytest.fixture(scope="module")
def P():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1508_02748_gb300 as P
    from paper_1508_02748_gb300 import build
    build.build()
    return P


def _pair(P, **kw):
    ocfg = OracleConfig(**{k: v for k, v in kw.items() if k in OracleConfig.__dataclass_fields__})
    gkw = {k: v for k, v in kw.items() if k in P.Config.__dataclass_fields__ and k != "drive_budget"}
    return OracleREWL(ocfg), P.REWL(P.Config(drive_budget=ocfg.drive_budget, **gkw))


def _compare(o, g):
    so, spo = o.walkers()
    sg, spg = g.walkers()
    np.testing.assert_array_equal(sg[:, :3], so[:, :3])
    np.testing.assert_array_equal(spg, spo)
    lo, Ho, _ = o.tables()
    lg, Hg = g.tables()
    np.testing.assert_array_equal(Hg, Ho)
    np.testing.assert_array_equal(lg, lo)
    io, st = o.info(), g.status()
    assert st["iteration"] == io["iter"] and st["done"] == io["done"] and st["lnf"] == io["lnf"]
    assert st["exch_attempts"] == io["exch_attempt"] and st["exch_accepts"] == io["exch_accept"]


def _late_tables(windows, W, T, lg_exact, rng, h_base):
    """Per walker: exact ln g on the window's occupied bins rounded to a
    multiple of 2^-20, plus a walker offset near 8192 and +-2^-11 of noise;
    H = h_base + 0..4 on occupied bins, -1 elsewhere."""
    n = windows.shape[0] * W
    lng = np.zeros(n * T)
    H = np.full(n * T, -1, dtype=np.int32)
    for k in range(n):
        e0, e1, m0, m1, _ = windows[k // W]
        blk = lg_exact[e0:e1 + 1, m0:m1 + 1]
        occ = np.isfinite(blk)
        off = 8192 + int(rng.integers(0, 2**12)) * 2.0**-10
        noise = rng.integers(-512, 512, size=blk.shape) * 2.0**-20
        v = np.where(occ, np.round(np.where(occ, blk, 0.0) * 2**20) / 2**20 + off + noise, 0.0)
        lng[k * T:(k + 1) * T] = v.ravel()
        H[k * T:(k + 1) * T] = np.where(occ, h_base + rng.integers(0, 5, size=blk.shape), -1).ravel()
    return lng, H


@pytest.mark.parametrize("sampler,lanes,prec", [(0, 32, 0), (0, 16, 1), (0, 8, 0), (1, 0, 0), (1, 0, 1)])
def test_late_run_state_bit_exact_L8_3x3(P, sampler, lanes, prec):
    g_ex = np.loadtxt(os.path.join(GOLD, "gEM_L8.txt"))
    with np.errstate(divide="ignore"):
        lg_ex = np.where(g_ex > 0, np.log(np.where(g_ex > 0, g_ex, 1.0)), -np.inf)
    o, g = _pair(P, L=8, n_win_E=3, n_win_M=3, walkers_per_window=4, exchange_interval=10000,
                 lnf_init=2.0**-15, seed=20152899, sampler=sampler, lanes_per_walker=lanes, precision=prec)
    w = g.windows()
    lng, H = g.tables()
    T = lng.size // (w.shape[0] * 4)
    lng, H = _late_tables(w, 4, T, lg_ex, np.random.default_rng(5), 1000)
    o.set_tables(lng, H)
    g.set_tables(lng, H)
    _compare(o, g)
    for chunk in (1, 10, 60, 120):
        o.run_cycles(chunk)
        g.run_cycles(chunk)
        _compare(o, g)
    assert o.info()["iter"] >= 1 and o.info()["lnf"] <= 2.0**-16


L64 = dict(L=64, n_win_E=32, n_win_M=8, walkers_per_window=1, exchange_interval=10000, check_every=16,
           drive_budget=10**8)


@pytest.mark.parametrize("prec", [0, 1])
def test_L64_32x8_geometry_two_cycles(P, prec):
    o, g = _pair(P, seed=20154811, precision=prec, **L64)
    np.testing.assert_array_equal(g.windows(), o.windows())
    assert (g.windows()[:, 4] == 0).sum() == 12
    o.run_cycles(2)
    g.run_cycles(2)
    _compare(o, g)


def test_L64_32x8_late_state_formats_agree(P):
    """From one late state (ln g = 2^14 plus up to 2^-7 in steps of 2^-27 on
    every bin, all bins marked visited, ln f = 2^-27, the finest ln f of the
    precision study) both exact formats and the oracle stay identical; plain
    float loses every increment (ln f is below half an ulp of 2^14)."""
    rng = np.random.default_rng(11)
    base = H0 = None
    out = {}
    for prec in (0, 1, 2):
        o, g = _pair(P, seed=20154812, precision=prec, lnf_init=2.0**-27, **L64)
        if base is None:
            n = g.tables()[1].size
            base = 16384 + rng.integers(0, 2**20, size=n) * 2.0**-27
            H0 = np.zeros(n, dtype=np.int32)
        g.set_tables(base, H0)
        g.run_cycles(2)
        if prec != 2:
            o.set_tables(base, H0)
            o.run_cycles(2)
            _compare(o, g)
        o.close()
        out[prec] = g.tables()
        g.close()
    np.testing.assert_array_equal(out[1][1], out[0][1])
    np.testing.assert_array_equal(out[1][0], out[0][0])
    lng32, H32 = out[2]
    assert (H32 > 0).sum() > 1000
    np.testing.assert_array_equal(lng32, base.astype(np.float32).astype(np.float64))


def test_batch_with_L48_and_L16_members(P):
    cfgs = [dict(L=48, n_win_E=16, n_win_M=4, walkers_per_window=8, exchange_interval=10000, check_every=1,
                 seed=20155801, precision=1, drive_budget=10**8),
            dict(L=16, n_win_E=4, n_win_M=2, walkers_per_window=32, exchange_interval=10000, check_every=1,
                 seed=20155802, precision=1, drive_budget=10**8)]
    runs = [P.REWL(P.Config(**{k: v for k, v in c.items() if k in P.Config.__dataclass_fields__})) for c in cfgs]
    b = P.Batch(runs)
    assert b.k == 1
    b.run_cycles(2)
    for c, g in zip(cfgs, runs):
        o = OracleREWL(OracleConfig(**{k: v for k, v in c.items() if k in OracleConfig.__dataclass_fields__}))
        o.run_cycles(2)
        _compare(o, g)
        o.close()
    b.close()
