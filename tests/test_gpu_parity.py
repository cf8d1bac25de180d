"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

Both sides draw their random numbers from their own Philox4x32-10 with the
same counter layout, so on the same seed they must produce the same
trajectory: integer state (spins, E, M, H, trial counters, exchange counters)
bit for bit, and ln g bit for bit too, because with ln f = 2^-k every ln g is
a dyadic rational that double additions represent exactly.  The join is
compared within 1e-9 (exp/log and summation order differ).
"""
import math
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


def _pair(P, init_spins=None, **kw):
    ocfg = OracleConfig(**{k: v for k, v in kw.items() if k in OracleConfig.__dataclass_fields__})
    gkw = dict(kw)
    gkw.pop("drive_budget", None)
    gcfg = P.Config(drive_budget=ocfg.drive_budget, **{k: v for k, v in gkw.items()
                                                        if k in P.Config.__dataclass_fields__})
    o = OracleREWL(ocfg, init_spins=init_spins)
    g = P.REWL(gcfg, init_spins=init_spins)
    return o, g


def _compare(o, g, tables=True):
    so, spo = o.walkers()
    sg, spg = g.walkers()
    np.testing.assert_array_equal(sg[:, :3], so[:, :3])          # e, m, trials
    np.testing.assert_array_equal(spg, spo)                      # spins
    if tables:
        lo, Ho, toff = o.tables()
        lg, Hg = g.tables()
        np.testing.assert_array_equal(Hg, Ho)
        np.testing.assert_array_equal(lg, lo)
    io, sg_ = o.info(), g.status()
    assert sg_["iteration"] == io["iter"] and sg_["done"] == io["done"]
    assert sg_["lnf"] == io["lnf"]
    assert sg_["exch_attempts"] == io["exch_attempt"] and sg_["exch_accepts"] == io["exch_accept"]


def test_philox_matches_oracle(P):
    import torch
    rng = np.random.default_rng(1)
    n = 1 << 20
    ctr = rng.integers(0, 2**32, size=(n, 4), dtype=np.uint64).astype(np.uint32)
    ctr[:64] = 0
    ctr[64:128] = 0xFFFFFFFF
    key = [0xDEADBEEF, 0x01234567]
    dev = torch.from_numpy(ctr.view(np.int32)).cuda()
    out = P.philox(dev, key).cpu().numpy().view(np.uint32)
    ref = oracle.philox4x32_10(ctr, key)
    np.testing.assert_array_equal(out, ref)


@pytest.mark.parametrize("L,nE,nM,W", [(8, 3, 3, 4), (32, 16, 4, 32), (64, 8, 4, 2), (24, 4, 2, 3),
                                       (33, 3, 3, 2), (5, 2, 2, 3)])
def test_geometry_init_and_drive(P, L, nE, nM, W):
    o, g = _pair(P, L=L, n_win_E=nE, n_win_M=nM, walkers_per_window=W, seed=20150811 + L,
                 drive_budget=10**8)
    np.testing.assert_array_equal(g.windows(), o.windows())
    _compare(o, g, tables=False)
    st, _ = g.walkers(spins=False)
    w = g.windows()
    for k in range(st.shape[0]):
        e0, e1, m0, m1, act = w[k // W]
        if act:
            assert e0 <= st[k, 0] <= e1 and m0 <= st[k, 1] <= m1


def test_host_init_spins(P):
    rng = np.random.default_rng(3)
    sp = rng.integers(0, 2, size=(2 * 2 * 2, 36), dtype=np.uint8)
    o, g = _pair(P, init_spins=sp, L=6, n_win_E=2, n_win_M=2, walkers_per_window=2, seed=9)
    _compare(o, g)


SAMPLERS = [0, 1]   # warp (tree speculation), thread


@pytest.mark.parametrize("sampler,lanes,prec", [(0, 32, 0), (0, 16, 1), (0, 8, 0), (0, 32, 1), (1, 0, 0), (1, 0, 1)])
@pytest.mark.parametrize("L", [4, 5, 6, 8, 24, 33, 48, 64])
def test_sweep_bit_exact_single_window(P, L, sampler, lanes, prec):
    """Sec. 2 trial/update rule, one window over the full (E, M) range; both
    ln g formats (double, compensated float pair) follow the same chain."""
    o, g = _pair(P, L=L, walkers_per_window=3, seed=77 + L, exchange_interval=5000, sampler=sampler,
                 lanes_per_walker=lanes, precision=prec)
    for n in (1, 2, 3, 999, 4000, 7):   # odd counts: the Philox pair straddles calls
        o.sweep(n)
        g.sweep(n)
        _compare(o, g)


@pytest.mark.parametrize("L,nE,nM,W", [(24, 2, 2, 3), (48, 4, 2, 2), (64, 4, 2, 2), (8, 3, 3, 4)])
@pytest.mark.parametrize("lanes", [32, 16, 8])
def test_table_modes_bit_exact(P, L, nE, nM, W, lanes):
    """Both places the warp sampler can keep S and H during a launch (global
    memory; all of a walker's bins staged in shared memory, where they fit)
    and both places it can keep a small lattice (N <= 64: one register, or
    shared memory like a larger one) follow the oracle's chain, through
    exchanges and checks, in both exact formats, for every group size."""
    modes = [(P.TABLES_GLOBAL, P.LATTICE_AUTO)] + ([(P.TABLES_STAGED, P.LATTICE_AUTO)] if L <= 8 else [])
    if L <= 8:
        modes += [(P.TABLES_GLOBAL, P.LATTICE_SHARED), (P.TABLES_STAGED, P.LATTICE_SHARED),
                  (P.TABLES_AUTO, P.LATTICE_REGISTER)]
    for prec in (0, 1):
        kw = dict(L=L, n_win_E=nE, n_win_M=nM, walkers_per_window=W, exchange_interval=4000, seed=91 + L,
                  drive_budget=10**8, lanes_per_walker=lanes, precision=prec)
        o = OracleREWL(OracleConfig(**{k: v for k, v in kw.items() if k in OracleConfig.__dataclass_fields__}))
        runs = [P.REWL(P.Config(table_mode=t, lattice_mode=m, **kw)) for t, m in modes]
        for chunk in (1, 6):
            o.run_cycles(chunk)
            for g in runs:
                g.run_cycles(chunk)
                _compare(o, g)
        for g in runs:
            g.close()
        o.close()


@pytest.mark.parametrize("sampler,prec", [(0, 0), (0, 1), (1, 0), (1, 1)])
def test_cycles_bit_exact_L8_3x3(P, sampler, prec):
    """The 2D REWL workload at L = 8 (3 x 3 windows at 75% overlap, 4 walkers
    per window, exchange every 10^4 trials): whole cycles of sampling,
    exchange (Eq. 2) and flatness checks stay bit-identical, through several
    iteration advances."""
    o, g = _pair(P, L=8, n_win_E=3, n_win_M=3, walkers_per_window=4, exchange_interval=10000,
                 seed=20152811, sampler=sampler, precision=prec)
    for chunk in (1, 3, 40, 100, 150):
        o.run_cycles(chunk)
        g.run_cycles(chunk)
        _compare(o, g)
    assert o.info()["iter"] >= 1
    assert o.info()["exch_accept"] > 0


@pytest.mark.parametrize("sampler,prec", [(0, 0), (1, 1)])
def test_plain_form_bit_exact_L8_3x3(P, sampler, prec):
    """The plain form (one launch per walker over several streams, host-driven
    exchange and check, no graph) is the same chain: bit-identical to the
    oracle, also when interleaved with batched cycles and with check_every > 1
    splitting check blocks between the two forms."""
    o, g = _pair(P, L=8, n_win_E=3, n_win_M=3, walkers_per_window=4, exchange_interval=10000,
                 check_every=3, seed=20152813, sampler=sampler, precision=prec)
    for chunk, plain in ((1, True), (2, False), (7, True), (40, False), (61, True), (150, False), (100, True)):
        o.run_cycles(chunk)
        (g.run_cycles_plain if plain else g.run_cycles)(chunk)
        _compare(o, g)
    assert o.info()["iter"] >= 2      # two iteration advances (the second one in plain cycles)


def test_plain_form_skips_empty_windows(P):
    """L = 8, 6 x 6 windows at 50% overlap (four windows can hold no
    configuration and get no walkers): the plain form launches only walkers of
    non-empty windows and matches the oracle."""
    o, g = _pair(P, L=8, n_win_E=6, n_win_M=6, overlap_E=0.5, overlap_M=0.5, walkers_per_window=2,
                 exchange_interval=2000, seed=4242)
    for chunk in (1, 5, 12):
        o.run_cycles(chunk)
        g.run_cycles_plain(chunk)
        _compare(o, g)


@pytest.mark.parametrize("sampler,wpb,lanes,prec", [(0, 3, 32, 0), (0, 8, 32, 1), (0, 3, 8, 1), (0, 2, 16, 0),
                                                     (1, 8, 0, 0), (1, 8, 0, 1)])
def test_cycles_with_check_interval_and_walkers_per_block(P, sampler, wpb, lanes, prec):
    """check_every > 1 (graph of several cycles) and a block size that leaves
    a ragged last block."""
    o, g = _pair(P, L=6, n_win_E=3, n_win_M=2, walkers_per_window=5, exchange_interval=3001,
                 check_every=3, walkers_per_block=wpb, seed=5, sampler=sampler, lanes_per_walker=lanes,
                 precision=prec)
    for chunk in (2, 7, 60):
        o.run_cycles(chunk)
        g.run_cycles(chunk)
        _compare(o, g)


@pytest.mark.parametrize("sampler,prec", [(0, 0), (0, 1), (1, 0)])
def test_run_to_done_L4_and_join(P, sampler, prec):
    """Serial WL at L = 4 run to ln f <= 1e-6: identical trajectory to the end,
    done flag, and the joined table equal to the oracle's within 1e-9."""
    o, g = _pair(P, L=4, exchange_interval=10000, seed=20151811, sampler=sampler, precision=prec)
    while not o.info()["done"]:
        o.run_cycles(64)
    st = g.run_cycles(o.info()["cycle"] + 5)   # extra cycles after done do nothing
    assert st["done"] == 1
    _compare(o, g)
    Jo, emo, mmo = o.join()
    Jg = g.lng()
    assert np.array_equal(np.isfinite(Jg), np.isfinite(Jo))
    fin = np.isfinite(Jo)
    np.testing.assert_allclose(Jg[fin], Jo[fin], rtol=0, atol=1e-9)
    mg = g.lng(P.LNG_MARGINAL_E)
    np.testing.assert_allclose(mg, oracle.marginal_e(Jo), rtol=0, atol=1e-9)


def test_join_matches_oracle_after_run_L8(P):
    o, g = _pair(P, L=8, n_win_E=3, n_win_M=3, walkers_per_window=4, exchange_interval=10000,
                 seed=20152812)
    o.run_cycles(300)
    g.run_cycles(300)
    _compare(o, g)
    Jo, emo, mmo = o.join()
    Jg, emg, mmg = g.lng(matches=True)
    np.testing.assert_array_equal(emg, emo)
    np.testing.assert_array_equal(mmg, mmo)
    fin = np.isfinite(Jo)
    assert np.array_equal(np.isfinite(Jg), fin)
    np.testing.assert_allclose(Jg[fin], Jo[fin], rtol=1e-12, atol=1e-9)


def test_join_reconstructs_exact_table_on_device(P):
    """Exact L = 6 ln g(E, M) per window with a random offset per walker: the
    device merge + join + normalisation returns the exact table."""
    L, N, W = 6, 36, 3
    gx = oracle.transfer_gEM(L).astype(np.float64)
    with np.errstate(divide="ignore"):
        lg = np.where(gx > 0, np.log(np.where(gx > 0, gx, 1)), -np.inf)
    g = P.REWL(P.Config(L=L, n_win_E=3, n_win_M=2, walkers_per_window=W, seed=8))
    w = g.windows()
    lng, H = g.tables()
    T = lng.size // (w.shape[0] * W)
    rng = np.random.default_rng(0)
    for k in range(w.shape[0] * W):
        e0, e1, m0, m1, _ = w[k // W]
        blk = lg[e0:e1 + 1, m0:m1 + 1]
        seen = np.isfinite(blk)
        lng[k * T:(k + 1) * T] = np.where(seen, blk + rng.normal() * 50, 0.0).ravel()
        H[k * T:(k + 1) * T] = np.where(seen, 1, -1).ravel()
    g.set_tables(lng, H)
    J = g.lng()
    occ = gx > 0
    assert np.array_equal(np.isfinite(J), occ)
    assert np.abs(J[occ] - lg[occ]).max() < 1e-9


def test_flatness_check_parity(P):
    o, g = _pair(P, L=6, n_win_E=2, n_win_M=1, walkers_per_window=2, seed=12)
    rng = np.random.default_rng(4)
    for trial in range(20):
        lng, H = g.tables()
        H[:] = rng.integers(-1, 12, size=H.size)
        H[rng.random(H.size) < 0.5] = -1
        if trial % 3 == 0:
            H[H >= 0] = 10
        g.set_tables(lng, H)
        lo, Ho, _ = o.tables()
        o.set_tables(lo, H)
        ao = o.check_advance()
        ag = g.check()
        assert ao == ag
        _compare(o, g)


@pytest.mark.parametrize("sampler", [0, 1])
def test_full_size_L32_batched_cycles(P, sampler):
    """The batched workload at full size (L = 32, 16 x 4 windows, 32 walkers
    per window = 2048 walkers, exchange every 10^4 trials) in the launch
    configuration the benchmark times: two full cycles bit-identical."""
    from paper_1508_02748_gb300.workloads import REWL_L32 as w
    o, g = _pair(P, L=w.L, n_win_E=w.n_win_E, n_win_M=w.n_win_M, walkers_per_window=w.walkers_per_window,
                 exchange_interval=w.exchange_interval, check_every=w.check_every, seed=w.seed(0),
                 drive_budget=10**8, precision=1, sampler=sampler)
    o.run_cycles(2)
    g.run_cycles(2)
    so, spo = o.walkers()
    sg, spg = g.walkers()
    np.testing.assert_array_equal(sg[:, :3], so[:, :3])
    np.testing.assert_array_equal(spg, spo)
    lo, Ho, _ = o.tables()
    lg, Hg = g.tables()
    np.testing.assert_array_equal(Hg, Ho)
    np.testing.assert_array_equal(lg, lo)
    assert g.status()["exch_attempts"] == o.info()["exch_attempt"]


@pytest.mark.parametrize("prec", [0, 1])
def test_empty_windows_cycles_and_join(P, prec):
    """L = 8, 6 x 6 windows at 50% overlap: four windows hold no configuration
    and get no walkers; sampling, exchange, checks and the join skip them
    exactly as the oracle does."""
    o, g = _pair(P, L=8, n_win_E=6, n_win_M=6, overlap_E=0.5, overlap_M=0.5, walkers_per_window=2,
                 exchange_interval=4000, seed=31, drive_budget=10**8, precision=prec)
    np.testing.assert_array_equal(g.windows(), o.windows())
    assert (g.windows()[:, 4] == 0).sum() == 4
    for chunk in (2, 30, 80):
        o.run_cycles(chunk)
        g.run_cycles(chunk)
        _compare(o, g)
    assert g.status()["n_walkers"] == 2 * 32
    Jo, emo, mmo = o.join()
    Jg, emg, mmg = g.lng(matches=True)
    np.testing.assert_array_equal(emg, emo)
    np.testing.assert_array_equal(mmg, mmo)
    fin = np.isfinite(Jo)
    assert np.array_equal(np.isfinite(Jg), fin)
    np.testing.assert_allclose(Jg[fin], Jo[fin], rtol=1e-12, atol=1e-9)


@pytest.mark.parametrize("what", [0, 1])
def test_jackknife_matches_oracle(P, what):
    """Jackknife over walkers (Sec. 2), device vs oracle on the same run."""
    o, g = _pair(P, L=8, n_win_E=3, n_win_M=3, walkers_per_window=4, exchange_interval=10000, seed=20152814)
    o.run_cycles(250)
    g.run_cycles(250)
    _compare(o, g)
    mo, eo = oracle.jackknife(o, marginal=(what == 1))
    mg, eg = g.jackknife(what)
    fin = np.isfinite(mo)
    assert np.array_equal(np.isfinite(mg), fin)
    np.testing.assert_allclose(mg[fin], mo[fin], rtol=1e-12, atol=1e-9)
    np.testing.assert_allclose(eg[fin], eo[fin], rtol=1e-6, atol=1e-9)
    assert np.nanmax(eo[fin]) > 0
