"""Pins of the serial REWL oracle (oracle/rewl_oracle.c).

Each test checks the oracle against something other than itself: the exact
density of states (enumeration / transfer matrix / closed forms), invariants
that follow from the update rule of Sec. 2, the detailed-balance acceptance
frequency of Eq. 2, and exact reconstruction of a known g(E,M) by the join of
Eqs. 3-4.
"""
import math
import os

import numpy as np
import pytest

import oracle
from oracle import OracleConfig, OracleREWL

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _lg(g):
    g = np.asarray(g, dtype=np.float64)
    with np.errstate(divide="ignore"):
        return np.where(g > 0, np.log(np.where(g > 0, g, 1.0)), -np.inf)


def _spin_E_M(sp, L):
    s = np.where(sp.reshape(L, L) > 0, 1, -1)
    E = -int((s * np.roll(s, 1, 0)).sum() + (s * np.roll(s, 1, 1)).sum())
    return E, int(s.sum())


def _run_to_done(r, step=50, max_cycles=10**7):
    while not r.info()["done"] and r.info()["cycle"] < max_cycles:
        r.run_cycles(step)
    return r.info()


# ------------------------------------------------------------------ geometry --

def test_window_geometry_L8_3x3():
    r = OracleREWL(OracleConfig(L=8, n_win_E=3, n_win_M=3, walkers_per_window=1, seed=1))
    w = r.windows()
    # 65 bins per axis, w = ceil(65 / 1.5) = 44, starts 0, 11 (10.5 rounded up), 21
    assert [tuple(x) for x in w[:3, :2]] == [(0, 43), (11, 54), (21, 64)]
    assert [tuple(x) for x in w[::3, 2:4]] == [(0, 43), (11, 54), (21, 64)]
    assert w[:, 4].all()
    for a in range(2):
        ov = w[a, 1] - w[a + 1, 0] + 1
        assert ov / 44 >= 0.74


def test_window_geometry_L32_16x4():
    r = OracleREWL(OracleConfig(L=32, n_win_E=16, n_win_M=4, walkers_per_window=1, seed=1,
                                drive_budget=10**8))
    w = r.windows()
    widths_e = set((w[:, 1] - w[:, 0] + 1).tolist())
    widths_m = set((w[:, 3] - w[:, 2] + 1).tolist())
    assert widths_e == {216} and widths_m == {586}
    assert w[15, 1] == 1024 and w[-1, 3] == 1024
    assert w[:, 4].all()
    st, _ = r.walkers()
    for k in range(w.shape[0]):
        assert w[k, 0] <= st[k, 0] <= w[k, 1] and w[k, 2] <= st[k, 1] <= w[k, 3]


# ---------------------------------------------------------------- invariants --

@pytest.mark.parametrize("L", [4, 5])
def test_trial_bookkeeping_invariants(L):
    """After n trials of iteration 0 (ln f = 1): the stored (E, M) is the one
    of the spins, sum H = trials, sum ln g = trials * ln f, visited bins are
    occupied bins inside the walker's window."""
    N = L * L
    g = oracle.enumerate_gEM(L)
    r = OracleREWL(OracleConfig(L=L, n_win_E=2, n_win_M=2, walkers_per_window=2,
                                overlap_E=0.6, overlap_M=0.6, exchange_interval=997, seed=7))
    r.sweep(997)
    r.exchange()
    r.sweep(1003)
    st, sp = r.walkers()
    lng, H, toff = r.tables()
    win = r.windows()
    for w in range(st.shape[0]):
        E, M = _spin_E_M(sp[w], L)
        assert st[w, 0] == (E + 2 * N) // 4 and st[w, 1] == (M + N) // 2
        assert st[w, 2] == 2000
        h = H[toff[w]:toff[w + 1]]
        gl = lng[toff[w]:toff[w + 1]]
        assert h[h >= 0].sum() == 2000
        assert gl.sum() == 2000.0
        e0, e1, m0, m1, _ = win[w // 2]
        wm = m1 - m0 + 1
        for i in np.nonzero(h >= 0)[0]:
            e, m = e0 + i // wm, m0 + i % wm
            assert g[e, m] > 0


def test_flatness_rule_and_advance():
    """80% rule (Sec. 3) on hand-set histograms, H reset and ln f halving."""
    r = OracleREWL(OracleConfig(L=4, walkers_per_window=1, seed=3))
    lng, H, toff = r.tables()
    H[:] = -1
    H[:3] = [10, 10, 8]          # min 8 >= 0.8 * 28/3
    r.set_tables(lng, H)
    assert r.check_advance()
    _, H2, _ = r.tables()
    assert list(H2[:3]) == [0, 0, 0] and (H2[3:] == -1).all()
    assert r.info()["lnf"] == 0.5 and r.info()["iter"] == 1
    H2[:3] = [10, 10, 7]         # 7 < 0.8 * 9
    r.set_tables(lng, H2)
    assert not r.check_advance()
    H2[:2] = [4, 6]              # tie: 4 = 0.8 * 5 counts as flat
    H2[2] = -1
    r.set_tables(lng, H2)
    assert r.check_advance()
    assert r.info()["lnf"] == 0.25


# ------------------------------------------------------------- convergence --

def test_serial_wl_L4_converges_to_enumeration():
    """Plain serial 2D WL over the whole (E, M) range, ln f 1 -> 1e-6 (the
    paper's serial WL of Sec. 2 at L = 4) reproduces the exact g(E, M).

    One walker at 80% flatness lands at a mean relative error of the E
    marginal near 1e-2 (measured over 8 seeds with this check interval: mean
    1.6e-2, largest 2.5e-2), above the 5e-3 that REWL with several walkers
    per window reaches; the bounds below are that distribution's."""
    g = oracle.enumerate_gEM(4)
    gE = g.sum(axis=1)
    lgE, lgEM = _lg(gE), _lg(g)
    mean_eps, signed = [], []
    for rep in range(4):
        r = OracleREWL(OracleConfig(L=4, exchange_interval=1000, seed=20151811 + rep))
        inf = _run_to_done(r)
        assert inf["done"] and inf["iter"] == 21
        J, _, _ = r.join()
        assert np.array_equal(np.isfinite(J), g > 0)     # exactly the occupied bins
        mE = oracle.marginal_e(J)
        occ = gE > 0
        eps = np.abs(mE[occ] - lgE[occ]) / lgE[occ]
        mean_eps.append(eps.mean())
        signed.append((mE[occ] - lgE[occ]).mean())
        big = g > 1
        assert np.abs(J[big] - lgEM[big]).max() < 0.25
    assert max(mean_eps) < 0.026
    assert np.mean(mean_eps) < 0.018
    assert abs(np.mean(signed)) < 0.02


def test_L4_sixteen_walkers_meet_error_gate():
    """The same run with 16 walkers in the one window, merged at the end
    (Sec. 2): the mean relative error of the E marginal against the
    enumeration falls below 5e-3 (largest over 64 seeds: 4.0e-3)."""
    g = oracle.enumerate_gEM(4)
    gE = g.sum(axis=1)
    lgE = _lg(gE)
    for rep in range(2):
        r = OracleREWL(OracleConfig(L=4, walkers_per_window=16, exchange_interval=1000, seed=20151811 + rep))
        inf = _run_to_done(r)
        assert inf["done"] and inf["iter"] == 21
        J, _, _ = r.join()
        mE = oracle.marginal_e(J)
        ok = gE > 1
        assert (np.abs(mE[ok] - lgE[ok]) / lgE[ok]).mean() < 5e-3


def test_serial_wl_L5_odd_lattice():
    g = oracle.enumerate_gEM(5)
    r = OracleREWL(OracleConfig(L=5, exchange_interval=5000, lnf_final=1e-4, seed=99))
    _run_to_done(r)
    J, _, _ = r.join()
    assert np.array_equal(np.isfinite(J), g > 0)
    lg = _lg(g)
    big = g > 1
    rel = np.abs(J[big] - lg[big]) / lg[big]
    assert rel.mean() < 0.03


def test_rewl_L6_2x2_joint_and_marginals():
    """2D REWL with E and M both split (Sec. 2, last paragraph): the joined
    table matches the exact joint g(E, M) (transfer matrix) and its M
    marginal matches the binomial closed form."""
    L, N = 6, 36
    g = oracle.transfer_gEM(L)
    r = OracleREWL(OracleConfig(L=L, n_win_E=2, n_win_M=2, walkers_per_window=2,
                                exchange_interval=2000, lnf_final=1e-5, seed=4242))
    _run_to_done(r)
    J, em, mm = r.join()
    w = r.windows()
    assert w[1, 0] <= em[0] <= w[0, 1] and w[2, 2] <= mm[0] <= w[0, 3]
    assert np.array_equal(np.isfinite(J), g > 0)
    lg = _lg(g)
    big = g > 1
    assert (np.abs(J[big] - lg[big]) / lg[big]).mean() < 0.02
    # M marginal against C(N, m)
    with np.errstate(divide="ignore"):
        mx = J.max(axis=0)
        mM = mx + np.log(np.exp(J - mx).sum(axis=0))
    lbin = np.array([math.log(math.comb(N, m)) for m in range(N + 1)])
    inner = slice(1, N)
    assert np.abs(mM[inner] - lbin[inner]).max() < 0.1
    inf = r.info()
    assert inf["exch_accept"] > 0 and inf["exch_attempt"] >= inf["exch_accept"]


# ---------------------------------------------------------------- exchange --

def test_exchange_acceptance_frequency_matches_eq2():
    """Two walkers in adjacent windows, tables held fixed: the swap is a
    two-state chain whose acceptance from the state (X at i, Y at j) must be
    min[1, g_i(X)/g_i(Y) * g_j(Y)/g_j(X)] (Eq. 2) and from the swapped state
    the reciprocal."""
    L, N = 4, 16
    rng = np.random.default_rng(5)
    for attempt in range(50):
        sp = rng.integers(0, 2, size=(2, N), dtype=np.uint8)
        r = OracleREWL(OracleConfig(L=L, n_win_E=2, n_win_M=1, overlap_E=0.75,
                                    walkers_per_window=1, seed=11), init_spins=sp)
        st, _ = r.walkers()
        w = r.windows()
        inside = all(w[1, 0] <= st[k, 0] <= w[0, 1] for k in range(2))
        if inside and (st[0, 0], st[0, 1]) != (st[1, 0], st[1, 1]):
            break
    else:
        pytest.skip("no suitable start found")
    lng, H, toff = r.tables()
    (eX, mX), (eY, mY) = (st[0, 0], st[0, 1]), (st[1, 0], st[1, 1])

    def idx(win, e, m):
        e0, _, m0, m1, _ = w[win]
        return (e - e0) * (m1 - m0 + 1) + (m - m0)

    gi = lng[toff[0]:toff[1]]
    gj = lng[toff[1]:toff[2]]
    gi[idx(0, eX, mX)], gi[idx(0, eY, mY)] = 0.0, 0.7
    gj[idx(1, eY, mY)], gj[idx(1, eX, mX)] = 0.0, 0.5
    r.set_tables(lng, H)
    ratio = math.exp((0.0 - 0.7) + (0.0 - 0.5))      # state a: X at walker 0
    acc = {"a": [0, 0], "b": [0, 0]}
    for _ in range(4 * 6000):
        s0, _ = r.walkers()
        state = "a" if (s0[0, 0], s0[0, 1]) == (eX, mX) else "b"
        before = r.info()["exch_accept"]
        r.exchange()
        inf = r.info()
        if inf["xstep"] % 4 == 1:                       # the E-even phase just ran
            acc[state][0] += 1
            acc[state][1] += inf["exch_accept"] - before
    pa = acc["a"][1] / acc["a"][0]
    pb = acc["b"][1] / acc["b"][0]
    na = acc["a"][0]
    assert abs(pa - ratio) < 4 * math.sqrt(ratio * (1 - ratio) / na)
    assert pb == 1.0


# -------------------------------------------------------------------- join --

def test_join_reconstructs_exact_table_L6():
    """Given exact ln g(E, M) restricted to each window, shifted by an
    arbitrary constant per walker, the merge + join + normalisation of
    Eqs. 3-4 returns the exact table (sum g = 2^N) on occupied bins."""
    L, N = 6, 36
    g = oracle.transfer_gEM(L)
    lg = _lg(g)
    r = OracleREWL(OracleConfig(L=L, n_win_E=3, n_win_M=2, walkers_per_window=3, seed=8))
    w = r.windows()
    lng, H, toff = r.tables()
    rng = np.random.default_rng(0)
    for k in range(toff.size - 1):
        e0, e1, m0, m1, _ = w[k // 3]
        blk = lg[e0:e1 + 1, m0:m1 + 1]
        seen = np.isfinite(blk)
        lng[toff[k]:toff[k + 1]] = np.where(seen, blk + rng.normal() * 50, 0.0).ravel()
        H[toff[k]:toff[k + 1]] = np.where(seen, 1, -1).ravel()
    r.set_tables(lng, H)
    J, em, mm = r.join()
    assert np.array_equal(np.isfinite(J), g > 0)
    occ = g > 0
    assert np.abs(J[occ] - lg[occ]).max() < 1e-9


def test_rewl_L8_short_run_tracks_exact():
    """A short L = 8, 3 x 3, 4-walker run (ln f to 1/256) already lands on the
    exact E marginal within a few percent."""
    gold = np.loadtxt(os.path.join(GOLD, "gEM_L8.txt"), dtype=np.float64)
    lgE = _lg(gold.sum(axis=1))
    r = OracleREWL(OracleConfig(L=8, n_win_E=3, n_win_M=3, walkers_per_window=4,
                                exchange_interval=10000, lnf_final=1.0 / 256, seed=20152811))
    _run_to_done(r)
    J, _, _ = r.join()
    mE = oracle.marginal_e(J)
    occ = np.isfinite(lgE) & (lgE > 0)
    eps = np.abs(mE[occ] - lgE[occ]) / lgE[occ]
    assert eps.mean() < 0.03


def test_empty_windows_L8_6x6_geometry_and_join():
    """Windows with no possible (E, M) bin (Sec. 1: cusps and empty regions)
    are dropped; the join over the remaining windows still reconstructs the
    exact table.  L = 8, 6 x 6 windows at 50% overlap: the four high-E windows
    of the two extreme-M rows hold no configuration."""
    gold = np.loadtxt(os.path.join(GOLD, "gEM_L8.txt"), dtype=np.float64)
    lg = _lg(gold)
    W = 2
    r = OracleREWL(OracleConfig(L=8, n_win_E=6, n_win_M=6, overlap_E=0.5, overlap_M=0.5,
                                walkers_per_window=W, seed=31, drive_budget=10**8))
    w = r.windows()
    inactive = sorted((k % 6, k // 6) for k in range(36) if not w[k, 4])
    assert inactive == [(4, 0), (4, 5), (5, 0), (5, 5)]
    for k in range(36):          # an empty window really holds no configuration
        e0, e1, m0, m1, act = w[k]
        assert bool(act) == bool((gold[e0:e1 + 1, m0:m1 + 1] > 0).any())
    st, _ = r.walkers()
    for k in range(st.shape[0]):
        e0, e1, m0, m1, act = w[k // W]
        if act:
            assert e0 <= st[k, 0] <= e1 and m0 <= st[k, 1] <= m1
    lng, H, toff = r.tables()
    rng = np.random.default_rng(2)
    for k in range(toff.size - 1):
        e0, e1, m0, m1, act = w[k // W]
        if not act:
            continue
        blk = lg[e0:e1 + 1, m0:m1 + 1]
        seen = np.isfinite(blk)
        lng[toff[k]:toff[k + 1]] = np.where(seen, blk + rng.normal() * 20, 0.0).ravel()
        H[toff[k]:toff[k + 1]] = np.where(seen, 1, -1).ravel()
    r.set_tables(lng, H)
    J, em, mm = r.join()
    occ = gold > 0
    assert np.array_equal(np.isfinite(J), occ)
    assert np.abs(J[occ] - lg[occ]).max() < 1e-8
    r.run_cycles(3)               # sampling and exchange skip the empty windows
    assert r.info()["exch_attempt"] >= 0


def test_jackknife_pins():
    """Jackknife over walkers (Sec. 2): identical walkers (up to offsets) give
    zero error and the common table; independent noise of known size gives
    an error of that size divided by sqrt(W)."""
    L, N, W = 6, 36, 4
    gx = oracle.transfer_gEM(L).astype(np.float64)
    lg = _lg(gx)
    r = OracleREWL(OracleConfig(L=L, n_win_E=2, n_win_M=1, walkers_per_window=W, seed=9))
    w = r.windows()
    lng, H, toff = r.tables()
    rng = np.random.default_rng(3)
    T = toff[1] - toff[0]
    for k in range(toff.size - 1):
        e0, e1, m0, m1, _ = w[k // W]
        blk = lg[e0:e1 + 1, m0:m1 + 1]
        seen = np.isfinite(blk)
        lng[toff[k]:toff[k + 1]] = np.where(seen, blk + rng.normal() * 5, 0.0).ravel()
        H[toff[k]:toff[k + 1]] = np.where(seen, 1, -1).ravel()
    r.set_tables(lng, H)
    mean, err = oracle.jackknife(r)
    occ = gx > 0
    assert np.abs(mean[occ] - lg[occ]).max() < 1e-9
    assert np.nanmax(err[occ]) < 1e-9
    # With per-walker noise, every replicate's pieces carry a common shift
    # (offsets, matching, normalisation) that cancels in a difference of two
    # bins of the same window; for such a difference the jackknife error must
    # equal the textbook standard error s / sqrt(W) of the walkers' values.
    lng2 = np.where(H >= 0, lng + rng.normal(0, 0.01, size=lng.size), lng)
    r.set_tables(lng2, H)
    R = oracle.jackknife_replicates(r)
    e0, e1, m0, m1, _ = w[0]
    wm = m1 - m0 + 1
    b1, b2 = (3, 2), (4, 3)                                  # occupied, inside window 0 only
    assert b2[0] < w[1, 0] and occ[b1] and occ[b2]
    y = np.array([lng2[toff[k] + (b1[0] - e0) * wm + (b1[1] - m0)] - lng2[toff[k] + (b2[0] - e0) * wm + (b2[1] - m0)]
                  for k in range(W)])                        # walkers of window 0
    d = R[:, b1[0], b1[1]] - R[:, b2[0], b2[1]]
    _, err_d = oracle.jackknife_stats(d[:, None])
    assert err_d[0] == pytest.approx(y.std(ddof=1) / math.sqrt(W), rel=1e-9)
