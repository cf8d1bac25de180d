"""The paper's own experiment shape (Sec. 3) on the oracle, and Eq. 5.

Sec. 3 splits the energy range only (M unrestricted) into equal windows at
50% overlap with three walkers per window, and compares the REWL result with
a serial WL run over the whole (E, M) range through the relative difference
of Eq. 5.  Pins: closed-form values of Eq. 5, the exact joint g(E, M) from the
transfer matrix, and the binomial M marginal.
"""
import math

import numpy as np

import oracle
from oracle import OracleConfig, OracleREWL


def _lg(g):
    g = np.asarray(g, dtype=np.float64)
    with np.errstate(divide="ignore"):
        return np.where(g > 0, np.log(np.where(g > 0, g, 1.0)), -np.inf)


def _run_to_done(r, step=50):
    while not r.info()["done"]:
        r.run_cycles(step)
    return r.info()


# ------------------------------------------------------------------- Eq. 5 --

def test_relative_difference_closed_forms():
    """Eq. 5: |g_a - g_b| / ((g_a + g_b) / 2).  g_a = g_b gives 0, g_a = 3 g_b
    gives 2/2 = 1, g_a = 2 g_b gives 1/(3/2) = 2/3, g_a = 9 g_b gives 8/5; the
    result is symmetric, depends only on the ratio (so it holds at the
    magnitudes of ln g at L = 64, ~2800), is 2 where one table is empty and
    undefined where both are."""
    base = np.array([0.0, 5.0, 2800.0, -3.0])
    for b in base:
        a = np.array([b, b + math.log(3.0), b + math.log(2.0), b + math.log(9.0), b - math.log(3.0)])
        bb = np.full_like(a, b)
        d = oracle.relative_difference(a, bb)
        # ln 3 added to b rounds to a multiple of ulp(b) (4.5e-13 at 2800)
        tol = 4 * np.spacing(max(abs(b), 1.0))
        np.testing.assert_allclose(d, [0.0, 1.0, 2.0 / 3.0, 8.0 / 5.0, 1.0], rtol=0, atol=tol)
        np.testing.assert_array_equal(oracle.relative_difference(bb, a), d)
    d = oracle.relative_difference(np.array([-np.inf, 1.0, -np.inf]), np.array([7.0, -np.inf, -np.inf]))
    assert d[0] == 2.0 and d[1] == 2.0 and np.isnan(d[2])


def test_relative_difference_of_small_perturbation():
    """For ln g_a = ln g_b + x with small x, Eq. 5 is |x| to first order
    (2 tanh(|x|/2) exactly); checked on a 2-D table with shapes kept."""
    rng = np.random.default_rng(3)
    b = rng.uniform(0.0, 100.0, size=(9, 9))
    x = rng.uniform(-1e-3, 1e-3, size=(9, 9))
    d = oracle.relative_difference(b + x, b)
    assert d.shape == (9, 9)
    np.testing.assert_allclose(d, np.abs(x), rtol=1e-6, atol=1e-12)


# ------------------------------------------------------ E-only split (Sec. 3) --

def test_E_split_join_reconstructs_exact_table_L6():
    """Three E windows at 50% overlap spanning all M (Sec. 3's split): exact
    ln g(E, M) restricted to each window and shifted by an arbitrary constant
    per walker is joined (Eqs. 3-4 along E only) back to the exact table."""
    L = 6
    g = oracle.transfer_gEM(L)
    lg = _lg(g)
    r = OracleREWL(OracleConfig(L=L, n_win_E=3, n_win_M=1, overlap_E=0.5, walkers_per_window=3, seed=9))
    w = r.windows()
    assert (w[:, 2] == 0).all() and (w[:, 3] == L * L).all()           # M unrestricted
    assert w[0, 0] == 0 and w[-1, 1] == L * L
    for a in range(2):                                                  # 50% overlap of equal windows
        width = w[a, 1] - w[a, 0] + 1
        assert abs((w[a, 1] - w[a + 1, 0] + 1) / width - 0.5) < 0.1
    lng, H, toff = r.tables()
    rng = np.random.default_rng(1)
    for k in range(toff.size - 1):
        e0, e1, m0, m1, _ = w[k // 3]
        blk = lg[e0:e1 + 1, m0:m1 + 1]
        seen = np.isfinite(blk)
        lng[toff[k]:toff[k + 1]] = np.where(seen, blk + rng.normal() * 30, 0.0).ravel()
        H[toff[k]:toff[k + 1]] = np.where(seen, 1, -1).ravel()
    r.set_tables(lng, H)
    J, em, mm = r.join()
    assert np.array_equal(np.isfinite(J), g > 0)
    occ = g > 0
    assert np.abs(J[occ] - lg[occ]).max() < 1e-9
    assert all(w[a + 1, 0] <= em[a] <= w[a, 1] for a in range(2))


def test_paper_shape_L6_rewl_against_serial_wl_eq5():
    """Sec. 3 at L = 6: E split into 3 windows at 50% overlap, 3 walkers per
    window, against serial WL over all (E, M) with one walker, both to
    ln f <= 1e-4.  Both land on the exact joint table; their Eq. 5 relative
    difference is small everywhere and of the order of each one's own error
    against the exact table; the M marginal is binomial."""
    L, N = 6, 36
    g = oracle.transfer_gEM(L)
    lg = _lg(g)
    re = OracleREWL(OracleConfig(L=L, n_win_E=3, n_win_M=1, overlap_E=0.5, walkers_per_window=3,
                                 exchange_interval=10000, lnf_final=1e-4, seed=20156811))
    wl = OracleREWL(OracleConfig(L=L, exchange_interval=10000, lnf_final=1e-4, seed=20156812))
    _run_to_done(re)
    _run_to_done(wl)
    Jre, _, _ = re.join()
    Jwl, _, _ = wl.join()
    occ = g > 0
    assert np.array_equal(np.isfinite(Jre), occ) and np.array_equal(np.isfinite(Jwl), occ)
    d = oracle.relative_difference(Jwl, Jre)
    assert np.isnan(d[~occ]).all()
    d_occ = d[occ]
    err_re = oracle.relative_difference(Jre, lg)[occ]
    err_wl = oracle.relative_difference(Jwl, lg)[occ]
    assert d_occ.mean() < 0.1 and d_occ.max() < 0.5
    assert d_occ.mean() < 2.5 * max(err_re.mean(), err_wl.mean())
    with np.errstate(divide="ignore"):
        mx = Jre.max(axis=0)
        mM = mx + np.log(np.exp(Jre - mx).sum(axis=0))
    lbin = np.array([math.log(math.comb(N, m)) for m in range(N + 1)])
    assert np.abs(mM[1:N] - lbin[1:N]).max() < 0.1


# ------------------------------------------- rescaling rule of a join step --

def _exact_pieces(r, lg, distort, rng):
    """Set every walker's table to the exact ln g of its window, plus a random
    constant per walker and distort(window, e, m) for the window's bins."""
    w = r.windows()
    W = r.cfg.walkers_per_window
    lng, H, toff = r.tables()
    for k in range(toff.size - 1):
        e0, e1, m0, m1, _ = w[k // W]
        ee, mm = np.meshgrid(np.arange(e0, e1 + 1), np.arange(m0, m1 + 1), indexing="ij")
        blk = lg[e0:e1 + 1, m0:m1 + 1]
        seen = np.isfinite(blk)
        val = blk + rng.normal() * 20 + distort(k // W, ee, mm)
        lng[toff[k]:toff[k + 1]] = np.where(seen, val, 0.0).ravel()
        H[toff[k]:toff[k + 1]] = np.where(seen, 1, -1).ravel()
    r.set_tables(lng, H)


def test_both_rescaling_rules_reconstruct_exact_pieces_L6():
    """Pieces that differ from the exact table by a constant per walker are
    joined back to the exact table by either rescaling rule, E and M split."""
    L = 6
    g = oracle.transfer_gEM(L)
    lg = _lg(g)
    occ = g > 0
    for rule in (oracle.JOIN_MARGINAL, oracle.JOIN_PER_SLICE):
        r = OracleREWL(OracleConfig(L=L, n_win_E=3, n_win_M=2, walkers_per_window=2, seed=21))
        _exact_pieces(r, lg, lambda win, e, m: 0.0, np.random.default_rng(rule))
        J, _, _ = r.join(rule)
        assert np.array_equal(np.isfinite(J), occ)
        assert np.abs(J[occ] - lg[occ]).max() < 1e-9


def _spread(x):
    return float(x.max() - x.min())


def test_per_slice_rule_removes_slice_offsets_E_join_L6():
    """Two E windows (M unrestricted); the upper one carries an offset that
    depends on M alone.  Rescaling per M slice at E_mat (rule 1) puts every
    slice that is occupied at E_mat back on the exact table (one common
    constant, fixed by the normalisation); the single marginal constant
    (rule 0) leaves the offsets in."""
    L = 6
    g = oracle.transfer_gEM(L)
    lg = _lg(g)
    occ = g > 0
    delta = np.random.default_rng(5).uniform(-0.3, 0.3, size=L * L + 1)
    out = {}
    for rule in (oracle.JOIN_MARGINAL, oracle.JOIN_PER_SLICE):
        r = OracleREWL(OracleConfig(L=L, n_win_E=2, n_win_M=1, overlap_E=0.5, walkers_per_window=2, seed=22))
        _exact_pieces(r, lg, lambda win, e, m: np.where(win == 1, delta[m], 0.0), np.random.default_rng(7))
        J, em, _ = r.join(rule)
        out[rule] = (J, int(em[0]))
    J1, p = out[oracle.JOIN_PER_SLICE]
    assert np.array_equal(np.isfinite(J1), occ)
    matched = occ & occ[p][None, :]          # bins of slices M occupied at E_mat
    d1 = J1[matched] - lg[matched]
    assert _spread(d1) < 1e-9
    J0, p0 = out[oracle.JOIN_MARGINAL]
    assert p0 == p
    upper = matched & (np.arange(L * L + 1)[:, None] >= p)
    assert _spread(J0[upper] - lg[upper]) > 0.1


def test_per_slice_rule_removes_slice_offsets_M_join_L6():
    """The same along M: two M windows (E unrestricted), the upper one offset
    by a function of E alone; rule 1 rescales each E slice at M_mat."""
    L = 6
    g = oracle.transfer_gEM(L)
    lg = _lg(g)
    occ = g > 0
    delta = np.random.default_rng(6).uniform(-0.3, 0.3, size=L * L + 1)
    r = OracleREWL(OracleConfig(L=L, n_win_E=1, n_win_M=2, overlap_M=0.5, walkers_per_window=2, seed=23))
    _exact_pieces(r, lg, lambda win, e, m: np.where(win == 1, delta[e], 0.0), np.random.default_rng(8))
    J1, _, mm = r.join(oracle.JOIN_PER_SLICE)
    q = int(mm[0])
    matched = occ & occ[:, q][:, None]
    assert np.array_equal(np.isfinite(J1), occ)
    assert _spread(J1[matched] - lg[matched]) < 1e-9
    J0, _, _ = r.join(oracle.JOIN_MARGINAL)
    upper = matched & (np.arange(L * L + 1)[None, :] >= q)
    assert _spread(J0[upper] - lg[upper]) > 0.1
