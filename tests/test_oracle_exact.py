"""Pins of the exact density-of-states tools the oracle is checked against.

Independent routes must agree exactly: brute-force enumeration (all 2^N
configurations), the site-by-site transfer matrix, and Kaufman's closed-form
partition function expanded into integer coefficients (Beale's g(E), the
paper's exact reference in Sec. 1 and Fig. 5a).  Closed forms that hold at
every L pin them further.
"""
import math
import os

import numpy as np
import pytest

import oracle
from oracle.exact_ge import exact_gE

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _obj(a):
    return a.astype(object)


@pytest.mark.parametrize("L", [4, 5])
def test_enumeration_equals_transfer_matrix(L):
    assert np.array_equal(oracle.enumerate_gEM(L), oracle.transfer_gEM(L))


@pytest.mark.parametrize("L", [4, 6])
def test_kaufman_equals_transfer_matrix(L):
    tm = _obj(oracle.transfer_gEM(L)).sum(axis=1)
    assert exact_gE(L) == [int(v) for v in tm]


def test_kaufman_equals_transfer_matrix_L8():
    tm = _obj(oracle.transfer_gEM(8))
    ge = exact_gE(8)
    assert ge == [int(v) for v in tm.sum(axis=1)]
    # the stored joint L=8 table (written by golden/make_golden.py) is this one
    stored = np.loadtxt(os.path.join(GOLD, "gEM_L8.txt"), dtype=object)
    assert [[int(x) for x in row] for row in stored] == [[int(x) for x in row] for row in tm]


@pytest.mark.parametrize("L", [4, 5, 6])
def test_closed_forms(L):
    N = L * L
    g = _obj(oracle.transfer_gEM(L))
    # sum g = 2^N
    assert sum(sum(r) for r in g) == 2 ** N
    # g(E, M) = g(E, -M)
    assert all(g[e][m] == g[e][N - m] for e in range(N + 1) for m in range(N + 1))
    # M marginal is binomial: sum_E g(E, M) = C(N, number of up spins)
    for m in range(N + 1):
        assert sum(g[e][m] for e in range(N + 1)) == math.comb(N, m)
    # ground states, one flipped spin, two adjacent flipped spins
    assert g[0][0] == 1 and g[0][N] == 1
    assert g[2][1] == N and g[2][N - 1] == N
    assert g[3][2] == 2 * N and g[3][N - 2] == 2 * N
    gE = [sum(r) for r in g]
    assert gE[1] == 0                                  # E = -2N + 4 is empty
    if L >= 5:
        assert gE[4] == 2 * (math.comb(N, 2) + 5 * N)
    if L % 2 == 0:
        assert gE == gE[::-1]                          # E -> -E (sublattice flip)
        assert gE[N - 1] == 0
        assert g[N][N // 2] == 2
        assert g[N - 2][N // 2 - 1] == N and g[N - 2][N // 2 + 1] == N
    # every occupied bin satisfies E <= 2N - 4|M|
    for e in range(N + 1):
        for m in range(N + 1):
            if g[e][m]:
                assert 4 * e - 2 * N <= 2 * N - 4 * abs(2 * m - N)


def test_L4_known_values():
    g = _obj(oracle.enumerate_gEM(4))
    gE = [int(sum(r)) for r in g]
    assert gE[:5] == [2, 0, 32, 64, 424]
    assert sum(1 for r in g for v in r if v) == 80


@pytest.mark.parametrize("L", [4, 5, 6])
def test_possible_bin_bounds(L):
    """The window-emptiness bounds admit every occupied bin and are tight:
    for each M the lowest admitted E is occupied."""
    N = L * L
    g = oracle.transfer_gEM(L)
    for m in range(N + 1):
        occ = [e for e in range(N + 1) if g[e, m]]
        adm = [e for e in range(N + 1) if oracle.bin_possible(L, e, m)]
        assert set(occ) <= set(adm)
        assert min(occ) == min(adm)


def test_golden_lngE_files_match_closed_form_sums():
    # ln g(E) for L = 16, 32 and 64 written by golden/make_golden.py
    for L in (16, 32, 64):
        path = os.path.join(GOLD, f"lngE_L{L}.txt")
        if not os.path.exists(path):
            continue
        v = np.loadtxt(path)
        N = L * L
        assert v.shape == (N + 1,)
        fin = np.isfinite(v)
        mx = v[fin].max()
        lz = mx + math.log(np.exp(v[fin] - mx).sum())
        assert abs(lz - N * math.log(2.0)) < 1e-9 * N
        assert np.allclose(v, v[::-1], rtol=0, atol=1e-9, equal_nan=True) or \
            np.array_equal(np.isinf(v), np.isinf(v[::-1]))
        assert abs(v[0] - math.log(2)) < 1e-12
        assert abs(v[2] - math.log(2 * N)) < 1e-12
        assert abs(v[3] - math.log(4 * N)) < 1e-12                       # two adjacent flips
        assert abs(v[4] - math.log(2 * (math.comb(N, 2) + 5 * N))) < 1e-12
        assert np.isinf(v[1]) and np.isinf(v[N - 1])
