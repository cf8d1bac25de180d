"""Exact energy density of states g(E) of the periodic L x L Ising model.

TEST INFRASTRUCTURE ONLY (the oracle side; see ``oracle/__init__.py``).

The paper (Sec. 1, Fig. 5a) compares the E marginal of its joint density of
states with the exact g(E) of Beale (Phys. Rev. Lett. 76, 78 (1996)), who
expanded Kaufman's finite-torus partition function into its exact integer
coefficients.  This module does the same expansion numerically at a
precision high enough to round every coefficient to its integer:

Kaufman (Phys. Rev. 76, 1232 (1949)), m x n torus, K = J/kT:
    Z = 1/2 (2 sinh 2K)^(mn/2) (Z1 + Z2 + Z3 + Z4)
    Z1 = prod_{r=0}^{n-1} 2 cosh(m g_{2r+1}/2),  Z2 = same with sinh,
    Z3 = prod_{r=0}^{n-1} 2 cosh(m g_{2r}/2),    Z4 = same with sinh,
    cosh g_l = cosh 2K coth 2K - cos(pi l / n),
    g_0 = 2K + ln tanh K (signed),  g_n = 2K + ln coth K.

For even m the half-angle functions are Chebyshev polynomials of c = cosh g:
cosh(m g/2) = T_{m/2}(c) and sinh(m g/2) = sinh(g) U_{m/2-1}(c).  The sinh g
factors pair up (l with 2n - l) into c^2 - 1, except l = 0 and l = n, whose
product sinh g_0 sinh g_n is written with the signed g_0 above.  Every term is
then a rational function of y = e^{2K}, and Z y^{-N} = sum_e g(e) z^e with
z = y^{-2} = e^{-4K} and e = (E + 2N)/4.  The coefficients are recovered by
evaluating at N+1 points z_k = exp(2 pi i (k + 1/2)/(N+1)) (the half step
keeps y away from the poles y = +-1) and applying the inverse discrete
Fourier transform, in mpmath at N log10(2) + 40 digits: coefficient e is
(1/(N+1)) Re sum_k Z(z_k) w_e^(k + 1/2) with w_e = exp(-2 pi i e/(N+1)),
summed in Horner form in powers of w_e.  Only e <= N/2 is summed: g(e) =
g(N - e) for even L (E -> -E maps the torus's ferromagnetic and
antiferromagnetic states onto each other).  Point evaluations and
coefficients can be spread over worker processes (``workers``); each is
the same sum.

Checked in the test suite against brute-force enumeration (L = 4) and the
transfer matrix (L = 6, 8) from ``exact.c``.
"""
from __future__ import annotations

import math

import mpmath


def _cheb_T(k: int, c):
    if k == 0:
        return mpmath.mpf(1)
    a, b = mpmath.mpf(1), c
    for _ in range(k - 1):
        a, b = b, 2 * c * b - a
    return b


def _cheb_U(k: int, c):
    if k < 0:
        return mpmath.mpf(0)
    a, b = mpmath.mpf(1), 2 * c
    if k == 0:
        return a
    for _ in range(k - 1):
        a, b = b, 2 * c * b - a
    return b


def _partition_scaled(L: int, y):
    """Z * y^{-N} at y = e^{2K} (complex allowed), square L x L torus, even L."""
    m = n = L
    N = L * L
    h = m // 2
    t = (y - 1) / (y + 1)                       # tanh K
    ch2 = (y + 1 / y) / 2                       # cosh 2K
    cth2 = (y * y + 1) / (y * y - 1)            # coth 2K
    a = ch2 * cth2
    cosv = [mpmath.cos(mpmath.pi * l / n) for l in range(2 * n)]
    c = [a - cosv[l] for l in range(2 * n)]
    # Z1, Z3: products of 2 T_h(c_l) over odd / even l.
    Z1 = mpmath.mpf(1)
    Z3 = mpmath.mpf(1)
    for r in range(n):
        Z1 *= 2 * _cheb_T(h, c[2 * r + 1])
        Z3 *= 2 * _cheb_T(h, c[2 * r])
    # Z2: prod over odd l of 2 sinh g_l U_{h-1}(c_l); sinh g_l sinh g_{2n-l} = c_l^2 - 1.
    Z2 = mpmath.mpf(1)
    for r in range(n):
        Z2 *= 2 * _cheb_U(h - 1, c[2 * r + 1])
    for l in range(1, n, 2):                    # odd l < n pairs with 2n - l
        Z2 *= c[l] * c[l] - 1
    # Z4: l = 0 and l = n unpaired, even l in (0, n) paired with 2n - l.
    Z4 = mpmath.mpf(1)
    for r in range(n):
        Z4 *= 2 * _cheb_U(h - 1, c[2 * r])
    for l in range(2, n, 2):
        Z4 *= c[l] * c[l] - 1
    e4 = y * y                                  # e^{4K}
    sh0_shn = (e4 + 1 / e4 - (t * t + 1 / (t * t))) / 4
    Z4 *= sh0_shn
    pref = (y - 1 / y) ** (N // 2)              # (2 sinh 2K)^{N/2}
    Z = pref * (Z1 + Z2 + Z3 + Z4) / 2
    return Z / y ** N


def _point(args):
    L, k, P, dps = args
    with mpmath.workdps(dps):
        z = mpmath.expjpi(2 * (k + mpmath.mpf(1) / 2) / P)
        return _partition_scaled(L, 1 / mpmath.sqrt(z))


def _coefficient(args):
    full, e, P, dps = args
    with mpmath.workdps(dps):
        w = mpmath.expjpi(-2 * mpmath.mpf(e) / P)
        acc = mpmath.mpc(0)
        for k in range(P - 1, -1, -1):
            acc = acc * w + full[k]
        acc *= mpmath.expjpi(-mpmath.mpf(e) / P)          # w^(1/2)
        return int(mpmath.nint(acc.real / P))


def exact_gE(L: int, workers: int = 1) -> list[int]:
    """Exact g(e), e = 0..N (E = 4e - 2N), as Python integers; even L >= 4."""
    if L < 4 or L % 2:
        raise ValueError("exact_gE needs even L >= 4")
    N = L * L
    P = N + 1
    dps = int(N * math.log10(2)) + 40
    # Real coefficients: P(conj z) = conj P(z), so half of the points suffice;
    # z_{P-1-k} = conj(z_k) because (P-1-k+1/2) = P - (k+1/2).
    half = P // 2 + 1
    pts = [(L, k, P, dps) for k in range(half)]
    if workers > 1:
        import multiprocessing as mp
        with mp.get_context("spawn").Pool(workers) as pool:
            vals = pool.map(_point, pts, chunksize=max(1, half // (8 * workers)))
    else:
        vals = [_point(a) for a in pts]
    with mpmath.workdps(dps):
        full = [None] * P
        for k in range(half):
            full[k] = vals[k]
            full[P - 1 - k] = mpmath.conj(vals[k])
    es = [(full, e, P, dps) for e in range(N // 2 + 1)]
    if workers > 1:
        import multiprocessing as mp
        with mp.get_context("spawn").Pool(workers) as pool:
            lo = pool.map(_coefficient, es, chunksize=max(1, len(es) // (8 * workers)))
    else:
        lo = [_coefficient(a) for a in es]
    return lo + lo[:P - len(lo)][::-1]


def exact_lngE(L: int, workers: int = 1) -> list[float]:
    """ln g(e) in double precision (-inf where g(e) = 0)."""
    out = []
    for g in exact_gE(L, workers):
        out.append(-math.inf if g == 0 else _log_int(g))
    return out


def _log_int(v: int) -> float:
    """Natural log of a positive Python integer of any size, to double precision."""
    b = v.bit_length()
    if b <= 1000:
        return math.log(v)
    sh = b - 900
    return math.log(v >> sh) + sh * math.log(2.0)
