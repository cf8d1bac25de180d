"""Writes the stored exact tables under tests/golden/ from the oracle alone.

    python tests/golden/make_golden.py [L ...]

gEM_L8.txt   exact joint g(e, m) of the 8 x 8 torus (transfer matrix, exact.c),
             (N+1) rows of (N+1) integers, e = (E + 2N)/4, m = (M + N)/2.
lngE_L<L>.txt  ln g(e) of the L x L torus from Kaufman's partition function
             expanded exactly (exact_ge.py, Beale's method), one value per e,
             -inf where g(e) = 0.
"""
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402
from oracle.exact_ge import exact_lngE  # noqa: E402


def write_gEM_L8():
    g = oracle.transfer_gEM(8)
    with open(os.path.join(HERE, "gEM_L8.txt"), "w") as f:
        for row in g:
            f.write(" ".join(str(int(v)) for v in row) + "\n")


def write_lngE(L):
    v = exact_lngE(L, workers=os.cpu_count() or 1)
    with open(os.path.join(HERE, f"lngE_L{L}.txt"), "w") as f:
        for x in v:
            f.write(("-inf" if x == float("-inf") else repr(float(x))) + "\n")


if __name__ == "__main__":
    # worker processes re-import this module: keep the work under this guard
    targets = sys.argv[1:] or ["8", "16", "32"]
    for t in targets:
        L = int(t)
        if L == 8:
            write_gEM_L8()
            write_lngE(8)
        else:
            write_lngE(L)
        print("wrote", L, flush=True)
