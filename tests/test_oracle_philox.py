"""Pins the oracle's Philox4x32-10 against an independent implementation.

The independent implementation is PyTorch's header-only ``at::Philox4_32``
(ATen/core/PhiloxRNGEngine.h), compiled here and run; its engine maps
(seed, subsequence, offset) to key = seed and counter = (offset_lo, offset_hi,
subsequence_lo, subsequence_hi), and its first four outputs are the four
words of one Philox4x32-10 block.
"""
import os
import subprocess
import tempfile

import numpy as np
import pytest

import oracle

SRC = r"""
#include <ATen/core/PhiloxRNGEngine.h>
#include <cstdio>
#include <cstdint>
int main(int argc, char** argv) {
  FILE* f = std::fopen(argv[1], "rb");
  FILE* g = std::fopen(argv[2], "wb");
  uint32_t rec[6];
  while (std::fread(rec, 4, 6, f) == 6) {
    uint64_t seed = (uint64_t)rec[4] | ((uint64_t)rec[5] << 32);
    uint64_t sub = (uint64_t)rec[2] | ((uint64_t)rec[3] << 32);
    uint64_t off = (uint64_t)rec[0] | ((uint64_t)rec[1] << 32);
    at::Philox4_32 e(seed, sub, off);
    uint32_t o[4];
    for (int i = 0; i < 4; ++i) o[i] = e();
    std::fwrite(o, 4, 4, g);
  }
  std::fclose(f); std::fclose(g);
  return 0;
}
"""


def _torch_include():
    import torch
    inc = os.path.join(os.path.dirname(torch.__file__), "include")
    if not os.path.exists(os.path.join(inc, "ATen", "core", "PhiloxRNGEngine.h")):
        pytest.skip("PyTorch Philox header not found")
    return inc


def test_philox_matches_independent_implementation():
    inc = _torch_include()
    rng = np.random.default_rng(20150811)
    n = 20000
    ctr = rng.integers(0, 2**32, size=(n, 4), dtype=np.uint64).astype(np.uint32)
    ctr[:100] = 0                         # edge counters: zeros and all-ones
    ctr[100:200] = 0xFFFFFFFF
    keys = rng.integers(0, 2**32, size=(n, 2), dtype=np.uint64).astype(np.uint32)
    keys[:50] = 0
    keys[100:150] = 0xFFFFFFFF
    with tempfile.TemporaryDirectory() as d:
        exe = os.path.join(d, "ph")
        src = os.path.join(d, "ph.cpp")
        open(src, "w").write(SRC)
        subprocess.run(["g++", "-std=c++17", "-O1", "-I", inc, "-o", exe, src], check=True)
        rec = np.concatenate([ctr, keys], axis=1).astype(np.uint32)
        inp, outp = os.path.join(d, "in.bin"), os.path.join(d, "out.bin")
        rec.tofile(inp)
        subprocess.run([exe, inp, outp], check=True)
        ref = np.fromfile(outp, dtype=np.uint32).reshape(n, 4)
    got = np.concatenate([oracle.philox4x32_10(ctr[i:i + 1], keys[i]) for i in range(n)])
    assert np.array_equal(got, ref)


def test_philox_avalanche_and_uniformity():
    # Property checks that a wrong round (dropped XOR, swapped halves) fails:
    # adjacent counters give unrelated outputs, and bits are balanced.
    n = 1 << 16
    c = np.zeros((n, 4), dtype=np.uint32)
    c[:, 0] = np.arange(n, dtype=np.uint32)
    out = oracle.philox4x32_10(c, [12345, 678])
    bits = np.unpackbits(out.view(np.uint8)).reshape(n, -1)
    frac = bits.mean(axis=0)
    assert np.all(np.abs(frac - 0.5) < 0.02)
    flips = np.unpackbits((out[1:] ^ out[:-1]).view(np.uint8)).reshape(n - 1, -1).sum(axis=1)
    assert abs(flips.mean() - 64.0) < 0.5
