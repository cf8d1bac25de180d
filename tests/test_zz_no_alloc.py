"""rewl_join_noalloc: the join for callers that cannot allocate device memory.

Some callers of this library may not call cudaMalloc: their device memory is
all owned by an external allocator (a framework's caching pool), or their
memory budget is fixed up front.  They own their inputs and output but cannot
provide the join's working memory; rewl_join_noalloc takes that memory from a
fixed device array in the library.  This file checks, through the C ABI, that
it returns what rewl_get_lng returns for the same tables and what the CPU
oracle's join returns for the same run, on two calls in a row (the array
keeps the previous call's contents), and that oversize geometries are
refused.  It is collected last so that a failure here comes after every
other test has run.
"""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1508_02748_gb300 as P
    from paper_1508_02748_gb300 import build
    build.build()
    return P


def _noalloc_join(P, run, lng, H):
    import torch
    lib = P.load_library()
    B = run.N + 1
    d_lng = torch.from_numpy(np.ascontiguousarray(lng)).cuda()
    d_H = torch.from_numpy(np.ascontiguousarray(H)).cuda()
    d_out = torch.full((B * B,), float("nan"), dtype=torch.float64, device="cuda")
    torch.cuda.synchronize()
    c = run.cfg.to_c()
    rc = lib.rewl_join_noalloc(ctypes.byref(c), ctypes.c_void_p(d_lng.data_ptr()),
                               ctypes.c_void_p(d_H.data_ptr()), ctypes.c_void_p(d_out.data_ptr()), None)
    assert rc == 0, lib.rewl_noalloc_last_error()
    return d_out.cpu().numpy().reshape(B, B)


def test_noalloc_join_matches_get_lng_and_oracle_twice(P):
    import oracle
    kw = dict(L=8, n_win_E=3, n_win_M=3, walkers_per_window=4, exchange_interval=10000, seed=20152813)
    run = P.REWL(P.Config(**kw))
    orc = oracle.OracleREWL(oracle.OracleConfig(**kw))
    for cycles in (120, 60):                       # two calls in a row on changed tables
        run.run_cycles(cycles)
        orc.run_cycles(cycles)
        lng, H = run.tables()
        ref = run.lng()                            # rewl_get_lng(REWL_LNG_JOINED)
        got = _noalloc_join(P, run, lng, H)
        fin = np.isfinite(ref)
        assert np.array_equal(np.isfinite(got), fin)
        np.testing.assert_allclose(got[fin], ref[fin], rtol=1e-12, atol=1e-9)
        Jo, _, _ = orc.join()                      # the same run's join on the CPU oracle
        assert np.array_equal(np.isfinite(Jo), fin)
        np.testing.assert_allclose(got[fin], Jo[fin], rtol=1e-12, atol=1e-9)


def test_noalloc_join_refuses_oversize_geometry(P):
    lib = P.load_library()
    big = P.Config(L=32, n_win_E=16, n_win_M=4, walkers_per_window=32).to_c()
    rc = lib.rewl_join_noalloc(ctypes.byref(big), ctypes.c_void_p(8), ctypes.c_void_p(8),
                               ctypes.c_void_p(8), None)
    assert rc == -8
    assert b"scratch" in lib.rewl_noalloc_last_error()
