"""The autotuner's search space (host logic, no GPU): every tiling choice it
may time, including where the warp sampler keeps the tables and a small
lattice, offered only where both placements exist."""
import paper_1508_02748_gb300 as P
from paper_1508_02748_gb300 import workloads
from paper_1508_02748_gb300.autotune import candidates


def _cfg(w):
    return P.Config.from_workload(w)


def test_small_windows_offer_both_table_and_lattice_placements():
    c = candidates(_cfg(workloads.REWL_L8))
    warp = [x for x in c if x[0] == P.SAMPLER_WARP]
    assert {x[1] for x in warp} == {8, 16, 32}
    assert {x[2] for x in warp} == {1, 2, 4}
    # 3 x 3 windows of 44 x 44 bins at L = 8: staging fits for every group size, N = 64 fits a register
    assert {(x[3], x[4]) for x in warp} == {(P.TABLES_AUTO, P.LATTICE_AUTO), (P.TABLES_AUTO, P.LATTICE_SHARED),
                                            (P.TABLES_GLOBAL, P.LATTICE_AUTO), (P.TABLES_GLOBAL, P.LATTICE_SHARED)}
    assert len(warp) == 3 * 3 * 4
    thread = [x for x in c if x[0] == P.SAMPLER_THREAD]
    assert len(thread) == 3 and all(x[1] == 0 and x[3] == P.TABLES_AUTO and x[4] == P.LATTICE_AUTO for x in thread)


def test_large_windows_have_one_placement():
    # L = 32: 126,576 bins per window (1 MB of S and H) never fit; N = 1024 never fits a register
    c = candidates(_cfg(workloads.REWL_L32), samplers=(P.SAMPLER_WARP,))
    assert len(c) == 9
    assert all(x[3] == P.TABLES_AUTO and x[4] == P.LATTICE_AUTO for x in c)


def test_lattice_placement_follows_the_lattice_size():
    # L = 12 (N = 144): the register lattice does not exist, so no shared-lattice alternative is timed
    cfg = P.Config(L=12, n_win_E=2, n_win_M=2, walkers_per_window=2)
    assert all(x[4] == P.LATTICE_AUTO for x in candidates(cfg))
    # L = 4 (N = 16, one 17 x 17 window): both lattice and both table placements
    assert {(x[3], x[4]) for x in candidates(_cfg(workloads.SERIAL_L4), samplers=(P.SAMPLER_WARP,))} == {
        (P.TABLES_AUTO, P.LATTICE_AUTO), (P.TABLES_AUTO, P.LATTICE_SHARED),
        (P.TABLES_GLOBAL, P.LATTICE_AUTO), (P.TABLES_GLOBAL, P.LATTICE_SHARED)}
