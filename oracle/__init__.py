"""CPU oracle for two-dimensional replica-exchange Wang-Landau sampling.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
package.  The product (``paper_1508_02748_gb300``) never does, and this
package never imports the product: the two share no code.

The arithmetic lives in plain C (``philox.c``, ``rewl_oracle.c``,
``exact.c``) compiled with gcc into ``_build/liboracle.so`` on first use (or
by :func:`build`); this module only marshals arguments.  ``exact_ge.py``
holds the closed-form energy density of states (Kaufman's torus partition
function expanded exactly, as Beale did).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "liboracle.so")
_SRCS = ["philox.c", "rewl_oracle.c", "exact.c"]
_lock = threading.Lock()
_lib = None

OK, E_INVALID, E_UNREACHABLE, E_JOIN = 0, -1, -4, -7
JOIN_MARGINAL, JOIN_PER_SLICE = 0, 1


def build(force: bool = False) -> str:
    """Compile the oracle's C sources with gcc (no FMA contraction)."""
    os.makedirs(_BUILD, exist_ok=True)
    srcs = [os.path.join(_HERE, s) for s in _SRCS]
    stale = force or not os.path.exists(_LIB) or any(
        os.path.getmtime(s) > os.path.getmtime(_LIB) for s in srcs)
    if stale:
        tmp = _LIB + f".{os.getpid()}.tmp"
        cmd = ["gcc", "-O2", "-std=gnu11", "-fPIC", "-shared", "-ffp-contract=off",
               "-fno-fast-math", "-o", tmp] + srcs + ["-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = ctypes.CDLL(_LIB)
            P, u64, i32, i64, dbl = ctypes.c_void_p, ctypes.c_uint64, ctypes.c_int, ctypes.c_int64, ctypes.c_double
            L.orc_philox4x32_10.argtypes = [P, P, P]
            L.orc_philox_batch.argtypes = [u64, P, P, P]
            L.orc_create.restype = P
            L.orc_create.argtypes = [i32, i32, i32, dbl, dbl, i32, dbl, dbl, dbl, dbl, u64, i32, u64,
                                     P, u64, ctypes.POINTER(ctypes.c_int)]
            L.orc_destroy.argtypes = [P]
            L.orc_sweep.argtypes = [P, u64]
            L.orc_exchange.argtypes = [P]
            L.orc_check_advance.argtypes = [P]
            L.orc_check_advance.restype = i32
            L.orc_run_cycles.argtypes = [P, u64]
            L.orc_info.argtypes = [P, P]
            L.orc_lnf.argtypes = [P]
            L.orc_lnf.restype = dbl
            L.orc_windows.argtypes = [P, P]
            L.orc_walkers.argtypes = [P, P, P]
            L.orc_tables.argtypes = [P, P, P, P]
            L.orc_set_tables.argtypes = [P, P, P]
            L.orc_join.argtypes = [P, P, P, P]
            L.orc_join.restype = i32
            L.orc_join_excl.argtypes = [P, i32, P, P, P]
            L.orc_join_excl.restype = i32
            L.orc_join_rule.argtypes = [P, i32, i32, P, P, P]
            L.orc_join_rule.restype = i32
            L.orc_marginal_e.argtypes = [i32, P, P]
            L.orc_rel_diff.argtypes = [ctypes.c_size_t, P, P, P]
            L.orc_bin_possible.argtypes = [i32, i32, i32]
            L.orc_bin_possible.restype = i32
            L.orc_enum_gEM.argtypes = [i32, P]
            L.orc_enum_gEM.restype = i32
            L.orc_tm_gEM.argtypes = [i32, P]
            L.orc_tm_gEM.restype = i32
            _lib = L
    return _lib


def _ptr(a: np.ndarray) -> int:
    return a.ctypes.data


# ------------------------------------------------------------------ Philox ---

def philox4x32_10(counters: np.ndarray, key) -> np.ndarray:
    """Philox4x32-10 of each row of ``counters`` (n x 4 uint32) under ``key``."""
    c = np.ascontiguousarray(counters, dtype=np.uint32).reshape(-1, 4)
    k = np.ascontiguousarray(np.asarray(key, dtype=np.uint32).reshape(2))
    out = np.empty_like(c)
    lib().orc_philox_batch(c.shape[0], _ptr(c), _ptr(k), _ptr(out))
    return out


# ------------------------------------------------------------ exact tables ---

def enumerate_gEM(L: int) -> np.ndarray:
    """Exact g(e, m) by visiting all 2^(L*L) configurations (L <= 5)."""
    N = L * L
    out = np.zeros((N + 1, N + 1), dtype=np.uint64)
    rc = lib().orc_enum_gEM(L, _ptr(out))
    if rc:
        raise ValueError(f"enumeration unsupported for L={L}")
    return out


def transfer_gEM(L: int) -> np.ndarray:
    """Exact g(e, m) by the site-by-site transfer matrix (L <= 8)."""
    N = L * L
    out = np.zeros((N + 1, N + 1), dtype=np.uint64)
    rc = lib().orc_tm_gEM(L, _ptr(out))
    if rc:
        raise ValueError(f"transfer matrix failed for L={L} (rc={rc})")
    return out


def bin_possible(L: int, e: int, m: int) -> bool:
    return bool(lib().orc_bin_possible(L, e, m))


# --------------------------------------------------------------- REWL run ---

@dataclass
class OracleConfig:
    L: int
    n_win_E: int = 1
    n_win_M: int = 1
    overlap_E: float = 0.75
    overlap_M: float = 0.75
    walkers_per_window: int = 1
    lnf_init: float = 1.0
    lnf_final: float = 1e-6
    lnf_factor: float = 0.5
    flatness: float = 0.8
    exchange_interval: int = 10000
    check_every: int = 1
    seed: int = 1
    drive_budget: int = 10_000_000


class OracleREWL:
    """Serial REWL run (``rewl_oracle.c``), one object per run."""

    def __init__(self, cfg: OracleConfig, init_spins: np.ndarray | None = None):
        self.cfg = cfg
        L = lib()
        err = ctypes.c_int(0)
        sp = None
        if init_spins is not None:
            sp = np.ascontiguousarray(init_spins, dtype=np.uint8)
            self._spins_keep = sp
        h = L.orc_create(cfg.L, cfg.n_win_E, cfg.n_win_M, cfg.overlap_E, cfg.overlap_M,
                         cfg.walkers_per_window, cfg.lnf_init, cfg.lnf_final, cfg.lnf_factor,
                         cfg.flatness, cfg.exchange_interval, cfg.check_every, cfg.seed,
                         None if sp is None else _ptr(sp), cfg.drive_budget, ctypes.byref(err))
        if not h:
            raise RuntimeError(f"oracle create failed: code {err.value}")
        self._h = h
        self.N = cfg.L * cfg.L

    def close(self):
        if getattr(self, "_h", None):
            lib().orc_destroy(self._h)
            self._h = None

    def __del__(self):
        self.close()

    # -- steps
    def sweep(self, n: int):
        lib().orc_sweep(self._h, n)

    def exchange(self):
        lib().orc_exchange(self._h)

    def check_advance(self) -> bool:
        return bool(lib().orc_check_advance(self._h))

    def run_cycles(self, n: int):
        lib().orc_run_cycles(self._h, n)

    # -- state
    def info(self) -> dict:
        a = np.zeros(11, dtype=np.int64)
        lib().orc_info(self._h, _ptr(a))
        keys = ["L", "N", "nwin", "nwalk", "cycle", "xstep", "iter", "done", "table_bins",
                "exch_attempt", "exch_accept"]
        d = dict(zip(keys, (int(x) for x in a)))
        d["lnf"] = float(lib().orc_lnf(self._h))
        return d

    def windows(self) -> np.ndarray:
        n = self.info()["nwin"]
        out = np.zeros((n, 5), dtype=np.int32)
        lib().orc_windows(self._h, _ptr(out))
        return out

    def walkers(self):
        inf = self.info()
        st = np.zeros((inf["nwalk"], 4), dtype=np.int64)
        sp = np.zeros((inf["nwalk"], self.N), dtype=np.uint8)
        lib().orc_walkers(self._h, _ptr(st), _ptr(sp))
        return st, sp

    def tables(self):
        inf = self.info()
        lng = np.zeros(inf["table_bins"], dtype=np.float64)
        H = np.zeros(inf["table_bins"], dtype=np.int32)
        toff = np.zeros(inf["nwalk"] + 1, dtype=np.int64)
        lib().orc_tables(self._h, _ptr(lng), _ptr(H), _ptr(toff))
        return lng, H, toff

    def set_tables(self, lng: np.ndarray, H: np.ndarray):
        lng = np.ascontiguousarray(lng, dtype=np.float64)
        H = np.ascontiguousarray(H, dtype=np.int32)
        lib().orc_set_tables(self._h, _ptr(lng), _ptr(H))

    def join(self, rule: int = JOIN_MARGINAL):
        """Merged, joined and normalised ln g(e, m) plus the matching points;
        rule JOIN_MARGINAL rescales each piece by one constant (the marginals'
        difference at the matching point), JOIN_PER_SLICE each M slice (each E
        slice in the join along M) by its own difference there."""
        B = self.N + 1
        c = self.cfg
        out = np.zeros((B, B), dtype=np.float64)
        em = np.zeros(max(1, c.n_win_M * max(1, c.n_win_E - 1)), dtype=np.int32)
        mm = np.zeros(max(1, c.n_win_M - 1), dtype=np.int32)
        rc = lib().orc_join_rule(self._h, -1, rule, _ptr(out), _ptr(em), _ptr(mm))
        if rc:
            raise RuntimeError(f"oracle join failed: code {rc}")
        return out, em, mm


def jackknife_replicates(run: "OracleREWL", marginal: bool = False) -> np.ndarray:
    """Replicate k (k = 0..W-1) is the join of the run without walker k of
    every window (the jackknife over walkers of Sec. 2); marginal=True gives
    each replicate's E marginal (Eq. 3) instead of the joint table."""
    B = run.N + 1
    c = run.cfg
    em = np.zeros(max(1, c.n_win_M * max(1, c.n_win_E - 1)), dtype=np.int32)
    mm = np.zeros(max(1, c.n_win_M - 1), dtype=np.int32)
    reps = []
    for k in range(c.walkers_per_window):
        out = np.zeros((B, B), dtype=np.float64)
        rc = lib().orc_join_excl(run._h, k, _ptr(out), _ptr(em), _ptr(mm))
        if rc:
            raise RuntimeError(f"oracle jackknife join failed: code {rc}")
        reps.append(marginal_e(out) if marginal else out)
    return np.stack(reps)


def jackknife_stats(R: np.ndarray):
    """Jackknife mean and error of replicates R (W x ...): mean = average,
    error = sqrt((W-1)/W * sum_k (R_k - mean)^2), per entry; entries missing
    from any replicate get mean -inf and error NaN.  Differences are taken
    from the first replicate to keep the sums small."""
    W = R.shape[0]
    ok = np.all(np.isfinite(R), axis=0)
    ref = np.where(ok, R[0], 0.0)
    d = np.where(ok, R - ref, 0.0)
    s1 = d.sum(axis=0)
    s2 = (d * d).sum(axis=0)
    mean = np.where(ok, ref + s1 / W, -np.inf)
    var = (W - 1) / W * (s2 - s1 * s1 / W)
    err = np.where(ok, np.sqrt(np.maximum(var, 0.0)), np.nan)
    return mean, err


def jackknife(run: "OracleREWL", marginal: bool = False):
    """Jackknife mean and error of ln g over the walkers of each window."""
    return jackknife_stats(jackknife_replicates(run, marginal))


def marginal_e(lng_joint: np.ndarray) -> np.ndarray:
    """Eq. 3 on a joined table: ln sum_m g(e, m)."""
    B = lng_joint.shape[0]
    a = np.ascontiguousarray(lng_joint, dtype=np.float64)
    out = np.zeros(B, dtype=np.float64)
    lib().orc_marginal_e(B - 1, _ptr(a), _ptr(out))
    return out


def relative_difference(lng_a: np.ndarray, lng_b: np.ndarray) -> np.ndarray:
    """Eq. 5 per bin from two ln g tables of the same shape: |g_a - g_b| / gbar,
    gbar = (g_a + g_b) / 2; 2 where one table is empty, NaN where both are."""
    a = np.ascontiguousarray(lng_a, dtype=np.float64)
    b = np.ascontiguousarray(lng_b, dtype=np.float64)
    if a.shape != b.shape:
        raise ValueError("tables differ in shape")
    out = np.empty_like(a)
    lib().orc_rel_diff(a.size, _ptr(a), _ptr(b), _ptr(out))
    return out
