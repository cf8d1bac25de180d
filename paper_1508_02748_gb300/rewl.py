"""Python binding of librewl (include/rewl.h): argument marshalling only.

Every step of the method runs in the library's CUDA kernels; PyTorch provides
the device workspace (one uint8 tensor) and the stream.  There is no CPU
fallback: constructing :class:`REWL` without the built library or without a
CUDA device raises.
"""
from __future__ import annotations

import ctypes
import os
import threading
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "librewl.so")

REWL_OK = 0
ERRORS = {-1: "INVALID", -2: "CUDA", -3: "TIMEOUT", -4: "UNREACHABLE", -5: "OVERFLOW",
          -6: "BUDGET", -7: "JOIN", -8: "CAPACITY"}
FP64, F32X2, F32 = 0, 1, 2
PART_SAMPLE, PART_REST, PART_SAMPLE_PLAIN = 1, 2, 4
SAMPLER_WARP, SAMPLER_THREAD = 0, 1
LNG_JOINED, LNG_MARGINAL_E = 0, 1
TABLES_AUTO, TABLES_GLOBAL, TABLES_STAGED = 0, 1, 2
LATTICE_AUTO, LATTICE_REGISTER, LATTICE_SHARED = 0, 1, 2
JOIN_MARGINAL, JOIN_PER_SLICE = 0, 0x100   # rescaling rule of a join step, OR-ed into `what`


class REWLError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"REWL_E_{ERRORS.get(code, code)}: {msg}")
        self.code = code


class rewl_config(ctypes.Structure):
    _fields_ = [("struct_size", ctypes.c_uint32), ("L", ctypes.c_int32),
                ("n_win_E", ctypes.c_int32), ("n_win_M", ctypes.c_int32),
                ("overlap_E", ctypes.c_double), ("overlap_M", ctypes.c_double),
                ("walkers_per_window", ctypes.c_int32), ("precision", ctypes.c_int32),
                ("lnf_init", ctypes.c_double), ("lnf_final", ctypes.c_double),
                ("lnf_factor", ctypes.c_double), ("flatness", ctypes.c_double),
                ("exchange_interval", ctypes.c_uint64), ("check_every", ctypes.c_int32),
                ("walkers_per_block", ctypes.c_int32), ("sampler", ctypes.c_int32), ("lanes_per_walker", ctypes.c_int32),
                ("seed", ctypes.c_uint64),
                ("drive_budget", ctypes.c_uint64), ("table_mode", ctypes.c_int32), ("lattice_mode", ctypes.c_int32)]


class rewl_status(ctypes.Structure):
    _fields_ = [("iteration", ctypes.c_int32), ("done", ctypes.c_int32), ("lnf", ctypes.c_double),
                ("cycles", ctypes.c_uint64), ("trials", ctypes.c_uint64),
                ("exch_attempts", ctypes.c_uint64), ("exch_accepts", ctypes.c_uint64),
                ("n_flat", ctypes.c_int32), ("n_walkers", ctypes.c_int32),
                ("error", ctypes.c_int32), ("reserved", ctypes.c_int32)]


class rewl_peaks(ctypes.Structure):
    _fields_ = [("lop3_ops_per_s", ctypes.c_double), ("iadd_ops_per_s", ctypes.c_double),
                ("imad_ops_per_s", ctypes.c_double), ("ffma_ops_per_s", ctypes.c_double),
                ("dep_iadd_cycles", ctypes.c_double), ("smem_bytes_per_s", ctypes.c_double),
                ("l2_bytes_per_s", ctypes.c_double), ("sms", ctypes.c_int32), ("reserved", ctypes.c_int32)]


# Every symbol include/rewl.h declares, with its ctypes signature.
_P = ctypes.c_void_p
SIGNATURES = {
    "rewl_workspace_size": (ctypes.c_int, [ctypes.POINTER(rewl_config), ctypes.POINTER(ctypes.c_size_t)]),
    "rewl_create": (ctypes.c_int, [ctypes.POINTER(rewl_config), _P, _P, ctypes.c_size_t, _P, ctypes.POINTER(_P)]),
    "rewl_run_cycles": (ctypes.c_int, [_P, ctypes.c_uint64, ctypes.POINTER(rewl_status)]),
    "rewl_run_cycles_plain": (ctypes.c_int, [_P, ctypes.c_uint64, ctypes.POINTER(rewl_status)]),
    "rewl_run_iteration": (ctypes.c_int, [_P, ctypes.c_uint64, ctypes.POINTER(rewl_status)]),
    "rewl_enqueue_cycle": (ctypes.c_int, [_P, ctypes.c_int]),
    "rewl_sweep": (ctypes.c_int, [_P, ctypes.c_uint64]),
    "rewl_exchange": (ctypes.c_int, [_P]),
    "rewl_check": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_int32)]),
    "rewl_get_status": (ctypes.c_int, [_P, ctypes.POINTER(rewl_status)]),
    "rewl_get_windows": (ctypes.c_int, [_P, _P, ctypes.c_size_t]),
    "rewl_get_walkers": (ctypes.c_int, [_P, _P, _P]),
    "rewl_get_tables": (ctypes.c_int, [_P, _P, _P, ctypes.c_size_t]),
    "rewl_set_tables": (ctypes.c_int, [_P, _P, _P, ctypes.c_size_t]),
    "rewl_tables_digest": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_uint64)]),
    "rewl_get_lng": (ctypes.c_int, [_P, ctypes.c_int, _P, ctypes.c_size_t, ctypes.POINTER(ctypes.c_size_t), _P, _P]),
    "rewl_get_lng_jackknife": (ctypes.c_int, [_P, ctypes.c_int, _P, _P, ctypes.c_size_t,
                                              ctypes.POINTER(ctypes.c_size_t)]),
    "rewl_save": (ctypes.c_int, [_P, ctypes.c_char_p]),
    "rewl_checkpoint_config": (ctypes.c_int, [ctypes.c_char_p, ctypes.POINTER(rewl_config)]),
    "rewl_load": (ctypes.c_int, [ctypes.c_char_p, _P, ctypes.c_size_t, _P, ctypes.POINTER(_P)]),
    "rewl_last_error": (ctypes.c_char_p, [_P]),
    "rewl_destroy": (ctypes.c_int, [_P]),
    "rewl_philox": (ctypes.c_int, [_P, _P, _P, ctypes.c_uint64, _P]),
    "rewl_relative_difference": (ctypes.c_int, [_P, _P, _P, ctypes.c_uint64, _P]),
    "rewl_batch_create": (ctypes.c_int, [_P, ctypes.c_int, _P, ctypes.POINTER(_P)]),
    "rewl_batch_cycles_per_launch": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_uint64)]),
    "rewl_batch_run_cycles": (ctypes.c_int, [_P, ctypes.c_uint64]),
    "rewl_batch_enqueue": (ctypes.c_int, [_P]),
    "rewl_batch_destroy": (ctypes.c_int, [_P]),
    "rewl_join_noalloc": (ctypes.c_int, [ctypes.POINTER(rewl_config), _P, _P, _P, _P]),
    "rewl_noalloc_last_error": (ctypes.c_char_p, []),
    "rewl_measure_peaks": (ctypes.c_int, [_P, ctypes.c_size_t, _P, ctypes.POINTER(rewl_peaks)]),
}

_lib = None
_lock = threading.Lock()


def load_library(path: str | None = None):
    """Loads librewl.so (built by ``paper_1508_02748_gb300.build``); raises if absent."""
    global _lib
    with _lock:
        if _lib is None:
            p = path or LIB_PATH
            if not os.path.exists(p):
                raise RuntimeError(f"librewl.so not built ({p}); run "
                                   "`python -m paper_1508_02748_gb300.build`")
            lib = ctypes.CDLL(p)
            for name, (res, args) in SIGNATURES.items():
                f = getattr(lib, name)
                f.restype = res
                f.argtypes = args
            _lib = lib
    return _lib


def _check(rc: int, handle=None):
    if rc != REWL_OK:
        msg = load_library().rewl_last_error(handle)
        raise REWLError(rc, msg.decode() if msg else "")


@dataclass
class Config:
    L: int
    n_win_E: int = 1
    n_win_M: int = 1
    overlap_E: float = 0.75
    overlap_M: float = 0.75
    walkers_per_window: int = 1
    precision: int = FP64
    lnf_init: float = 1.0
    lnf_final: float = 1e-6
    lnf_factor: float = 0.5
    flatness: float = 0.8
    exchange_interval: int = 10000
    check_every: int = 1
    walkers_per_block: int = 0
    sampler: int = 0
    lanes_per_walker: int = 0
    seed: int = 1
    drive_budget: int = 10_000_000
    table_mode: int = 0
    lattice_mode: int = 0

    def to_c(self) -> rewl_config:
        c = rewl_config()
        c.struct_size = ctypes.sizeof(rewl_config)
        for name, _ in rewl_config._fields_[1:]:
            setattr(c, name, getattr(self, name))
        return c

    @classmethod
    def from_workload(cls, w, replicate: int = 0, **kw) -> "Config":
        d = dict(L=w.L, n_win_E=w.n_win_E, n_win_M=w.n_win_M, overlap_E=w.overlap_E,
                 overlap_M=w.overlap_M, walkers_per_window=w.walkers_per_window,
                 lnf_init=w.lnf_init, lnf_final=w.lnf_final, lnf_factor=w.lnf_factor,
                 flatness=w.flatness, exchange_interval=w.exchange_interval,
                 check_every=w.check_every, seed=w.seed(replicate))
        d.update(kw)
        return cls(**d)


def _status_dict(s: rewl_status) -> dict:
    return {name: getattr(s, name) for name, _ in rewl_status._fields_ if name != "reserved"}


class REWL:
    """One REWL run on a CUDA device (handle of include/rewl.h)."""

    def __init__(self, cfg: Config, init_spins: np.ndarray | None = None, device: str = "cuda:0",
                 stream=None):
        import torch
        lib = load_library()
        if not torch.cuda.is_available():
            raise RuntimeError("REWL needs a CUDA device")
        self.cfg = cfg
        self._c = cfg.to_c()
        self.device = torch.device(device)
        nbytes = ctypes.c_size_t(0)
        _check(lib.rewl_workspace_size(ctypes.byref(self._c), ctypes.byref(nbytes)))
        self.workspace_bytes = int(nbytes.value)
        self.workspace = torch.empty(self.workspace_bytes, dtype=torch.uint8, device=self.device)
        self.stream = stream if stream is not None else torch.cuda.Stream(device=self.device)
        sp = None
        if init_spins is not None:
            sp = np.ascontiguousarray(init_spins, dtype=np.uint8)
        h = ctypes.c_void_p(0)
        with torch.cuda.device(self.device):
            rc = lib.rewl_create(ctypes.byref(self._c), None if sp is None else sp.ctypes.data,
                                 ctypes.c_void_p(self.workspace.data_ptr()), self.workspace_bytes,
                                 ctypes.c_void_p(self.stream.cuda_stream), ctypes.byref(h))
        _check(rc, None)
        self._h = h
        self.N = cfg.L * cfg.L
        self.n_windows = cfg.n_win_E * cfg.n_win_M
        self.n_walkers = self.n_windows * cfg.walkers_per_window

    # ---------------------------------------------------------------- run --
    def run_cycles(self, n: int) -> dict:
        s = rewl_status()
        _check(load_library().rewl_run_cycles(self._h, n, ctypes.byref(s)), self._h)
        return _status_dict(s)

    def run_cycles_plain(self, n: int) -> dict:
        """The same cycles in the plain form: one launch per walker, no graph."""
        s = rewl_status()
        _check(load_library().rewl_run_cycles_plain(self._h, n, ctypes.byref(s)), self._h)
        return _status_dict(s)

    def run_iteration(self, max_cycles: int) -> tuple[bool, dict]:
        """Runs until an iteration ends; (False, status) if max_cycles ran first."""
        s = rewl_status()
        rc = load_library().rewl_run_iteration(self._h, max_cycles, ctypes.byref(s))
        if rc == -6:
            return False, _status_dict(s)
        _check(rc, self._h)
        return True, _status_dict(s)

    def enqueue_cycle(self, parts: int = PART_SAMPLE | PART_REST):
        """Queues one cycle (or its SAMPLE / REST part) on self.stream without waiting."""
        _check(load_library().rewl_enqueue_cycle(self._h, parts), self._h)

    def sweep(self, n_trials: int):
        _check(load_library().rewl_sweep(self._h, n_trials), self._h)

    def exchange(self):
        _check(load_library().rewl_exchange(self._h), self._h)

    def check(self) -> bool:
        f = ctypes.c_int32(0)
        _check(load_library().rewl_check(self._h, ctypes.byref(f)), self._h)
        return bool(f.value)

    def status(self) -> dict:
        s = rewl_status()
        _check(load_library().rewl_get_status(self._h, ctypes.byref(s)), self._h)
        return _status_dict(s)

    # -------------------------------------------------------------- state --
    def windows(self) -> np.ndarray:
        out = np.zeros((self.n_windows, 5), dtype=np.int32)
        _check(load_library().rewl_get_windows(self._h, out.ctypes.data, out.size), self._h)
        return out

    def walkers(self, spins: bool = True):
        st = np.zeros((self.n_walkers, 4), dtype=np.int64)
        sp = np.zeros((self.n_walkers, self.N), dtype=np.uint8) if spins else None
        _check(load_library().rewl_get_walkers(self._h, st.ctypes.data,
                                               None if sp is None else sp.ctypes.data), self._h)
        return st, sp

    def _bins(self) -> int:
        w = self.windows()[0]
        return int((w[1] - w[0] + 1) * (w[3] - w[2] + 1))

    def tables(self):
        n = self.n_walkers * self._bins()
        lng = np.zeros(n, dtype=np.float64)
        H = np.zeros(n, dtype=np.int32)
        _check(load_library().rewl_get_tables(self._h, lng.ctypes.data, H.ctypes.data, n), self._h)
        return lng, H

    def set_tables(self, lng: np.ndarray, H: np.ndarray):
        lng = np.ascontiguousarray(lng, dtype=np.float64)
        H = np.ascontiguousarray(H, dtype=np.int32)
        _check(load_library().rewl_set_tables(self._h, lng.ctypes.data, H.ctypes.data, lng.size), self._h)

    def digest(self) -> int:
        """Order-independent digest of every walker's ln g and H (rewl_tables_digest)."""
        d = ctypes.c_uint64(0)
        _check(load_library().rewl_tables_digest(self._h, ctypes.byref(d)), self._h)
        return int(d.value)

    def lng(self, what: int = LNG_JOINED, matches: bool = False, rule: int = JOIN_MARGINAL):
        """Joined ln g (or its E marginal); rule JOIN_PER_SLICE rescales each
        slice at the matching point instead of each piece as a whole."""
        B = self.N + 1
        n = B * B if what == LNG_JOINED else B
        what = what | rule
        out = np.zeros(n, dtype=np.float64)
        need = ctypes.c_size_t(0)
        nE, nM = self.cfg.n_win_E, self.cfg.n_win_M
        em = np.zeros(max(1, nM * max(1, nE - 1)), dtype=np.int32)
        mm = np.zeros(max(1, nM - 1), dtype=np.int32)
        _check(load_library().rewl_get_lng(self._h, what, out.ctypes.data, n, ctypes.byref(need),
                                           em.ctypes.data, mm.ctypes.data), self._h)
        out = out.reshape(B, B) if n == B * B else out
        return (out, em, mm) if matches else out

    def jackknife(self, what: int = LNG_JOINED, rule: int = JOIN_MARGINAL):
        """Jackknife mean and error of ln g over the walkers of each window."""
        B = self.N + 1
        n = B * B if what == LNG_JOINED else B
        joined = what == LNG_JOINED
        what = what | rule
        mean = np.zeros(n, dtype=np.float64)
        err = np.zeros(n, dtype=np.float64)
        need = ctypes.c_size_t(0)
        _check(load_library().rewl_get_lng_jackknife(self._h, what, mean.ctypes.data, err.ctypes.data, n,
                                                     ctypes.byref(need)), self._h)
        if joined:
            return mean.reshape(B, B), err.reshape(B, B)
        return mean, err

    def save(self, path: str):
        """Writes a checkpoint of the whole run (rewl_save)."""
        _check(load_library().rewl_save(self._h, os.fsencode(path)), self._h)

    @classmethod
    def load(cls, path: str, device: str = "cuda:0", stream=None) -> "REWL":
        """Restores a run from a checkpoint into a new workspace (rewl_load)."""
        import torch
        lib = load_library()
        c = rewl_config()
        _check(lib.rewl_checkpoint_config(os.fsencode(path), ctypes.byref(c)))
        kw = {name: getattr(c, name) for name, _ in rewl_config._fields_[1:]}
        self = cls.__new__(cls)
        self.cfg = Config(**kw)
        self._c = c
        self.device = torch.device(device)
        nbytes = ctypes.c_size_t(0)
        _check(lib.rewl_workspace_size(ctypes.byref(c), ctypes.byref(nbytes)))
        self.workspace_bytes = int(nbytes.value)
        self.workspace = torch.empty(self.workspace_bytes, dtype=torch.uint8, device=self.device)
        self.stream = stream if stream is not None else torch.cuda.Stream(device=self.device)
        h = ctypes.c_void_p(0)
        with torch.cuda.device(self.device):
            rc = lib.rewl_load(os.fsencode(path), ctypes.c_void_p(self.workspace.data_ptr()), self.workspace_bytes,
                               ctypes.c_void_p(self.stream.cuda_stream), ctypes.byref(h))
        _check(rc, None)
        self._h = h
        self.N = self.cfg.L * self.cfg.L
        self.n_windows = self.cfg.n_win_E * self.cfg.n_win_M
        self.n_walkers = self.n_windows * self.cfg.walkers_per_window
        return self

    def close(self):
        if getattr(self, "_h", None):
            load_library().rewl_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def philox(counters, key) -> "object":
    """Device Philox4x32-10 of n counters (torch uint32-compatible int32 tensor n x 4 on CUDA)."""
    import torch
    c = counters.contiguous()
    out = torch.empty_like(c)
    k = np.ascontiguousarray(np.asarray(key, dtype=np.uint32).reshape(2))
    s = torch.cuda.current_stream(c.device)
    _check(load_library().rewl_philox(ctypes.c_void_p(c.data_ptr()), k.ctypes.data,
                                      ctypes.c_void_p(out.data_ptr()), c.shape[0],
                                      ctypes.c_void_p(s.cuda_stream)))
    return out


def relative_difference(lng_a, lng_b) -> "object":
    """Eq. 5 per bin on the device: |g_a - g_b| / ((g_a + g_b) / 2) from two
    float64 CUDA tensors of ln g of the same shape (2 where one is empty,
    NaN where both are)."""
    import torch
    a = lng_a.contiguous()
    b = lng_b.contiguous()
    if a.shape != b.shape or a.dtype != torch.float64 or b.dtype != torch.float64 or not a.is_cuda or b.device != a.device:
        raise ValueError("two float64 CUDA tensors of one shape on one device expected")
    out = torch.empty_like(a)
    s = torch.cuda.current_stream(a.device)
    _check(load_library().rewl_relative_difference(ctypes.c_void_p(a.data_ptr()), ctypes.c_void_p(b.data_ptr()),
                                                   ctypes.c_void_p(out.data_ptr()), a.numel(),
                                                   ctypes.c_void_p(s.cuda_stream)))
    return out


def measure_peaks(device: str = "cuda:0") -> dict:
    """Issue and bandwidth rates of the GPU (rewl_measure_peaks), with a
    64 MiB torch scratch buffer; per second of device time."""
    import torch
    dev = torch.device(device)
    scratch = torch.empty((64 << 20) + 4096, dtype=torch.uint8, device=dev)
    out = rewl_peaks()
    s = torch.cuda.current_stream(dev)
    with torch.cuda.device(dev):
        _check(load_library().rewl_measure_peaks(ctypes.c_void_p(scratch.data_ptr()), scratch.numel(),
                                                 ctypes.c_void_p(s.cuda_stream), ctypes.byref(out)))
    return {name: getattr(out, name) for name, _ in rewl_peaks._fields_ if name != "reserved"}


class Batch:
    """Several REWL runs advanced together by one CUDA graph (rewl_batch_*).

    The runs sample concurrently on the GPU; each keeps exactly the trajectory
    it would have alone.  Keep the runs alive while the batch exists and do
    not drive them individually meanwhile."""

    def __init__(self, runs, stream=None):
        import torch
        self.runs = list(runs)
        lib = load_library()
        self.stream = stream if stream is not None else torch.cuda.Stream(device=self.runs[0].device)
        arr = (ctypes.c_void_p * len(self.runs))(*[r._h.value for r in self.runs])
        h = ctypes.c_void_p(0)
        rc = lib.rewl_batch_create(ctypes.cast(arr, ctypes.c_void_p), len(self.runs),
                                   ctypes.c_void_p(self.stream.cuda_stream), ctypes.byref(h))
        _check(rc, None)
        self._h = h
        k = ctypes.c_uint64(0)
        _check(lib.rewl_batch_cycles_per_launch(self._h, ctypes.byref(k)))
        self.k = int(k.value)

    def run_cycles(self, n: int):
        _check(load_library().rewl_batch_run_cycles(self._h, n), None)

    def enqueue(self):
        """Queues one graph launch (self.k cycles of every run) without waiting."""
        _check(load_library().rewl_batch_enqueue(self._h), None)

    def close(self):
        if getattr(self, "_h", None):
            load_library().rewl_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
