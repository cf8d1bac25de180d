"""Benchmark: Wang-Landau spin-flip trials/s of two-dimensional REWL on one GB300.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--workload NAME] [--impl reference]

One step is one cycle of the whole sampling path on the synthetic workload:
every walker does `exchange_interval` single-spin-flip trials (Eq. 1 and the
update of Sec. 2), one replica-exchange sweep (Eq. 2) and the flatness check /
iteration advance (Sec. 2-3).  The default workload is batched 2D REWL of the
32 x 32 periodic Ising model: 16 x 4 (E, M) windows at 75% overlap, 32 walkers
per window (2048 walkers), exchange every 10^4 trials per walker, FP64 ln g.

Timed state: the run first advances through its own cycles, untimed, for
--warm-seconds of wall time (or restores a saved run with --checkpoint), so
the timed cycles are not the first cycles of iteration 0; the line states the
iteration and ln f they ran at.

value    trials/s with the run resident in HBM, CUDA events on the run's stream
         around each step, L2 flushed (256 MiB write) between steps;
plain    the same cycles in the plain one-walker-per-launch form (one
         single-thread launch per walker over 4 streams, host-driven exchange
         and check, no graph), trials/s over --plain-cycles cycles;
e2e      the same metric through the C ABI with host buffers: creation from
         host spin bytes (host->device), K synchronous steps each reading the
         run status back (device->host), and the joined ln g(E,M) copied to
         host memory, wall clock;
roofline the sampling kernel (the dominant one) against the integer-logic
         issue rate measured on this GPU (rewl_measure_peaks): algorithmic
         integer/float operations per trial x trials per launch / mean launch
         time from its own CUDA events in the timed steps; the memory side
         (algorithmic bytes per trial against the measured shared-memory
         bandwidth) beside it;
cpu_baseline the CPU oracle (test infrastructure) on every host core: one
         process per core, each running a bounded sample of the workload.
With --impl reference the CPU oracle is the timed implementation.
Under torchrun with N > 1 ranks each rank runs an independent replica of the
run on its own GPU (the method's windows share one GPU; replicas only).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_1508_02748_gb300 import workloads  # noqa: E402

METRIC = "WL spin-flip trials/s & time-to-ln f=1e-6 at fixed ln g error, batched vs plain"
# Algorithmic operations per trial (integer and float ALU), counted from the
# method: half a Philox4x32-10 call (10 rounds x 10 ops / 2 trials = 50), the
# float log of u (~15), site/row/column and 5 spin-bit extractions with the
# periodic neighbours (~25), bin move, window test and table index (~12),
# the screened acceptance (~10) and the bookkeeping of ln g / H (~8).
OPS_PER_TRIAL = 120

# Algorithmic bytes per trial to shared memory / L1 (the method's own
# traffic): lattice 12 B read + 4 B written on an accepted flip, table 24 B
# (ln g of the proposed bin 8 B, ln g and H of the current bin read and
# written 16 B).
BYTES_PER_TRIAL = 40

# Counters of the sampling kernel from ncu captures (their summaries are in
# the profiles directory), per launch in the benchmark's launch
# configuration, keyed by workload, kernel, table format, lanes per walker,
# table and lattice placement (as configured; 0 = automatic) and the hash of
# the kernel sources (any other case reports null):
# dram_bytes = dram__bytes_read.sum + dram__bytes_write.sum of one launch;
# warp_inst_per_trial = smsp__inst_executed.sum / trials of one launch.
TRAFFIC_SOURCES = ("paper_1508_02748_gb300/csrc/rewl_sweep_tree.cu", "paper_1508_02748_gb300/csrc/rewl_tab.cuh",
                   "paper_1508_02748_gb300/csrc/rewl_internal.cuh")
PROFILE = {
    # L = 32, 16 x 4 windows, 32 walkers each, 32 lanes per walker: DRAM bytes from a one-pass capture
    # of the full workload after 512 warm-up cycles; instructions per trial from the full capture of
    # the same kernel at 16 walkers per window
    ("rewl_L32_16x4_w32", "k_sweep_tree", "fp64", 32, 0, 0, "3eb3a9b855675b6e"): {"dram_bytes": 143_505_408,
                                                               "warp_inst_per_trial": 53.22},
    # L = 8, 3 x 3 windows, 4 walkers each, 32 lanes per walker (tables staged in shared memory)
    ("rewl_L8_3x3_w4", "k_sweep_tree", "fp64", 32, 0, 0, "3eb3a9b855675b6e"): {"dram_bytes": 608_256,
                                                            "warp_inst_per_trial": 60.50},
}


def sources_hash() -> str:
    import hashlib
    h = hashlib.sha256()
    for f in TRAFFIC_SOURCES:
        with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]
ALU_LANES_PER_SM = 128          # 32-bit lanes per SM (4 partitions x 32)
FALLBACK_SMS = 152


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--workload", default=workloads.REWL_L32.name,
                    choices=sorted(workloads.ALL) + [workloads.BATCH_NAME])
    ap.add_argument("--impl", default="gpu", choices=["gpu", "reference"])
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-peaks", action="store_true", help="skip the peak microbenchmarks (derived ALU peak)")
    ap.add_argument("--no-others", action="store_true",
                    help="skip the short timings of the L = 64 workload and the uneven batch added to the line")
    ap.add_argument("--no-time-to", action="store_true",
                    help="skip the time-to-ln f <= 1e-6 run of the L = 8 workload added to the line")
    ap.add_argument("--warm-seconds", type=float, default=20.0,
                    help="untimed cycles of the run itself before the timed ones (wall seconds)")
    ap.add_argument("--warm-cycles", type=int, default=None,
                    help="untimed cycles of the run itself before the timed ones (a cycle count; replaces "
                         "--warm-seconds, for profiler captures that skip to a fixed launch)")
    ap.add_argument("--checkpoint", default=None, help="time a run restored from this checkpoint (rewl_save)")
    ap.add_argument("--plain-cycles", type=int, default=1,
                    help="cycles of the plain one-walker-per-launch form timed after the batched ones (0: skip)")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU-oracle baseline (profiling runs)")
    ap.add_argument("--no-autotune", action="store_true", help="use the default tiling")
    ap.add_argument("--lanes", type=int, default=None, choices=[8, 16, 32],
                    help="warp sampler: lanes per walker (fixes the tiling, no autotuning)")
    ap.add_argument("--wpb", type=int, default=None,
                    help="warps (warp sampler) or threads (thread sampler) per block (fixes the tiling)")
    ap.add_argument("--tables", choices=["auto", "global", "staged"], default="auto",
                    help="with --lanes/--wpb: where the warp sampler keeps S and H")
    ap.add_argument("--lattice", choices=["auto", "register", "shared"], default="auto",
                    help="with --lanes/--wpb: where the warp sampler keeps a lattice of N <= 64 sites")
    ap.add_argument("--lnf-final", type=float, default=None, help="override the workload's final ln f")
    ap.add_argument("--walkers-per-window", type=int, default=None,
                    help="override the workload's walkers per window (small cases for profiler captures)")
    ap.add_argument("--max-seconds", type=float, default=300.0,
                    help="--time-to: stop (and report the iteration reached) after this wall time")
    ap.add_argument("--precision", default=None, choices=["fp64", "f32x2", "f32"],
                    help="ln g tables (default: the workload's: fp64)")
    ap.add_argument("--sampler", default="auto", choices=["auto", "warp", "thread"],
                    help="auto: the autotuner picks the sampler too (with --no-autotune: warp)")
    ap.add_argument("--replicate", type=int, default=0,
                    help="seed replicate of the run (seed 20150811 + 1000 workload id + replicate + rank)")
    ap.add_argument("--replicates", type=int, default=1,
                    help="--impl reference --time-to: seeds run at once, one process each")
    ap.add_argument("--form", default="batched", choices=["batched", "plain"],
                    help="plain: each walker's trials as a launch of their own (one thread, 4 streams), "
                         "exchange and check launched from the host, no graph; same trajectory")
    ap.add_argument("--experiment", default=None, choices=["eq5", "precision"],
                    help="eq5: serial WL vs the paper's REWL split at L = 8, Eq. 5 relative difference; "
                         "precision: the L = 64 precision study (FP64, f32x2, plain float)")
    ap.add_argument("--late-cycles", type=int, default=8, help="--experiment precision: cycles from the late state")
    ap.add_argument("--time-to", action="store_true",
                    help="run the workload to its final ln f and report the wall time and ln g error")
    return ap.parse_args()


def reduce_max_ms(local_ms: float, world: int, device) -> float:
    """Max over ranks of a per-rank time (the contract's max-over-ranks clock)."""
    if world <= 1:
        return local_ms
    import torch
    import torch.distributed as dist
    t = torch.tensor([local_ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def aggregate_rate(trials_per_step: int, steps: int, world: int, total_ms: float) -> float:
    """Whole-job trials/s: every rank runs an independent replica of the
    workload (same size, its own seed), so the job does world x the trials
    in the slowest rank's time."""
    return trials_per_step * steps * world / (total_ms / 1e3)


def replica_seed_index(rank: int) -> int:
    """Replicate index of a rank's run (its seed is 20150811 + 1000 id + this)."""
    return rank


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


# ------------------------------------------------------------------ clocks --

class ClockSampler:
    """nvidia-smi clock / throttle-reason samples while the timed region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.lines: list[str] = []
        self.proc = None
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# -------------------------------------------------------------- CPU oracle --

def cpu_model() -> str:
    """The host CPU's model name (lscpu, else /proc/cpuinfo, else the machine type)."""
    import platform
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for ln in out.splitlines():
            if ln.lower().startswith("model name"):
                return ln.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    try:
        for ln in open("/proc/cpuinfo"):
            if ln.lower().startswith("model name"):
                return ln.split(":", 1)[1].strip()
    except OSError:
        pass
    return platform.machine()


def host_cores() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def oracle_sample_walkers(w, table_budget_bytes: int = 256 << 20) -> int:
    """Walkers per window of the CPU sample: the workload's geometry with at
    most `table_budget_bytes` of oracle tables per process (12 bytes per bin
    and walker), at least one walker per window."""
    import math as _m
    B = w.N + 1

    def width(n, o):
        return B if n == 1 else min(B, _m.ceil(B / (1 + (n - 1) * (1 - o))))
    per_walker = width(w.n_win_E, w.overlap_E) * width(w.n_win_M, w.overlap_M) * 12
    nwin = w.n_win_E * w.n_win_M
    return max(1, min(w.walkers_per_window, table_budget_bytes // (per_walker * nwin)))


def _oracle_cfg(w, wpw: int, seed: int):
    import oracle
    return oracle.OracleConfig(L=w.L, n_win_E=w.n_win_E, n_win_M=w.n_win_M, overlap_E=w.overlap_E,
                               overlap_M=w.overlap_M, walkers_per_window=wpw,
                               lnf_init=w.lnf_init, lnf_final=w.lnf_final, lnf_factor=w.lnf_factor,
                               flatness=w.flatness, exchange_interval=w.exchange_interval,
                               check_every=w.check_every, seed=seed, drive_budget=10**8)


def _oracle_worker(task):
    """One host process of the CPU oracle: `warm` untimed cycles, then timed
    cycles until `steps` cycles or `seconds` of wall time have run; returns
    (trials timed, seconds timed, cycles timed)."""
    w, wpw, seed, warm, steps, seconds = task
    sys.path.insert(0, ROOT)
    import oracle
    r = oracle.OracleREWL(_oracle_cfg(w, wpw, seed))
    live = int(r.windows()[:, 4].sum()) * wpw
    for _ in range(warm):
        r.run_cycles(1)
    cyc = 0
    t0 = time.perf_counter()
    while True:
        r.run_cycles(1)
        cyc += 1
        dt = time.perf_counter() - t0
        if (steps and cyc >= steps) or (not steps and dt >= seconds):
            break
    r.close()
    return cyc * w.exchange_interval * live, dt, cyc


def oracle_all_cores(w, seconds: float = 0.0, steps: int = 0, warm: int = 0) -> dict:
    """The CPU oracle on every host core: one process per core (spawned, so
    safe after CUDA work), each an independent run of the bounded sample
    (the workload's geometry, oracle_sample_walkers walkers per window, its
    own seed); trials/s = all processes' trials / the slowest one's time."""
    import multiprocessing as mp
    cores = host_cores()
    wpw = oracle_sample_walkers(w)
    tasks = [(w, wpw, w.seed(0) + 7919 * (k + 1), warm, steps, seconds) for k in range(cores)]
    with mp.get_context("spawn").Pool(cores) as pool:
        res = pool.map(_oracle_worker, tasks)
    trials = sum(r[0] for r in res)
    t = max(r[1] for r in res)
    cyc = res[0][2]
    return {"value": trials / t, "unit": "trials/s", "cores": cores, "kind": "oracle",
            "cpu_model": cpu_model(), "seconds": t, "cycles_per_process": cyc,
            "sample": f"{cores} processes, each an independent run of {w.name} with {wpw} walker(s) per "
                      f"window (same geometry, {w.exchange_interval} trials per walker per cycle); "
                      f"{trials} trials in {t:.1f} s"}


def run_reference(args, w):
    """The reference arm: the CPU oracle on every host core.  One step is one
    cycle of the bounded sample in each process."""
    rank, world, _ = dist_env()
    if rank != 0:
        return
    cb = oracle_all_cores(w, steps=args.steps, warm=args.warmup)
    value = cb["value"]
    line = {"metric": METRIC, "value": value, "unit": "trials/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": cb["seconds"] / args.steps * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "impl": "reference",
            "config": _config_dict(w, "none (CPU)"),
            "cpu_baseline": cb,
            "e2e": {"value": value, "unit": "trials/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def _oracle_time_to_worker(task):
    """One host process: the oracle run of workload `w` with seed `seed` from
    creation to its final ln f (or `seconds` of wall time), polled every 64
    checks like the GPU run; returns its time, cycles and E-marginal error."""
    w, seed, seconds = task
    sys.path.insert(0, ROOT)
    import numpy as np
    import oracle
    r = oracle.OracleREWL(_oracle_cfg(w, w.walkers_per_window, seed))
    t0 = time.perf_counter()
    capped = False
    while not r.info()["done"]:
        r.run_cycles(64 * w.check_every)
        if time.perf_counter() - t0 > seconds:
            capped = True
            break
    dt = time.perf_counter() - t0
    inf = r.info()
    eps = None
    ex = exact_lngE(w.L)
    if ex is None and w.L <= 6:                # small lattices: g(E) by enumeration
        g = oracle.enumerate_gEM(w.L).sum(axis=1)
        with np.errstate(divide="ignore"):
            ex = np.where(g > 0, np.log(np.where(g > 0, g, 1)), -np.inf)
    if ex is not None and not capped:
        J, _, _ = r.join()
        mE = oracle.marginal_e(J)
        ok = np.isfinite(ex) & (ex > 0) & np.isfinite(mE)
        eps = float(np.mean(np.abs(mE[ok] - ex[ok]) / ex[ok]))
    r.close()
    return {"seed": seed, "seconds": dt, "capped": capped, "cycles": inf["cycle"], "iterations": inf["iter"],
            "mean_eps_E_marginal_vs_exact": eps}


def run_reference_time_to(args, w):
    """The CPU oracle's time to the workload's final ln f: `--replicates` seeds
    (replicate, replicate + 1, ...), each run to done on one core in its own
    spawned process, all at once."""
    import multiprocessing as mp
    rank, _, _ = dist_env()
    if rank != 0:
        return
    n = max(1, args.replicates)
    tasks = [(w, w.seed(args.replicate + k), args.max_seconds) for k in range(n)]
    with mp.get_context("spawn").Pool(min(n, host_cores())) as pool:
        runs = pool.map(_oracle_time_to_worker, tasks)
    secs = [r["seconds"] for r in runs]
    line = {"metric": "time-to-ln f<=%g" % w.lnf_final, "value": sum(secs) / len(secs), "unit": "s",
            "higher_is_better": False, "impl": "reference", "dtype": "f64", "data": "synthetic",
            "config": _config_dict(w, "none (CPU)"), "cpu_model": cpu_model(),
            "cores_per_run": 1, "runs": runs}
    print(json.dumps(line), flush=True)


def _sampler_name(code: int) -> str:
    return "warp" if code == 0 else "thread"


def _config_dict(w, l2: str, precision: str = "fp64", sampler: str = "oracle") -> dict:
    return {"workload": w.name, "L": w.L, "windows": f"{w.n_win_E}x{w.n_win_M}",
            "overlap": w.overlap_E, "walkers_per_window": w.walkers_per_window,
            "walkers": w.n_walkers, "exchange_interval": w.exchange_interval,
            "check_every": w.check_every, "ln_g": precision, "sampler": sampler,
            "step": "one cycle: sample + exchange + check", "l2": l2}


def exact_lngE(L: int):
    """Exact ln g(E) stored under tests/golden (written from the closed form)."""
    import numpy as np
    path = os.path.join(ROOT, "tests", "golden", f"lngE_L{L}.txt")
    if not os.path.exists(path):
        return None
    return np.loadtxt(path)


def exact_lngEM(L: int):
    """Exact ln g(e, m) stored under tests/golden (transfer matrix), or None."""
    import numpy as np
    path = os.path.join(ROOT, "tests", "golden", f"gEM_L{L}.txt")
    if not os.path.exists(path):
        return None
    g = np.loadtxt(path, dtype=np.float64)
    with np.errstate(divide="ignore"):
        return np.where(g > 0, np.log(np.where(g > 0, g, 1.0)), -np.inf)


# ------------------------------------------------------------------- GPU ----

def run_eq5(args):
    """Sec. 3's comparison: serial WL over the whole (E, M) range with one
    walker against REWL in the paper's split (3 E-windows, 50% overlap, 3
    walkers per window), both to the same final ln f; the relative
    difference of Eq. 5 between the two joint tables is computed on the
    device.  Each run is capped at --max-seconds."""
    import numpy as np
    import torch

    import paper_1508_02748_gb300 as P
    from paper_1508_02748_gb300 import build as pkg_build

    pkg_build.build()
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    lnf_final = args.lnf_final if args.lnf_final is not None else 1e-6
    prec = {"fp64": P.FP64, "f32x2": P.F32X2, "f32": P.F32}[args.precision]
    out = {}
    tables = {}
    for key, w in (("serial_wl", workloads.SERIAL_L8), ("rewl", workloads.PAPER_L8)):
        w = w.with_(lnf_final=lnf_final)
        run = P.REWL(P.Config.from_workload(w, replicate=args.replicate, drive_budget=10**8, precision=prec),
                     device=str(dev))
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        st = run.status()
        capped = False
        while not st["done"]:
            st = run.run_cycles(64)
            if time.perf_counter() - t0 > args.max_seconds:
                capped = True
                break
        elapsed = time.perf_counter() - t0
        tables[key] = run.lng()
        out[key] = {"workload": w.name, "seed": run.cfg.seed, "seconds": elapsed, "capped": capped,
                    "iterations": st["iteration"], "lnf": st["lnf"], "trials_per_walker": st["trials"],
                    "walkers": st["n_walkers"]}
        run.close()
    d = P.relative_difference(torch.from_numpy(tables["serial_wl"]).to(dev),
                              torch.from_numpy(tables["rewl"]).to(dev)).cpu().numpy()
    both = np.isfinite(tables["serial_wl"]) & np.isfinite(tables["rewl"])
    B = d.shape[0]
    e_idx = np.repeat(np.arange(B)[:, None], B, axis=1)
    band = {}
    for name, lo, hi in (("low_E_third", 0, B // 3), ("middle_third", B // 3, 2 * B // 3),
                         ("high_E_third", 2 * B // 3, B)):
        sel = both & (e_idx >= lo) & (e_idx < hi)
        band[name] = float(d[sel].mean()) if sel.any() else None
    ex = exact_lngEM(8)
    vs_exact = {}
    if ex is not None:
        occ = np.isfinite(ex)
        for key in tables:
            de = P.relative_difference(torch.from_numpy(tables[key]).to(dev),
                                       torch.from_numpy(ex).to(dev)).cpu().numpy()
            vs_exact[key] = {"mean": float(np.nanmean(de[occ])), "max": float(np.nanmax(de[occ])),
                             "support_equal": bool(np.array_equal(np.isfinite(tables[key]), occ))}
    line = {"metric": "eq5_relative_difference_serial_wl_vs_rewl", "value": float(d[both].mean()),
            "unit": "mean over bins occupied in both tables", "higher_is_better": False, "n_gpus": 1,
            "dtype": {"fp64": "f64", "f32x2": "f32x2", "f32": "f32"}[args.precision], "data": "synthetic",
            "config": {"workload": "eq5_L8_serial_vs_paper_split", "L": 8, "lnf_final": lnf_final,
                       "max_seconds_per_run": args.max_seconds},
            "max": float(d[both].max()), "median": float(np.median(d[both])), "bins": int(both.sum()),
            "bins_in_one_table_only": int((np.isfinite(tables["serial_wl"]) ^ np.isfinite(tables["rewl"])).sum()),
            "mean_by_energy": band, "vs_exact_joint": vs_exact, "runs": out}
    print(json.dumps(line), flush=True)


def warm_run(run, seconds: float, chunk: int, cycles: int | None = None) -> dict:
    """Advances a run through its own cycles (untimed): exactly `cycles`
    cycles when given, else whole check blocks for `seconds` of wall time;
    returns where it got to."""
    t0 = time.perf_counter()
    st = run.status()
    if cycles is not None:
        if cycles > 0:
            st = run.run_cycles(cycles)
        seconds = 0
    while seconds > 0 and not st["done"] and time.perf_counter() - t0 < seconds:
        st = run.run_cycles(chunk)
    return {"warm_seconds": time.perf_counter() - t0, "cycles_before_timing": st["cycles"],
            "iteration": st["iteration"], "lnf": st["lnf"], "done": st["done"]}


def run_gpu(args, w):
    import numpy as np
    import torch

    import paper_1508_02748_gb300 as P
    from paper_1508_02748_gb300 import build as pkg_build

    rank, world, local = dist_env()
    pkg_build.build()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)

    def barrier():
        if world > 1:
            import torch.distributed as dist
            dist.barrier()

    prec = {"fp64": P.FP64, "f32x2": P.F32X2, "f32": P.F32}[args.precision]
    smp = {"auto": P.SAMPLER_WARP, "warp": P.SAMPLER_WARP, "thread": P.SAMPLER_THREAD}[args.sampler]
    if args.lnf_final is not None:
        w = w.with_(lnf_final=args.lnf_final)
    if args.walkers_per_window is not None:
        w = w.with_(walkers_per_window=args.walkers_per_window,
                    name=f"{w.name.rsplit('_w', 1)[0]}_w{args.walkers_per_window}")
    cfg = P.Config.from_workload(w, replicate=args.replicate + replica_seed_index(rank), drive_budget=10**8,
                                 precision=prec,
                                 sampler=smp)
    plain = args.form == "plain"
    if args.lanes is not None or args.wpb is not None:
        import dataclasses
        cfg = dataclasses.replace(cfg, lanes_per_walker=args.lanes or 0, walkers_per_block=args.wpb or 0,
                                  table_mode={"auto": P.TABLES_AUTO, "global": P.TABLES_GLOBAL,
                                              "staged": P.TABLES_STAGED}[args.tables],
                                  lattice_mode={"auto": P.LATTICE_AUTO, "register": P.LATTICE_REGISTER,
                                                "shared": P.LATTICE_SHARED}[args.lattice])
    elif not args.no_autotune and not plain:
        from paper_1508_02748_gb300.autotune import autotune
        allowed = (P.SAMPLER_WARP, P.SAMPLER_THREAD) if args.sampler == "auto" else (smp,)
        cfg = autotune(cfg, device=str(dev), samplers=allowed)
    if args.time_to:
        return run_time_to(args, w, cfg, dev)
    peaks = None if args.no_peaks else P.measure_peaks(str(dev))

    # the timed state: a restored run, or the run after its own warm-up cycles
    if args.checkpoint:
        run = P.REWL.load(args.checkpoint, device=str(dev))
        st0 = run.status()
        state = {"checkpoint": os.path.basename(args.checkpoint), "cycles_before_timing": st0["cycles"],
                 "iteration": st0["iteration"], "lnf": st0["lnf"], "done": st0["done"]}
    else:
        run = P.REWL(cfg, device=str(dev))
        state = warm_run(run, args.warm_seconds, 16 * w.check_every, args.warm_cycles)
    s = run.stream
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    nwalk_active = run.status()["n_walkers"]
    trials_per_step = w.exchange_interval * nwalk_active
    sample_part = P.PART_SAMPLE_PLAIN if plain else P.PART_SAMPLE
    with torch.cuda.stream(s):
        for _ in range(args.warmup):
            run.enqueue_cycle(sample_part | P.PART_REST)
    s.synchronize()
    cyc0 = run.status()["cycles"]

    K = args.steps
    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(K)]
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    barrier()
    torch.cuda.synchronize()
    launches = 0
    with torch.cuda.stream(s):
        for k in range(K):
            flush.zero_()                                # L2 flush, outside the step's events
            ev[k][0].record(s)
            run.enqueue_cycle(sample_part)
            ev[k][1].record(s)
            run.enqueue_cycle(P.PART_REST)
            ev[k][2].record(s)
            check = ((cyc0 + k + 1) % w.check_every) == 0
            launches += (nwalk_active if plain else 1) + 2 + (2 if check else 0)
    s.synchronize()
    torch.cuda.synchronize()
    barrier()
    clk = clocks.stop()
    step_ms = [ev[k][0].elapsed_time(ev[k][2]) for k in range(K)]
    sweep_ms = [ev[k][0].elapsed_time(ev[k][1]) for k in range(K)]
    total_ms = reduce_max_ms(sum(step_ms), world, dev)
    st = run.status()
    value = aggregate_rate(trials_per_step, K, world, total_ms)

    # the plain one-walker-per-launch FP64 form on the same run, continuing its chain
    plain_line = None
    if not plain and args.plain_cycles > 0:
        with torch.cuda.stream(s):
            run.enqueue_cycle(P.PART_SAMPLE_PLAIN | P.PART_REST)      # untimed: creates its streams
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(s)
            for _ in range(args.plain_cycles):
                run.enqueue_cycle(P.PART_SAMPLE_PLAIN | P.PART_REST)
            e1.record(s)
        s.synchronize()
        pms = e0.elapsed_time(e1)
        plain_line = {"value": trials_per_step * args.plain_cycles / (pms / 1e3), "unit": "trials/s",
                      "cycles": args.plain_cycles, "ms_per_step": pms / args.plain_cycles,
                      "form": "one single-thread launch of k_sweep_thread per walker over 4 streams, "
                              "host-driven exchange and check, no graph; " + args.precision}

    # roofline of the sampling kernel: the method's operations per launch
    # against the measured integer-logic issue rate, and its algorithmic
    # bytes against the measured shared-memory bandwidth
    sm_count = torch.cuda.get_device_properties(dev).multi_processor_count
    mhz = clk.get("sm_mhz") or 1920.0
    sweep_s = statistics.mean(sweep_ms) / 1e3
    achieved = OPS_PER_TRIAL * trials_per_step / sweep_s
    kname = "k_sweep_tree" if cfg.sampler == P.SAMPLER_WARP and not plain and prec != P.F32 else "k_sweep_thread"
    prof = PROFILE.get((w.name, kname, args.precision, cfg.lanes_per_walker, cfg.table_mode, cfg.lattice_mode,
                        sources_hash())) if not plain else None
    traffic = prof["dram_bytes"] if prof else None
    if peaks:
        peak_ops = peaks["lop3_ops_per_s"]
        basis = (f"measured on this GPU by rewl_measure_peaks: independent lop3.b32 issue "
                 f"{peaks['lop3_ops_per_s'] / 1e12:.2f} Tops/s (integer-logic pipe), iadd "
                 f"{peaks['iadd_ops_per_s'] / 1e12:.2f}, imad {peaks['imad_ops_per_s'] / 1e12:.2f}, ffma "
                 f"{peaks['ffma_ops_per_s'] / 1e12:.2f} Tops/s, at median SM clock {mhz:.0f} MHz")
    else:
        peak_ops = sm_count * ALU_LANES_PER_SM * mhz * 1e6
        basis = f"{sm_count} SMs x {ALU_LANES_PER_SM} lanes x median SM clock {mhz:.0f} MHz (derived)"
    roof = {"bound": "alu", "achieved": achieved / 1e12, "peak": peak_ops / 1e12, "unit": "Tops/s",
            "frac": achieved / peak_ops, "traffic": traffic,
            "traffic_unit": "DRAM bytes per launch (ncu dram__bytes_read.sum + dram__bytes_write.sum)",
            "kernel": kname + (" (one launch per walker, 4 streams)" if plain else ""),
            "kernel_ms_mean": sweep_s * 1e3,
            "kernel_share_of_step": sum(sweep_ms) / total_ms,
            "ops_per_trial": OPS_PER_TRIAL,
            "peak_basis": basis}
    if peaks and prof:
        # instruction issue: the kernel's measured instructions per trial at the
        # live trial rate against one warp instruction per cycle per SM
        # sub-partition (the independent-add stream of rewl_measure_peaks)
        lane_inst = prof["warp_inst_per_trial"] * 32
        roof["issue"] = {"lane_instructions_per_trial": lane_inst, "algorithmic_ops_per_trial": OPS_PER_TRIAL,
                         "achieved": lane_inst * trials_per_step / sweep_s / 1e12,
                         "peak": peaks["iadd_ops_per_s"] / 1e12, "unit": "Tlane-instructions/s",
                         "frac": lane_inst * trials_per_step / sweep_s / peaks["iadd_ops_per_s"]}
    if peaks:
        mem_achieved = BYTES_PER_TRIAL * trials_per_step / sweep_s
        roof["memory"] = {"bound": "shared memory / L1", "bytes_per_trial": BYTES_PER_TRIAL,
                          "achieved": mem_achieved / 1e9, "peak": peaks["smem_bytes_per_s"] / 1e9,
                          "unit": "GB/s", "frac": mem_achieved / peaks["smem_bytes_per_s"],
                          "l2_peak_gbs": peaks["l2_bytes_per_s"] / 1e9}

    # end to end through the C ABI with host buffers: the run created from
    # host spin bytes, K synchronous steps each reading the run status back,
    # then every walker's state (e, m, trials, flat verdict) copied to host
    # memory as the result (the joined table needs every window overlap
    # visited, which a run this young may not have)
    e2e = None
    if not args.no_e2e:
        rng = np.random.default_rng(w.seed(rank) + 7)
        host_spins = rng.integers(0, 2, size=(w.n_walkers, w.N), dtype=np.uint8)
        pinned = torch.from_numpy(host_spins).pin_memory().numpy()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        run2 = P.REWL(cfg, init_spins=pinned, device=str(dev), stream=s)
        for _ in range(K):
            (run2.run_cycles_plain if plain else run2.run_cycles)(1)
        states, _ = run2.walkers(spins=False)
        t1 = time.perf_counter()
        e2e_trials = trials_per_step * K
        status_bytes = 64
        e2e = {"value": e2e_trials * world / (t1 - t0), "unit": "trials/s",
               "h2d_bytes_per_step": (host_spins.nbytes + 128) / K,
               "d2h_bytes_per_step": status_bytes + states.nbytes / K,
               "includes": "create from host spins + drive, K synchronous steps with status readback, "
                           "walker states to host"}
        run2.close()

    tt = None
    if rank == 0 and not args.no_time_to:
        tt = time_to_line(args, dev)
    others = None
    if rank == 0 and not args.no_others and w.name == workloads.REWL_L32.name:
        others = other_workloads_line(args, dev)

    if rank == 0:
        cpu = None if args.no_cpu else oracle_all_cores(w, seconds=args.cpu_seconds)
        state.update({"timed_iteration": st["iteration"], "timed_lnf": st["lnf"]})
        line = {"metric": METRIC, "value": value, "unit": "trials/s", "n_gpus": world, "steps": K,
                "warmup": args.warmup, "ms_per_step": total_ms / K, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": {"fp64": "f64", "f32x2": "f32x2", "f32": "f32"}[args.precision],
                "data": "synthetic",
                "config": dict(_config_dict(w, "flushed between steps (256 MiB write, outside the step events)",
                                            args.precision, "thread" if plain else _sampler_name(cfg.sampler)),
                               form=args.form, state=state,
                               tiling={"sampler": cfg.sampler, "lanes_per_walker": cfg.lanes_per_walker,
                                       "walkers_per_block": cfg.walkers_per_block,
                                       "tables": ["auto", "global", "staged"][cfg.table_mode],
                                       "lattice": ["auto", "register", "shared"][cfg.lattice_mode]}),
                "roofline": roof, "plain": plain_line, "time_to": tt, "others": others, "cpu_baseline": cpu, "e2e": e2e,
                "gpu_launches": launches * world, "clocks": clk, "peaks": peaks,
                "run": {"iteration": st["iteration"], "lnf": st["lnf"], "exch_accepts": st["exch_accepts"],
                        "exch_attempts": st["exch_attempts"]}}
        print(json.dumps(line), flush=True)
    run.close()
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def other_workloads_line(args, dev) -> dict:
    """Short device-timed runs of the other workloads the metric is quoted
    on, in the same line: the L = 64 precision-study geometry (32 x 8
    windows, 16 walkers per window, FP64, 16 lanes per walker) after 10 s
    of its own cycles, 20 timed cycles; and the uneven batch of 24 runs
    (L = 16, 24, 32, 48; compensated f32; 16 lanes), 5 timed graph launches
    of 8 cycles.  L2 flushed between steps; CUDA events on the run's stream."""
    import torch

    import paper_1508_02748_gb300 as P
    out = {}
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)

    def timed(stream, n, enqueue):
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(n)]
        with torch.cuda.stream(stream):
            for k in range(n):
                flush.zero_()
                ev[k][0].record(stream)
                enqueue()
                ev[k][1].record(stream)
        stream.synchronize()
        return sum(a.elapsed_time(b) for a, b in ev) / n

    try:
        w = workloads.REWL_L64
        cfg = P.Config.from_workload(w, replicate=args.replicate, drive_budget=10**8, precision=P.FP64,
                                     lanes_per_walker=16, walkers_per_block=1)
        run = P.REWL(cfg, device=str(dev))
        state = warm_run(run, 10.0, 16 * w.check_every)
        nw = run.status()["n_walkers"]
        ms = timed(run.stream, 20, lambda: run.enqueue_cycle(P.PART_SAMPLE | P.PART_REST))
        st = run.status()
        out[w.name] = {"value": w.exchange_interval * nw / (ms / 1e3), "unit": "trials/s", "ms_per_step": ms,
                       "steps": 20, "ln_g": "fp64", "lanes_per_walker": 16, "walkers": nw,
                       "state": dict(state, timed_iteration=st["iteration"], timed_lnf=st["lnf"])}
        run.close()
        del run
        torch.cuda.empty_cache()
    except Exception as e:                      # noqa: BLE001 -- reported in the line
        out[workloads.REWL_L64.name] = {"error": str(e)}
    try:
        wl = workloads.mixed_batch()
        runs = [P.REWL(P.Config.from_workload(w, replicate=i, drive_budget=10**8, precision=P.F32X2,
                                              lanes_per_walker=16), device=str(dev)) for i, w in enumerate(wl)]
        b = P.Batch(runs)
        with torch.cuda.stream(b.stream):
            for _ in range(3):
                b.enqueue()
        b.stream.synchronize()
        ms = timed(b.stream, 5, b.enqueue)
        active = sum(r.status()["n_walkers"] for r in runs)
        out[workloads.BATCH_NAME] = {"value": b.k * wl[0].exchange_interval * active / (ms / 1e3), "unit": "trials/s",
                                     "ms_per_step": ms, "cycles_per_step": b.k, "steps": 5, "ln_g": "f32x2",
                                     "lanes_per_walker": 16, "walkers": active, "runs": len(runs)}
        b.close()
        for r in runs:
            r.close()
        del runs, b
        torch.cuda.empty_cache()
    except Exception as e:                      # noqa: BLE001 -- reported in the line
        out[workloads.BATCH_NAME] = {"error": str(e)}
    return out


def time_to_line(args, dev) -> dict:
    """The metric's time-to half on the workload where a run reaches its final
    ln f inside a benchmark: 2D REWL at L = 8 (3 x 3 windows, 4 walkers per
    window), FP64, batched, run from creation to ln f <= 1e-6; the plain
    one-walker-per-launch form follows the same chain (same cycles, same
    tables), so its wall time is its measured time per cycle on this workload
    times the batched run's cycles (labelled extrapolated)."""
    import numpy as np
    import torch

    import paper_1508_02748_gb300 as P
    w = workloads.REWL_L8
    cfg = P.Config.from_workload(w, replicate=args.replicate, drive_budget=10**8, precision=P.FP64,
                                 lanes_per_walker=32, walkers_per_block=2)
    run = P.REWL(cfg, device=str(dev))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    st = run.status()
    while not st["done"] and time.perf_counter() - t0 < args.max_seconds:
        st = run.run_cycles(64)
    elapsed = time.perf_counter() - t0
    eps = None
    if st["done"]:
        mE = run.lng(P.LNG_MARGINAL_E)
        ex = exact_lngE(w.L)
        ok = np.isfinite(ex) & (ex > 0) & np.isfinite(mE)
        eps = float(np.mean(np.abs(mE[ok] - ex[ok]) / ex[ok]))
    run.close()
    # the plain form's time per cycle on the same workload (a fresh run, 24 cycles after 2)
    pr = P.REWL(cfg, device=str(dev))
    s = pr.stream
    with torch.cuda.stream(s):
        for _ in range(2):
            pr.enqueue_cycle(P.PART_SAMPLE_PLAIN | P.PART_REST)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(s)
        for _ in range(24):
            pr.enqueue_cycle(P.PART_SAMPLE_PLAIN | P.PART_REST)
        e1.record(s)
    s.synchronize()
    plain_ms = e0.elapsed_time(e1) / 24
    pr.close()
    return {"workload": w.name, "seed": cfg.seed, "final_lnf": st["lnf"], "done": bool(st["done"]),
            "iterations": st["iteration"], "cycles": st["cycles"],
            "batched_fp64_seconds": elapsed, "mean_eps_E_marginal_vs_exact": eps,
            "plain_fp64_ms_per_cycle": plain_ms,
            "plain_fp64_seconds_extrapolated": plain_ms * st["cycles"] / 1e3,
            "note": "plain = same chain (bit for bit), so the same cycles and the same tables; its wall time is "
                    "its measured ms per cycle times those cycles"}


def run_time_to(args, w, cfg, dev):
    """Wall time from the first cycle until the iteration with ln f <= lnf_final
    is flat, and the error of the joined E marginal against the exact g(E)."""
    import numpy as np
    import torch

    import paper_1508_02748_gb300 as P
    run = P.REWL(cfg, device=str(dev))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    st = run.status()
    chunk = 64 * w.check_every
    capped = False
    step = run.run_cycles_plain if args.form == "plain" else run.run_cycles
    while not st["done"]:
        st = step(chunk)
        if time.perf_counter() - t0 > args.max_seconds:
            capped = True
            break
    elapsed = time.perf_counter() - t0
    try:
        mE = run.lng(P.LNG_MARGINAL_E)
    except P.REWLError:               # a capped run may not have pieces to join yet
        mE = np.full(w.N + 1, np.nan)
    ex = exact_lngE(w.L)
    eps = None
    if ex is not None:
        ok = np.isfinite(ex) & (ex > 0) & np.isfinite(mE)
        eps = float(np.mean(np.abs(mE[ok] - ex[ok]) / ex[ok]))
    line = {"metric": "time-to-ln f<=%g" % w.lnf_final, "value": elapsed, "unit": "s",
            "higher_is_better": False, "n_gpus": 1, "dtype": {"fp64": "f64", "f32x2": "f32x2", "f32": "f32"}[args.precision],
            "data": "synthetic",
            "config": dict(_config_dict(w, "n/a", args.precision,
                                        "thread" if args.form == "plain" else _sampler_name(cfg.sampler)),
                           form=args.form),
            "seed": cfg.seed, "capped": capped, "max_seconds": args.max_seconds,
            "iterations": st["iteration"], "cycles": st["cycles"], "trials_per_walker": st["trials"],
            "lnf_final": st["lnf"], "mean_eps_E_marginal_vs_exact": eps,
            "exchange_acceptance": st["exch_accepts"] / max(1, st["exch_attempts"])}
    print(json.dumps(line), flush=True)
    run.close()


def run_precision(args):
    """The precision study of the L = 64 workload (32 x 8 windows at 75%
    overlap, 16 walkers per window, ln f halved from 1 down to 1e-8), one GPU.

    A: from creation, the FP64 run advances --max-seconds of wall time; the
       compensated-pair (f32x2) and plain-float runs do the same number of
       cycles from the same seed.  Their tables are compared by the device
       digest of every walker's ln g and H; the joined E marginal's error
       against the exact g(E) is given where every window overlap has been
       visited (else null).
    B: a late state at the finest ln f of the study, 2^-27: every bin of the
       one-walker-per-window geometry at ln g = 2^14 plus up to 2^-7 in steps
       of 2^-27, H = 0; --late-cycles cycles in each format, then each
       visited entry's gain is compared with its visits x ln f exactly."""
    import numpy as np
    import torch

    import paper_1508_02748_gb300 as P
    from paper_1508_02748_gb300 import build as pkg_build

    pkg_build.build()
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    w = workloads.REWL_L64
    fmt = {"fp64": P.FP64, "f32x2": P.F32X2, "f32": P.F32}
    ex = exact_lngE(64)
    out = {"A": {}, "B": {}}
    cycles = None
    for name in ("fp64", "f32x2", "f32"):
        cfg = P.Config.from_workload(w, replicate=args.replicate, drive_budget=10**8, precision=fmt[name])
        run = P.REWL(cfg, device=str(dev))
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        st = run.status()
        if cycles is None:
            while time.perf_counter() - t0 < args.max_seconds and not st["done"]:
                st = run.run_cycles(16 * w.check_every)
            cycles = st["cycles"]
        else:
            st = run.run_cycles(cycles)
        dt = time.perf_counter() - t0
        eps = None
        try:
            mE = run.lng(P.LNG_MARGINAL_E)
            ok = np.isfinite(ex) & (ex > 0) & np.isfinite(mE)
            eps = float(np.mean(np.abs(mE[ok] - ex[ok]) / ex[ok]))
        except P.REWLError as e:
            eps = f"not joinable yet: {e}"
        out["A"][name] = {"cycles": st["cycles"], "iteration": st["iteration"], "lnf": st["lnf"],
                          "seconds": dt, "trials_per_s": st["cycles"] * w.exchange_interval * st["n_walkers"] / dt,
                          "digest": f"{run.digest():016x}", "mean_eps_E_marginal_vs_exact": eps}
        run.close()
        del run
        torch.cuda.empty_cache()
    A = out["A"]
    out["A"]["f32x2_equals_fp64"] = A["f32x2"]["digest"] == A["fp64"]["digest"]
    out["A"]["f32_equals_fp64"] = A["f32"]["digest"] == A["fp64"]["digest"]

    rng = np.random.default_rng(11)
    base = H0 = None
    tabs = {}
    for name in ("fp64", "f32x2", "f32"):
        cfg = P.Config.from_workload(w.with_(walkers_per_window=1, lnf_init=2.0 ** -27), replicate=args.replicate,
                                     drive_budget=10**8, precision=fmt[name])
        run = P.REWL(cfg, device=str(dev))
        if base is None:
            n = run.tables()[1].size
            base = 16384 + rng.integers(0, 2**20, size=n) * 2.0 ** -27
            H0 = np.zeros(n, dtype=np.int32)
        run.set_tables(base, H0)
        run.run_cycles(args.late_cycles)
        lng, H = run.tables()
        vis = H > 0
        stored = base if name != "f32" else base.astype(np.float32).astype(np.float64)
        gain = lng[vis] - stored[vis]
        want = H[vis] * 2.0 ** -27
        out["B"][name] = {"visited_entries": int(vis.sum()), "visits": int(H.sum()),
                          "entries_gaining_exactly_visits_x_lnf": int((gain == want).sum()),
                          "entries_gaining_nothing": int((gain == 0).sum()),
                          "lost_lng_total": float((want - gain).sum()), "digest": f"{run.digest():016x}"}
        tabs[name] = lng
        run.close()
        del run
        torch.cuda.empty_cache()
    out["B"]["f32x2_equals_fp64"] = bool(np.array_equal(tabs["f32x2"], tabs["fp64"]))
    line = {"metric": "precision study: ln g tables of the exact formats and plain float", "value":
            float(out["A"]["f32x2_equals_fp64"] and out["B"]["f32x2_equals_fp64"]), "unit": "1 = f32x2 equals FP64",
            "higher_is_better": True, "n_gpus": 1, "data": "synthetic",
            "config": {"workload": w.name, "L": 64, "windows": "32x8", "walkers_per_window": 16,
                       "max_seconds": args.max_seconds, "late_cycles": args.late_cycles,
                       "late_state": "one walker per window, ln g = 2^14 + U{0..2^20} 2^-27, H = 0, ln f = 2^-27"},
            "runs": out}
    print(json.dumps(line), flush=True)


def run_gpu_batch(args):
    """The uneven batch: 24 runs of L = 16, 24, 32, 48 advanced together by
    one CUDA graph per step (K = 8 cycles of every run)."""
    import numpy as np
    import torch

    import paper_1508_02748_gb300 as P
    from paper_1508_02748_gb300 import build as pkg_build

    rank, world, local = dist_env()
    pkg_build.build()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    prec = {"fp64": P.FP64, "f32x2": P.F32X2, "f32": P.F32}[args.precision]
    wl = workloads.mixed_batch()

    def make(tiling):
        sampler, lanes, wpb = tiling
        rs = [P.REWL(P.Config.from_workload(w, replicate=i + 24 * replica_seed_index(rank), drive_budget=10**8,
                                            precision=prec, sampler=sampler, lanes_per_walker=lanes,
                                            walkers_per_block=wpb), device=str(dev))
              for i, w in enumerate(wl)]
        return rs, P.Batch(rs)

    choices = []
    if args.lanes is not None:
        choices = [(P.SAMPLER_WARP, args.lanes, args.wpb or 0)]
    elif args.sampler in ("auto", "warp"):
        choices += [(P.SAMPLER_WARP, lanes, 0) for lanes in (32, 16, 8)]
    if args.lanes is None and args.sampler in ("auto", "thread"):
        choices += [(P.SAMPLER_THREAD, 0, wpb) for wpb in (32, 64)]
    best, tune = choices[0], {}
    if not args.no_autotune and len(choices) > 1:
        # the tiling does not change any run's trajectory; time one launch per choice
        for tiling in choices:
            rs, bt = make(tiling)
            with torch.cuda.stream(bt.stream):
                bt.enqueue()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(bt.stream)
                bt.enqueue()
                e1.record(bt.stream)
            bt.stream.synchronize()
            tune[tiling] = e0.elapsed_time(e1)
            bt.close()
            for r in rs:
                r.close()
            del rs, bt
            torch.cuda.empty_cache()
        best = min(tune, key=tune.get)
    runs, batch = make(best)
    s = batch.stream
    active = sum(r.status()["n_walkers"] for r in runs)
    trials_per_step = batch.k * wl[0].exchange_interval * active
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    with torch.cuda.stream(s):
        for _ in range(args.warmup):
            batch.enqueue()
    s.synchronize()
    K = args.steps
    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(2)] for _ in range(K)]
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
    torch.cuda.synchronize()
    with torch.cuda.stream(s):
        for k in range(K):
            flush.zero_()
            ev[k][0].record(s)
            batch.enqueue()
            ev[k][1].record(s)
    s.synchronize()
    torch.cuda.synchronize()
    clk = clocks.stop()
    total_ms = reduce_max_ms(sum(ev[k][0].elapsed_time(ev[k][1]) for k in range(K)), world, dev)
    value = aggregate_rate(trials_per_step, K, world, total_ms)
    sm_count = torch.cuda.get_device_properties(dev).multi_processor_count
    mhz = clk.get("sm_mhz") or 1920.0
    peak_ops = sm_count * ALU_LANES_PER_SM * mhz * 1e6
    achieved = OPS_PER_TRIAL * trials_per_step / (total_ms / K / 1e3)
    launches_per_step = sum(batch.k * 3 + 2 * (batch.k // r.cfg.check_every) for r in runs)
    if rank == 0:
        cpu = None
        if not args.no_cpu:
            cpu = oracle_all_cores(wl[0], seconds=args.cpu_seconds)
            cpu["sample"] += " (the L=16 member of the batch, as the per-trial CPU cost)"
        line = {"metric": METRIC, "value": value, "unit": "trials/s", "n_gpus": world, "steps": K,
                "warmup": args.warmup, "ms_per_step": total_ms / K, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": {"fp64": "f64", "f32x2": "f32x2", "f32": "f32"}[args.precision],
                "data": "synthetic",
                "config": {"workload": workloads.BATCH_NAME, "runs": len(runs), "walkers": active,
                           "tiling": {"sampler": _sampler_name(best[0]), "lanes_per_walker": best[1] or "auto",
                                      "walkers_per_block": best[2] or "auto",
                                      "tried_ms_per_launch": {"%s/%d/%d" % (_sampler_name(k[0]), k[1], k[2]): v
                                                              for k, v in tune.items()}},
                           "L": [16, 24, 32, 48], "cycles_per_step": batch.k, "ln_g": args.precision,
                           "sampler": _sampler_name(best[0]),
                           "l2": "flushed between steps (256 MiB write, outside the step events)"},
                "roofline": {"bound": "alu", "achieved": achieved / 1e12, "peak": peak_ops / 1e12, "unit": "Tops/s",
                             "frac": achieved / peak_ops, "traffic": None,
                             "kernel": ("k_sweep_tree" if best[0] == P.SAMPLER_WARP else "k_sweep_thread")
                                       + " (24 concurrent)",
                             "peak_basis": f"{sm_count} SMs x {ALU_LANES_PER_SM} lanes x median SM clock {mhz:.0f} MHz "
                                           "(derived); achieved over the whole step"},
                "cpu_baseline": cpu, "e2e": None, "gpu_launches": launches_per_step * K * world, "clocks": clk}
        print(json.dumps(line), flush=True)
    batch.close()
    for r in runs:
        r.close()


def main():
    args = parse()
    if args.warmup < 3:
        args.warmup = 3
    w = workloads.ALL.get(args.workload)
    if args.precision is None and w is not None:
        args.precision = "fp64"
    if args.experiment == "eq5":
        args.precision = args.precision or "fp64"
        run_eq5(args)
        return
    if args.experiment == "precision":
        run_precision(args)
        return
    if args.workload == workloads.BATCH_NAME:
        if args.precision is None or args.precision == "fp64":
            args.precision = "f32x2" if args.precision is None else args.precision
        if args.impl == "reference":
            print(json.dumps({"impl": "reference", "unavailable": "the batch workload needs ~35 GB of oracle "
                              "tables; time the oracle on a single run instead"}))
            return
        run_gpu_batch(args)
        return
    if args.impl == "reference":
        if args.time_to:
            run_reference_time_to(args, w)
        else:
            run_reference(args, w)
    else:
        run_gpu(args, w)


if __name__ == "__main__":
    main()
