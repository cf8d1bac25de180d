"""Tiling autotuner for the sampling kernels.

The sampler's mapping onto the GPU -- one thread per walker, or a group of
8, 16 or 32 lanes per walker (3, 4 or 5 trials resolved per step), how many
threads or warps share a block, whether a walker's screen and visit counts
are staged in shared memory or read from global memory, and whether a small
lattice (N <= 64) is held in a register or in shared memory -- does not
change the trajectory (every variant is the same chain trial for trial),
only its speed.  ``autotune`` times a few
candidate tilings on the actual configuration for a couple of cycles with
CUDA events and returns the configuration with the fastest one; results are
cached in a JSON file keyed by GPU name and problem shape.
"""
from __future__ import annotations

import dataclasses
import json
import os

import math

from .rewl import (LATTICE_AUTO, LATTICE_SHARED, REWL, SAMPLER_THREAD, SAMPLER_WARP, TABLES_AUTO, TABLES_GLOBAL, Config,
                   REWLError)

DEFAULT_CACHE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "_build", "autotune.json")


def _key(cfg: Config, gpu: str, samplers) -> str:
    return (f"{gpu}|s{''.join(str(x) for x in sorted(samplers))}|L{cfg.L}|{cfg.n_win_E}x{cfg.n_win_M}|o{cfg.overlap_E:g},{cfg.overlap_M:g}"
            f"|W{cfg.walkers_per_window}|p{cfg.precision}|x{cfg.exchange_interval}|c{cfg.check_every}")


def _window_bins(cfg: Config) -> int:
    B = cfg.L * cfg.L + 1

    def width(n, o):
        return B if n == 1 else min(B, math.ceil(B / (1 + (n - 1) * (1 - o))))
    return width(cfg.n_win_E, cfg.overlap_E) * width(cfg.n_win_M, cfg.overlap_M)


def candidates(cfg: Config, samplers=(SAMPLER_WARP, SAMPLER_THREAD)):
    """(sampler, lanes, warps or threads per block, table_mode, lattice_mode) choices."""
    out = []
    if SAMPLER_WARP in samplers:
        lattices = [LATTICE_AUTO] + ([LATTICE_SHARED] if cfg.L * cfg.L <= 64 else [])
        for lanes in (32, 16, 8):
            # global tables are a separate choice only where staging is (a warp's share of
            # shared memory at 8 bytes per bin, the ring and mailbox beside them)
            stageable = (_window_bins(cfg) * 8 + 2400) * (32 // lanes) <= 100 * 1024
            tables = [TABLES_AUTO, TABLES_GLOBAL] if stageable else [TABLES_AUTO]
            out += [(SAMPLER_WARP, lanes, wpb, tm, lm) for wpb in (1, 2, 4) for tm in tables for lm in lattices]
    if SAMPLER_THREAD in samplers:
        out += [(SAMPLER_THREAD, 0, wpb, TABLES_AUTO, LATTICE_AUTO) for wpb in (8, 32, 64)]
    return out


def autotune(cfg: Config, device: str = "cuda:0", cycles: int = 2, cache_path: str | None = DEFAULT_CACHE,
             verbose: bool = False, samplers=(SAMPLER_WARP, SAMPLER_THREAD)) -> Config:
    """Fastest tiling of ``cfg`` among ``candidates(cfg, samplers)``."""
    import torch
    gpu = torch.cuda.get_device_name(torch.device(device))
    key = _key(cfg, gpu, samplers)
    cache = {}
    if cache_path and os.path.exists(cache_path):
        try:
            cache = json.load(open(cache_path))
        except (OSError, ValueError):
            cache = {}
    if key in cache and "tables" in cache[key]:
        c = cache[key]
        return dataclasses.replace(cfg, sampler=c["sampler"], lanes_per_walker=c["lanes"],
                                   walkers_per_block=c["wpb"], table_mode=c["tables"], lattice_mode=c["lattice"])
    best = None
    for sampler, lanes, wpb, tm, lm in candidates(cfg, samplers):
        trial = dataclasses.replace(cfg, sampler=sampler, lanes_per_walker=lanes, walkers_per_block=wpb,
                                    table_mode=tm, lattice_mode=lm)
        try:
            run = REWL(trial, device=device)
            with torch.cuda.stream(run.stream):
                run.enqueue_cycle()
                t0 = torch.cuda.Event(enable_timing=True)
                t1 = torch.cuda.Event(enable_timing=True)
                t0.record(run.stream)
                for _ in range(cycles):
                    run.enqueue_cycle()
                t1.record(run.stream)
            run.stream.synchronize()
            run.status()                    # surfaces a failed launch
        except REWLError as err:            # a tiling this shape cannot use
            if verbose:
                print(f"autotune {key}: sampler={sampler} lanes={lanes} wpb={wpb} tables={tm} lattice={lm}: "
                      f"skipped ({err})", flush=True)
            continue
        ms = t0.elapsed_time(t1) / cycles
        if verbose:
            print(f"autotune {key}: sampler={sampler} lanes={lanes} wpb={wpb} tables={tm} lattice={lm}: "
                  f"{ms:.3f} ms/cycle", flush=True)
        if best is None or ms < best[0]:
            best = (ms, sampler, lanes, wpb, tm, lm)
        run.close()
        del run
        torch.cuda.empty_cache()
    ms, sampler, lanes, wpb, tm, lm = best
    cache[key] = {"sampler": sampler, "lanes": lanes, "wpb": wpb, "tables": tm, "lattice": lm, "ms_per_cycle": ms}
    if cache_path:
        os.makedirs(os.path.dirname(cache_path), exist_ok=True)
        tmp = cache_path + f".{os.getpid()}.tmp"
        json.dump(cache, open(tmp, "w"), indent=1, sort_keys=True)
        os.replace(tmp, cache_path)
    return dataclasses.replace(cfg, sampler=sampler, lanes_per_walker=lanes, walkers_per_block=wpb, table_mode=tm,
                               lattice_mode=lm)
