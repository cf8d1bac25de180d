"""Tiling autotuner for the sampling kernels.

The sampler's mapping onto the GPU -- one thread per walker, or a group of
8, 16 or 32 lanes per walker (3, 4 or 5 trials resolved per step), and how
many threads or warps share a block -- does not change the trajectory (every variant is
the same chain trial for trial), only its speed.  ``autotune`` times a few
candidate tilings on the actual configuration for a couple of cycles with
CUDA events and returns the configuration with the fastest one; results are
cached in a JSON file keyed by GPU name and problem shape.
"""
from __future__ import annotations

import dataclasses
import json
import os

from .rewl import REWL, SAMPLER_THREAD, SAMPLER_WARP, Config, REWLError

DEFAULT_CACHE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "_build", "autotune.json")


def _key(cfg: Config, gpu: str, samplers) -> str:
    return (f"{gpu}|s{''.join(str(x) for x in sorted(samplers))}|L{cfg.L}|{cfg.n_win_E}x{cfg.n_win_M}|o{cfg.overlap_E:g},{cfg.overlap_M:g}"
            f"|W{cfg.walkers_per_window}|p{cfg.precision}|x{cfg.exchange_interval}|c{cfg.check_every}")


def candidates(cfg: Config, samplers=(SAMPLER_WARP, SAMPLER_THREAD)):
    out = []
    if SAMPLER_WARP in samplers:
        out += [(SAMPLER_WARP, lanes, wpb) for lanes in (32, 16, 8) for wpb in (1, 2, 4)]
    if SAMPLER_THREAD in samplers:
        out += [(SAMPLER_THREAD, 0, wpb) for wpb in (8, 32, 64)]
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
    if key in cache:
        c = cache[key]
        return dataclasses.replace(cfg, sampler=c["sampler"], lanes_per_walker=c["lanes"],
                                   walkers_per_block=c["wpb"])
    best = None
    for sampler, lanes, wpb in candidates(cfg, samplers):
        trial = dataclasses.replace(cfg, sampler=sampler, lanes_per_walker=lanes, walkers_per_block=wpb)
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
                print(f"autotune {key}: sampler={sampler} lanes={lanes} wpb={wpb}: skipped ({err})", flush=True)
            continue
        ms = t0.elapsed_time(t1) / cycles
        if verbose:
            print(f"autotune {key}: sampler={sampler} lanes={lanes} wpb={wpb}: {ms:.3f} ms/cycle", flush=True)
        if best is None or ms < best[0]:
            best = (ms, sampler, lanes, wpb)
        run.close()
        del run
        torch.cuda.empty_cache()
    ms, sampler, lanes, wpb = best
    cache[key] = {"sampler": sampler, "lanes": lanes, "wpb": wpb, "ms_per_cycle": ms}
    if cache_path:
        os.makedirs(os.path.dirname(cache_path), exist_ok=True)
        tmp = cache_path + f".{os.getpid()}.tmp"
        json.dump(cache, open(tmp, "w"), indent=1, sort_keys=True)
        os.replace(tmp, cache_path)
    return dataclasses.replace(cfg, sampler=sampler, lanes_per_walker=lanes, walkers_per_block=wpb)
