"""Autotuner for the package scheduler's free parameters.

For one program it times candidate configurations of (devices D, CTAs per
device C, scheduler, HGuided constant k, minimum package size) with CUDA
events and keeps the fastest.  Results are cached in a JSON file keyed by
(kernel, gws, lws), so a configuration is searched once per problem shape.
"""
from __future__ import annotations

import json
import os
import statistics
from typing import Callable, Dict, List, Optional

import torch

from . import ECL_HGUIDED, Engine, SCHEDULERS, current_device, ecl_kernel_occupancy

DEFAULT_CACHE = os.path.join(os.path.expanduser("~"), ".cache", "ecl_autotune.json")


def default_space(kernel: str, G: int, device: Optional[int] = None) -> List[Dict]:
    """Candidate configurations for a program of G work-groups."""
    sms, per_sm = ecl_kernel_occupancy(kernel, current_device(device))
    resident = sms * max(1, per_sm)
    space = []
    for D in sorted({1, 4, 8, 12, 16, 24, 64, resident}):
        if D > resident:
            continue
        C = 0  # automatic: fill the GPU
        for k in (0.5, 1.0, 2.0, 4.0):
            for mn in (1, 2, 4, 8):
                if mn > max(1, G // max(1, D)):
                    continue
                space.append(dict(scheduler="hguided", params=[k, mn], devices=D, ctas=C))
        for npk in (64, 256, 1024):  # 256: the Gaussian configuration's package count
            if npk <= G:
                space.append(dict(scheduler="dynamic", params=[npk], devices=D, ctas=C))
    return space


def _time(engine: Engine, reps: int, warmup: int) -> float:
    s = torch.cuda.current_stream()
    for _ in range(warmup):
        engine.run()
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    ts = []
    for _ in range(reps):
        a.record(s)
        engine.run()
        b.record(s)
        b.synchronize()
        ts.append(a.elapsed_time(b))
    return statistics.median(ts)


def autotune(kernel: str, make_program: Callable[[], object], gws: int, lws: int,
             space: Optional[List[Dict]] = None, reps: int = 3, warmup: int = 1,
             cache_path: Optional[str] = DEFAULT_CACHE, device: Optional[int] = None,
             refresh: bool = False) -> Dict:
    """Returns {'config': best, 'ms': time, 'table': [(config, ms), ...]}.

    ``make_program()`` builds a fresh Program for each candidate (an engine
    owns its program).  With a cache path, a previous result for the same
    (kernel, gws, lws) is returned without timing.
    """
    key = "%s|%d|%d" % (kernel, gws, lws)
    cache = {}
    if cache_path and os.path.exists(cache_path):
        try:
            with open(cache_path) as f:
                cache = json.load(f)
        except (OSError, ValueError):
            cache = {}
    if not refresh and key in cache:
        return cache[key]
    if space is None:
        space = default_space(kernel, gws // lws, device)
    table = []
    for cfg in space:
        eng = Engine(device)
        try:
            eng.work_items(gws, lws).scheduler(SCHEDULERS[cfg["scheduler"]], cfg["params"])
            eng.workers(cfg["devices"], cfg["ctas"])
            eng.program(make_program())
            table.append((cfg, _time(eng, reps, warmup)))
        finally:
            eng.close()
    best, ms = min(table, key=lambda t: t[1])
    res = {"config": best, "ms": ms, "table": table}
    if cache_path:
        cache[key] = res
        os.makedirs(os.path.dirname(cache_path), exist_ok=True)
        tmp = cache_path + ".tmp"
        with open(tmp, "w") as f:
            json.dump(cache, f)
        os.replace(tmp, cache_path)
    return res


def apply(engine: Engine, config: Dict) -> Engine:
    """Sets an engine's scheduler and workers from a tuned configuration."""
    engine.scheduler(SCHEDULERS.get(config["scheduler"], ECL_HGUIDED), config["params"])
    engine.workers(config["devices"], config["ctas"])
    return engine
