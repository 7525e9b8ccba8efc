"""Schedule and tile autotuner for multi-system batches (nqs_local_energy_batch).

For a workload signature (the device, and per system its K, N_alpha, N_beta, D,
a bucket of its sample count and the precision form) it times candidate
schedules on the real batch with CUDA events and keeps the fastest in a JSON
cache file:

  workers            host threads that drive the systems' streams
  tile_blocks_per_sm blocks per multiprocessor of each shared-prefix site-tile
                     launch (nqs_options.tile_blocks_per_sm)
  table_mb           cap on one sample batch's shared-prefix tables
                     (nqs_options.table_mb; 0 = the library's default)

The library's results do not depend on these parameters (each result row is
formed by the same arithmetic whatever the tiling), so tuning changes only the
time. The search is coordinate-wise: workers, then tiles, then the table cap,
each candidate timed `reps` times after one untimed call.
"""
from __future__ import annotations

import hashlib
import json
import os
import time

from . import nqs

CANDIDATES = {
    "workers": [4, 8, 16],
    "tile_blocks_per_sm": [2, 4, 8],
    "table_mb": [0, 1024],
}
DEFAULT = {"workers": 8, "tile_blocks_per_sm": 4, "table_mb": 0}
CACHE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "_build", "autotune.json")


def signature(systems, precision: int, device_name: str) -> str:
    """Stable key of a batch: device, precision and each system's shape with
    its sample count rounded up to a power of two."""
    parts = [device_name, str(precision)]
    for s in systems:
        n = len(s.samples)
        bucket = 1 << max(0, (n - 1).bit_length())
        parts.append(f"{s.K}:{s.n_alpha}:{s.n_beta}:{s.D}:{bucket}:{s.n_hidden}")
    return hashlib.sha1("|".join(parts).encode()).hexdigest()[:16]


def load_cache(path: str = CACHE) -> dict:
    try:
        with open(path) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def save_cache(cache: dict, path: str = CACHE) -> None:
    os.makedirs(os.path.dirname(path), exist_ok=True)
    tmp = f"{path}.{os.getpid()}.tmp"
    with open(tmp, "w") as f:
        json.dump(cache, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


def apply(contexts, config: dict, precision: int, energy_tol: float) -> None:
    for c in contexts:
        c.set_precision(precision, timing=False, energy_tolerance=energy_tol,
                        tile_blocks_per_sm=config["tile_blocks_per_sm"], table_mb=config["table_mb"])


def _time(contexts, args, config, precision, energy_tol, reps):
    import torch
    apply(contexts, config, precision, energy_tol)
    nqs.local_energy_batch(contexts, args, n_workers=config["workers"])      # untimed
    torch.cuda.synchronize()
    best = float("inf")
    for _ in range(reps):
        t0 = time.perf_counter()
        nqs.local_energy_batch(contexts, args, n_workers=config["workers"])
        torch.cuda.synchronize()
        best = min(best, time.perf_counter() - t0)
    return best


def tune(contexts, args, systems, precision: int, energy_tol: float = 0.0, reps: int = 2,
         cache_path: str = CACHE, force: bool = False):
    """Best schedule for this batch (from the cache unless `force`), with the
    timings of every candidate tried. The contexts are left configured with
    the chosen tile parameters (timing off)."""
    import torch
    key = signature(systems, precision, torch.cuda.get_device_name())
    cache = load_cache(cache_path)
    if not force and key in cache:
        cfg = cache[key]["config"]
        apply(contexts, cfg, precision, energy_tol)
        return cfg, cache[key]
    cfg = dict(DEFAULT)
    trials = []
    for name in ("workers", "tile_blocks_per_sm", "table_mb"):
        results = {}
        for v in CANDIDATES[name]:
            trial = dict(cfg, **{name: v})
            t = _time(contexts, args, trial, precision, energy_tol, reps)
            results[v] = t
            trials.append({"config": trial, "seconds": t})
        cfg[name] = min(results, key=results.get)
    entry = {"config": cfg, "trials": trials, "when": time.strftime("%Y-%m-%dT%H:%M:%SZ", time.gmtime())}
    cache[key] = entry
    save_cache(cache, cache_path)
    apply(contexts, cfg, precision, energy_tol)
    return cfg, entry
