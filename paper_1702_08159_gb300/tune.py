"""Autotuner for grouped (uneven-batch) launches.

The tunable is the grain of mck_group_create: how many warp steps a warp
takes from its phase's work counter at a time. Small grains balance the end
of each phase better; large grains cost fewer atomic fetches on the one
counter every warp of the GPU draws from. The tuner
times each candidate on the caller's own data with CUDA events and keeps the
fastest; results are cached in a JSON file keyed by the batch's signature
(the multiset of (d, E, kernel) per item and the GPU name), so the sweep runs
once per workload shape.
"""

import hashlib
import json
import os

import numpy as np
import torch

DEFAULT_GRAINS = (1, 2, 4, 8, 16)


def signature(group):
    plans = group.plans
    keys = np.stack([np.array([plans[p].d for p in group.items["plan"]]),
                     group.items["E"], np.array([plans[p].kernel for p in group.items["plan"]])])
    uniq, counts = np.unique(keys, axis=1, return_counts=True)
    h = hashlib.sha256(uniq.tobytes() + counts.tobytes())
    h.update(torch.cuda.get_device_name(group.device).encode())
    return h.hexdigest()[:24]


def _time(group, x, phi, reps):
    for _ in range(2):
        group.features(x, phi)
    torch.cuda.synchronize(group.device)
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    a.record()
    for _ in range(reps):
        group.features(x, phi)
    b.record()
    torch.cuda.synchronize(group.device)
    return a.elapsed_time(b) / reps


def tune_grain(group, x, phi, grains=DEFAULT_GRAINS, reps=5, cache=None):
    """Pick and set the fastest grain; returns (grain, {grain: ms}).

    cache: path of a JSON file (default: $MCK_TUNE_CACHE if set, else no cache).
    """
    cache = cache if cache is not None else os.environ.get("MCK_TUNE_CACHE")
    key = signature(group)
    if cache:
        entry = _read_cache(cache).get(key)
        if entry:
            group.set_grain(entry["grain"])
            return entry["grain"], {int(k): v for k, v in entry["ms"].items()}
    times = {}
    for g in grains:
        group.set_grain(g)
        times[g] = _time(group, x, phi, reps)
    best = min(times, key=times.get)
    group.set_grain(best)
    if cache:
        data = _read_cache(cache)
        data[key] = {"grain": best, "ms": {str(k): v for k, v in times.items()}}
        # write-then-rename: several processes sharing the file (one per GPU)
        # never see a half-written cache
        tmp = f"{cache}.{os.getpid()}.tmp"
        with open(tmp, "w") as f:
            json.dump(data, f, indent=1)
        os.replace(tmp, cache)
    return best, times


def _read_cache(path):
    """The cache's entries, or none if the file is missing or unreadable."""
    try:
        with open(path) as f:
            data = json.load(f)
        return data if isinstance(data, dict) else {}
    except (OSError, ValueError):
        return {}
