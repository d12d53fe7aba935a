"""Autotuner for the library's launch choices.

Three tunables, each with bit-identical results for every setting:

* tune_grain: the grain of a grouped (uneven-batch) launch, how many warp
  steps a warp takes from its phase's work counter at a time. Small grains
  balance the end of each phase better; large grains cost fewer atomic
  fetches on the one counter every warp of the GPU draws from.
* tune_features: the launch shape of a plan's batched feature kernel
  (mck_plan_set_launch): at d <= 1024 one round of a warp's vectors per work
  item or a full tile (one table load per 4 samples); at 2^11 <= d <= 2^14 the
  rows per work item (1, 2 or 4, tables kept in registers across them) and
  whether the next row's input is staged through shared memory with cp.async.
* tune_fwht: the regime of the FP32 transform at d = 2^16 and 2^17 (one pass
  on clusters of 2^15- or 2^14-float blocks, or two passes).

and one choice between arithmetic forms held to the same accuracy bar:

* tune_logits: the contraction of the fused logits at d = 1024 (FP32 FMAs or
  the tensor-core fp16 hi/lo split). The two round differently, both within
  the fused logits' 1e-4 bar against the FP64 oracle; the tuner returns the
  faster precision for fused_logits(..., prec=...) and sets nothing.

The tuner times each candidate on the caller's own data with CUDA events and
keeps the fastest; results are cached in a JSON file keyed by the workload's
signature (sizes and the GPU name), so a sweep runs once per workload shape.
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


def _events_ms(fn, reps, device):
    for _ in range(2):
        fn()
    torch.cuda.synchronize(device)
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    a.record()
    for _ in range(reps):
        fn()
    b.record()
    torch.cuda.synchronize(device)
    return a.elapsed_time(b) / reps


def _write_cache(cache, key, entry):
    data = _read_cache(cache)
    data[key] = entry
    # write-then-rename: several processes sharing the file (one per GPU)
    # never see a half-written cache
    tmp = f"{cache}.{os.getpid()}.tmp"
    with open(tmp, "w") as f:
        json.dump(data, f, indent=1)
    os.replace(tmp, cache)


def _cache_path(cache):
    return cache if cache is not None else os.environ.get("MCK_TUNE_CACHE")


def features_signature(plan, x):
    """Key of a feature workload: d, E, the batch size rounded up to a power
    of two, the input width, whether rows are 16-byte aligned (the staged
    kernels need it) and the GPU name."""
    n, in_dim = x.shape
    aligned = (x.data_ptr() % 16 == 0) and in_dim % 4 == 0 and (x.stride(0) % 4 == 0 or n == 1)
    nb = 1 << max(0, int(n - 1).bit_length())
    h = hashlib.sha256(f"features:{plan.d}:{plan.E}:{nb}:{in_dim}:{int(aligned)}".encode())
    h.update(torch.cuda.get_device_name(plan.device).encode())
    return h.hexdigest()[:24]


def tune_features(plan, x, out=None, candidates=None, reps=5, cache=None):
    """Pick and set the fastest launch shape of plan's feature kernel for
    inputs like x; returns ((rows_per_item, staged), {shape: ms}, from_cache).

    candidates: (rows_per_item, staged) pairs (default: every shape the plan
    accepts). out: a feature buffer to write into (default: allocated).
    cache: JSON path (default: $MCK_TUNE_CACHE if set, else no cache).
    """
    from . import features

    cache = _cache_path(cache)
    key = features_signature(plan, x)
    if cache:
        entry = _read_cache(cache).get(key)
        if entry and entry.get("kind") == "features":
            shape = (int(entry["rows_per_item"]), int(entry["staged"]))
            plan.set_launch(*shape)
            return shape, {tuple(map(int, k.split(","))): v for k, v in entry["ms"].items()}, True
    cands = list(candidates) if candidates is not None else plan.launch_candidates()
    if out is None:
        out = torch.empty((x.shape[0], plan.num_features), device=x.device)
    times = {}
    for shape in cands:
        plan.set_launch(*shape)
        times[tuple(shape)] = _events_ms(lambda: features(plan, x, out=out), reps, x.device)
    best = min(times, key=times.get)
    plan.set_launch(*best)
    if cache:
        _write_cache(cache, key, {"kind": "features", "rows_per_item": best[0], "staged": best[1],
                                  "ms": {f"{k[0]},{k[1]}": v for k, v in times.items()}})
    return best, times, False


FWHT_REGIMES = ("cluster_2_15", "cluster_2_14", "two_pass")


def tune_fwht(x, regimes=FWHT_REGIMES, reps=5, cache=None):
    """The fastest FP32 regime for transforming x in place (rows of d = 2^16
    or 2^17); returns (regime, {regime: ms}, from_cache). x is overwritten
    (the candidates transform it repeatedly)."""
    from . import fwht_

    d = x.shape[-1]
    if d not in (1 << 16, 1 << 17):
        return "auto", {}, False
    cache = _cache_path(cache)
    n = x.numel() // d
    nb = 1 << max(0, int(n - 1).bit_length())
    h = hashlib.sha256(f"fwht:{d}:{nb}".encode())
    h.update(torch.cuda.get_device_name(x.device).encode())
    key = h.hexdigest()[:24]
    if cache:
        entry = _read_cache(cache).get(key)
        if entry and entry.get("kind") == "fwht":
            return entry["regime"], dict(entry["ms"]), True
    times = {r: _events_ms(lambda: fwht_(x, "fp32", r), reps, x.device) for r in regimes}
    best = min(times, key=times.get)
    if cache:
        _write_cache(cache, key, {"kind": "fwht", "regime": best, "ms": times})
    return best, times, False


LOGIT_PRECISIONS = ("fp32", "fp16_split")


def tune_logits(plan, x, W, b=None, precs=LOGIT_PRECISIONS, reps=5, cache=None):
    """The faster contraction of fused_logits for inputs like x and weights
    like W; returns (prec, {prec: ms}, from_cache). Below or above d = 1024
    only the FP32 contraction exists and is returned untimed."""
    from . import fused_logits

    if plan.d != 1024:
        return "fp32", {}, False
    cache = _cache_path(cache)
    n = x.shape[0]
    nb = 1 << max(0, int(n - 1).bit_length())
    h = hashlib.sha256(f"logits:{plan.d}:{plan.E}:{nb}:{x.shape[1]}:{W.shape[0]}".encode())
    h.update(torch.cuda.get_device_name(plan.device).encode())
    key = h.hexdigest()[:24]
    if cache:
        entry = _read_cache(cache).get(key)
        if entry and entry.get("kind") == "logits":
            return entry["prec"], dict(entry["ms"]), True
    out = torch.empty((n, W.shape[0]), device=x.device)
    times = {p: _events_ms(lambda: fused_logits(plan, x, W, b, out=out, prec=p), reps, x.device)
             for p in precs}
    best = min(times, key=times.get)
    if cache:
        _write_cache(cache, key, {"kind": "logits", "prec": best, "ms": times})
    return best, times, False


def tune_grain(group, x, phi, grains=DEFAULT_GRAINS, reps=5, cache=None):
    """Pick and set the fastest grain; returns (grain, {grain: ms}).

    cache: path of a JSON file (default: $MCK_TUNE_CACHE if set, else no cache).
    """
    cache = _cache_path(cache)
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
        _write_cache(cache, key, {"grain": best, "ms": {str(k): v for k, v in times.items()}})
    return best, times


def _read_cache(path):
    """The cache's entries, or none if the file is missing or unreadable."""
    try:
        with open(path) as f:
            data = json.load(f)
        return data if isinstance(data, dict) else {}
    except (OSError, ValueError):
        return {}
