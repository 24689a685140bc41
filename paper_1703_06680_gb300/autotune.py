"""Autotuner for the library's tunables (ddm_set_param).

For one workload class -- GPU name, d, size bucket (log2 of N) and output
density bucket (log2 of K/N) -- every candidate value of each tunable is timed
with CUDA events on the context's stream (median of a few ddm_match calls
after a warm-up) and the fastest is kept.  Results are cached in a JSON file
so that later contexts can apply them without re-measuring.
"""
from __future__ import annotations

import json
import math
import os
import statistics

from ._lib import (PARAM_JOIN_SHIFT, PARAM_ND_PATH, PARAM_ND_WRITE, PARAM_SORT_ITEMS,
                   PARAM_SWEEP_DIM, PARAM_WIN_SHIFT)

# Candidate values per tunable, in the order they are tuned (one at a time, each
# with the best values found so far for the earlier ones), and which
# dimensionalities a tunable affects.  Algorithm choices first, then tile sizes:
# the sort's keys per thread (tiles of 3072 / 4096 / 4608 keys), the window of
# the d = 1 emission and the window of the d > 1 join.
CANDIDATES = {PARAM_ND_PATH: (1, 2), PARAM_SWEEP_DIM: (0, 1), PARAM_ND_WRITE: (1, 2),
              PARAM_SORT_ITEMS: (12, 16, 18), PARAM_WIN_SHIFT: (8, 9, 10),
              PARAM_JOIN_SHIFT: (9, 10, 11)}
NAMES = {PARAM_WIN_SHIFT: "win_shift", PARAM_ND_PATH: "nd_path", PARAM_SWEEP_DIM: "sweep_dim",
         PARAM_SORT_ITEMS: "sort_items", PARAM_JOIN_SHIFT: "join_shift",
         PARAM_ND_WRITE: "nd_write"}
APPLIES = {PARAM_WIN_SHIFT: lambda d: d == 1, PARAM_ND_PATH: lambda d: d > 1,
           PARAM_SWEEP_DIM: lambda d: d > 1, PARAM_SORT_ITEMS: lambda d: True,
           PARAM_JOIN_SHIFT: lambda d: d > 1, PARAM_ND_WRITE: lambda d: d > 1}
DEFAULT_CACHE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "_build", "autotune.json")


def workload_key(gpu: str, d: int, N: int, K: int) -> str:
    size = int(math.log2(max(N, 1)))
    dens = int(math.floor(math.log2(max(K, 1) / max(N, 1)))) if K else -99
    return f"{gpu}|d{d}|n{size}|k{dens}"


def _load(path: str) -> dict:
    if os.path.exists(path):
        with open(path) as fh:
            return json.load(fh)
    return {}


def _save(path: str, cache: dict):
    os.makedirs(os.path.dirname(path), exist_ok=True)
    tmp = path + f".tmp{os.getpid()}"
    with open(tmp, "w") as fh:
        json.dump(cache, fh, indent=1, sort_keys=True)
    os.replace(tmp, path)


def cuda_timer(ctx, tensors, K: int, reps: int) -> float:
    """Median device time (ms) of `reps` ddm_match calls, CUDA events on the
    context's stream, after one warm-up call."""
    import torch
    out = torch.empty((max(K, 1), 2), dtype=torch.int32, device=tensors[0].device)
    ctx.match_into(out[:K], *tensors)
    ms = []
    for _ in range(reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(ctx.stream)
        ctx.match_into(out[:K], *tensors)
        e1.record(ctx.stream)
        e1.synchronize()
        ms.append(e0.elapsed_time(e1))
    return statistics.median(ms)


def _gpu_name(ctx) -> str:
    import torch
    return torch.cuda.get_device_name(ctx.device)


def tune(ctx, tensors, reps: int = 5, cache_path: str = DEFAULT_CACHE, gpu: str | None = None,
         timer=cuda_timer) -> dict:
    """Times every candidate for the workload `tensors` (d, n, m CUDA tensors), applies
    the best values to `ctx`, caches them and returns {name: value, ..., "key": key}.
    `timer(ctx, tensors, K, reps)` returns the time of one candidate in ms."""
    K = ctx.count(*tensors)
    d, n = tensors[0].shape
    N = n + tensors[2].shape[1]
    key = workload_key(gpu if gpu is not None else _gpu_name(ctx), d, N, K)
    chosen = {"key": key}
    for param, values in CANDIDATES.items():
        if not APPLIES[param](d):
            continue
        best, best_ms, times = None, float("inf"), {}
        for v in values:
            ctx.set_param(param, v)
            times[str(v)] = timer(ctx, tensors, K, reps)
            if times[str(v)] < best_ms:
                best, best_ms = v, times[str(v)]
        ctx.set_param(param, best)
        chosen[NAMES[param]] = best
        chosen[NAMES[param] + "_ms"] = times
    cache = _load(cache_path)
    cache[key] = {k: v for k, v in chosen.items() if k != "key"}
    _save(cache_path, cache)
    return chosen


def apply_cached(ctx, tensors, K: int | None = None, cache_path: str = DEFAULT_CACHE,
                 gpu: str | None = None) -> bool:
    """Applies cached tunables for this workload class, if any; returns whether it did."""
    if K is None:
        K = ctx.count(*tensors)
    d, n = tensors[0].shape
    key = workload_key(gpu if gpu is not None else _gpu_name(ctx), d, n + tensors[2].shape[1], K)
    entry = _load(cache_path).get(key)
    if not entry:
        return False
    for param, name in NAMES.items():
        if name in entry:
            ctx.set_param(param, int(entry[name]))
    return True
