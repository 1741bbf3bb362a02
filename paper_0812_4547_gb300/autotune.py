"""Launch-shape autotuner for the library's closed-form choices.

The knobs are the fields of ``rnnls_tuning`` (see include/rnnls.h): the
sketch's SM cap and full-step threshold, the tensor-core Gram's K-split
limits, the batched Gram's chunks per CTA, the batched sketch's step cost
and the largest Lawson-Hanson problem that runs as a one-warp block.
None changes what is computed beyond FP32 summation order.  The tuner
times a caller-supplied step (CUDA events on the context's stream) for each
candidate value of one knob at a time, keeping the others at their best so
far (coordinate search), and stores the winner per device and shape in a
JSON cache::

    {"version": 1, "entries": {"<device>|<kind>|<shape>": {"tuning": {...},
     "ms": t_best, "default_ms": t_default, "trials": [[{...}, t], ...]}}}

The cache path is ``$RNNLS_TUNING_CACHE`` or ``~/.cache/rnnls/tuning.json``.
"""
from __future__ import annotations

import json
import os
import statistics
import tempfile

CACHE_VERSION = 1

#: candidate values per knob (0 = the library's built-in default)
CANDIDATES = {
    "full_step_min_slots": [0, 64, 96, 1024],
    "gram_min_chunks": [0, 4, 16, 32],
    "gram_max_splits": [0, 8, 16, 64],
    "batch_gram_chunks": [0, 32, 64, 256],
    "batch_step_cost": [0, 60, 180, 300],
    "lh_warp_max_d": [0, 32, 64],
}

#: the knobs that act on each kind of workload
KNOBS_FOR = {
    "single": ["full_step_min_slots", "gram_min_chunks", "gram_max_splits", "lh_warp_max_d"],
    "batched": ["full_step_min_slots", "batch_step_cost", "batch_gram_chunks", "lh_warp_max_d"],
}


def cache_path() -> str:
    return os.environ.get("RNNLS_TUNING_CACHE") or os.path.join(os.path.expanduser("~"), ".cache", "rnnls",
                                                                "tuning.json")


def cache_key(device: str, kind: str, **shape) -> str:
    return f"{device}|{kind}|" + ",".join(f"{k}={shape[k]}" for k in sorted(shape))


def load_cache(path: str | None = None) -> dict:
    """The cache, or an empty one when the file is missing, unreadable or of
    another version."""
    path = path or cache_path()
    try:
        with open(path) as f:
            data = json.load(f)
        if isinstance(data, dict) and data.get("version") == CACHE_VERSION and isinstance(data.get("entries"), dict):
            return data
    except (OSError, ValueError):
        pass
    return {"version": CACHE_VERSION, "entries": {}}


def save_cache(cache: dict, path: str | None = None) -> None:
    """Write the cache atomically (a temporary file renamed over it)."""
    path = path or cache_path()
    os.makedirs(os.path.dirname(os.path.abspath(path)), exist_ok=True)
    fd, tmp = tempfile.mkstemp(dir=os.path.dirname(os.path.abspath(path)), suffix=".tmp")
    with os.fdopen(fd, "w") as f:
        json.dump(cache, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


def coordinate_search(time_fn, knobs: list, candidates: dict | None = None, base: dict | None = None,
                      rounds: int = 1):
    """Minimise time_fn(tuning dict) one knob at a time.  Returns (best
    tuning, its time, the time of `base`, every trial as (tuning, time))."""
    candidates = candidates or CANDIDATES
    best = dict(base or {})
    t_base = time_fn(dict(best))
    trials = [(dict(best), t_base)]
    t_best = t_base
    for _ in range(rounds):
        for k in knobs:
            for v in candidates.get(k, ()):
                if best.get(k, 0) == v:
                    continue
                trial = dict(best)
                trial[k] = v
                t = time_fn(dict(trial))
                trials.append((dict(trial), t))
                if t < t_best:
                    best, t_best = trial, t
    return best, t_best, t_base, trials


def time_step(ctx, step, repeats: int = 3, warmup: int = 1) -> float:
    """Median milliseconds of `step()` on the context's stream (CUDA events)."""
    import torch

    s = ctx.stream
    for _ in range(warmup):
        step()
    torch.cuda.synchronize()
    times = []
    for _ in range(repeats):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(s)
        step()
        e1.record(s)
        torch.cuda.synchronize()
        times.append(e0.elapsed_time(e1))
    return statistics.median(times)


def tune(contexts, step, kind: str, shape: dict, path: str | None = None, force: bool = False,
         repeats: int = 3, candidates: dict | None = None) -> dict:
    """The best tuning of `step` (a callable that runs one workload step on
    the contexts) for this device and shape: from the cache unless `force`,
    else by coordinate search over KNOBS_FOR[kind], stored in the cache.
    Every context in `contexts` gets the result applied; returns the cache
    entry (tuning, ms, default_ms, trials, cached)."""
    import torch

    ctxs = contexts if isinstance(contexts, (list, tuple)) else [contexts]
    key = cache_key(torch.cuda.get_device_name(ctxs[0].device), kind, **shape)
    cache = load_cache(path)
    entry = cache["entries"].get(key)
    if entry is None or force:
        base = ctxs[0].get_tuning()

        def timed(t):
            for c in ctxs:
                c.set_tuning(t)
            return time_step(ctxs[0], step, repeats=repeats)

        best, t_best, t_base, trials = coordinate_search(timed, KNOBS_FOR[kind], candidates, base)
        entry = {"tuning": best, "ms": t_best, "default_ms": t_base, "trials": [[t, ms] for t, ms in trials]}
        cache["entries"][key] = entry
        save_cache(cache, path)
        entry = dict(entry, cached=False)
    else:
        entry = dict(entry, cached=True)
    for c in ctxs:
        c.set_tuning(entry["tuning"])
    return dict(entry, key=key)


__all__ = ["CANDIDATES", "KNOBS_FOR", "cache_key", "cache_path", "coordinate_search", "load_cache", "save_cache",
           "time_step", "tune"]
