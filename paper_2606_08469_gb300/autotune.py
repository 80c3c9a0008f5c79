"""Autotuner of the library's launch knobs (octa_tuning).

For a given workload (a callable that runs one step or one query batch
through the library on the current stream) it times every candidate setting
of the knobs that matter for that workload -- resident CTAs per SM (how many
128-query tiles each SM keeps in flight) and the order in which persistent
CTAs take work (interleaved, or one contiguous chunk per CTA, which means
fewer scene switches in a multi-scene launch) -- with CUDA events after a
warm-up, picks the fastest and caches the result in a JSON file keyed by the
GPU name and a workload signature.
"""
from __future__ import annotations

import ctypes as C
import itertools
import json
import os

import torch

from . import _lib as L

KNOBS = ("fwd_ctas_per_sm", "encode_ctas_per_sm", "engine_ctas_per_sm", "fwd_order", "train_order",
         "fwd_threads_per_query", "encode_threads_per_query", "train_threads_per_row", "fwd_run",
         "train_run", "gather_stages", "l1_carveout")


def get_tuning():
    t = L.octa_tuning()
    L.check(L.load().octa_get_tuning(C.byref(t)), "octa_get_tuning")
    return {k: getattr(t, k) for k in KNOBS}


def set_tuning(values=None):
    """Apply a dict of knob values (missing keys = default); None resets."""
    if values is None:
        L.check(L.load().octa_set_tuning(None), "octa_set_tuning")
        return
    t = L.octa_tuning()
    for k, v in values.items():
        setattr(t, k, int(v))
    L.check(L.load().octa_set_tuning(C.byref(t)), "octa_set_tuning")


def time_fn(fn, reps=10, warmup=3, flush_bytes=256 << 20):
    """Median device time (ms) of fn, L2 flushed before every timed run."""
    flush = torch.empty(flush_bytes, dtype=torch.uint8, device="cuda")
    stream = torch.cuda.current_stream()
    for _ in range(warmup):
        fn()
    evs = []
    for _ in range(reps):
        flush.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        fn()
        b.record(stream)
        evs.append((a, b))
    torch.cuda.synchronize()
    ts = sorted(a.elapsed_time(b) for a, b in evs)
    return ts[len(ts) // 2]


def _key(signature):
    return f"{torch.cuda.get_device_name()}|{signature}"


def autotune(fn, space, signature, cache_path=None, reps=10):
    """Grid search over `space` ({knob: [values]}) for the callable fn.

    Returns (best_setting, report) where report lists every candidate's
    time and the default's.  The best setting is applied and, with
    cache_path, stored under (GPU name, signature)."""
    if cache_path and os.path.exists(cache_path):
        with open(cache_path) as f:
            cache = json.load(f)
        hit = cache.get(_key(signature))
        if hit:
            set_tuning(hit["best"])
            return hit["best"], hit
    set_tuning(None)
    default_ms = time_fn(fn, reps)
    names = sorted(space)
    trials = []
    for combo in itertools.product(*[space[n] for n in names]):
        setting = dict(zip(names, combo))
        set_tuning(setting)
        trials.append({"setting": setting, "ms": round(time_fn(fn, reps), 5)})
    best = min(trials, key=lambda r: r["ms"])
    report = {"best": best["setting"], "best_ms": best["ms"], "default_ms": round(default_ms, 5),
              "gain": round(default_ms / best["ms"], 4), "trials": trials}
    set_tuning(best["setting"])
    if cache_path:
        cache = {}
        if os.path.exists(cache_path):
            with open(cache_path) as f:
                cache = json.load(f)
        cache[_key(signature)] = report
        os.makedirs(os.path.dirname(os.path.abspath(cache_path)), exist_ok=True)
        with open(cache_path, "w") as f:
            json.dump(cache, f, indent=1)
    return best["setting"], report
