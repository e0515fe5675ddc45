"""Autotuner for the SpGEMM plan options.

Picks, for a given product, the numeric window width (columns per warp
accumulator), the product count above which rows are split into window
tiles, and the product count at which the symbolic pass switches from one
warp to a whole block per row.  Each candidate is timed on the product
itself (symbolic and numeric passes, CUDA events on the current stream,
best of ``reps``).  Winners are cached in a JSON file keyed by the GPU
(name, SM count), the value type and a size class of the product
(log2 buckets of rows, nnz(A) and total and largest row product counts), so
products of the same shape reuse the choice.

The cache holds only option values, never results of the product.
"""
from __future__ import annotations

import itertools
import json
import math
import os
import threading

import torch

from . import _native as nat
from .api import DeviceCSR, Plan

DEFAULT_CACHE = os.path.join(os.path.expanduser("~"), ".cache", "paper_2112_10037_gb300", "autotune.json")

CANDIDATES = {
    "window_warp": [1024, 2048],
    "num_block_min": [8192, 32768, 65536, 131072],
    "window_block": [4096, 8192],
    "block_warps": [8, 16],
    "warp_max": [8192],
}

_lock = threading.Lock()


def _bucket(x: int) -> int:
    return int(math.log2(x)) if x > 0 else -1


def signature(A: DeviceCSR, B: DeviceCSR, dtype, stats) -> str:
    """Cache key: device, dtype and log2 size classes of the product."""
    dev = A.row_ptr.device
    props = torch.cuda.get_device_properties(dev)
    total, mx, _ = stats
    parts = [props.name.replace(" ", "_"), str(props.multi_processor_count), str(dtype).split(".")[-1],
             "r%d" % _bucket(A.nrows), "c%d" % _bucket(B.ncols), "a%d" % _bucket(A.nnz),
             "p%d" % _bucket(total), "m%d" % _bucket(mx)]
    return "|".join(parts)


def _load(path):
    try:
        with open(path) as fh:
            return json.load(fh)
    except (OSError, ValueError):
        return {}


def _store(path, data):
    d = os.path.dirname(path)
    if d:
        os.makedirs(d, exist_ok=True)
    tmp = path + ".tmp%d" % os.getpid()
    with open(tmp, "w") as fh:
        json.dump(data, fh, indent=1, sort_keys=True)
    os.replace(tmp, path)


def time_options(A: DeviceCSR, B: DeviceCSR, dtype=torch.float64, reps: int = 2, **opts) -> float:
    """Best-of-reps milliseconds of symbolic + numeric with these options."""
    best = float("inf")
    stream = torch.cuda.current_stream()
    for _ in range(reps):
        plan = Plan(A, B, dtype=dtype, **opts)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        plan.symbolic()
        plan.numeric(A.vals.to(dtype), B.vals.to(dtype))
        e1.record(stream)
        torch.cuda.synchronize()
        best = min(best, e0.elapsed_time(e1))
        plan.close()
    return best


def autotune(A: DeviceCSR, B: DeviceCSR, dtype=torch.float64, candidates=None, cache_path=DEFAULT_CACHE,
             reps: int = 2, refresh: bool = False) -> dict:
    """Best option set for C = A*B from ``candidates`` (a dict of option ->
    list of values; defaults to CANDIDATES), using and updating the cache."""
    probe = Plan(A, B, dtype=dtype)
    stats = probe.stats()
    probe.close()
    key = signature(A, B, dtype, stats)
    with _lock:
        cache = _load(cache_path) if cache_path else {}
    if not refresh and key in cache:
        return dict(cache[key]["options"])
    cand = candidates or CANDIDATES
    names = sorted(cand)
    results = []
    for values in itertools.product(*(cand[n] for n in names)):
        opts = dict(zip(names, values))
        results.append((time_options(A, B, dtype, reps, **opts), opts))
    results.sort(key=lambda t: t[0])
    best_ms, best = results[0]
    if cache_path:
        with _lock:
            cache = _load(cache_path)
            cache[key] = {"options": best, "ms": best_ms,
                          "tried": [{"options": o, "ms": t} for t, o in results]}
            _store(cache_path, cache)
    return dict(best)


def autotune_batch(pairs, dtype=torch.float64, candidates=None, cache_path=DEFAULT_CACHE, reps: int = 1,
                   refresh: bool = False) -> dict:
    """Best option set for a batch of products (timing the stacked batch's
    symbolic and numeric passes), cached under a key built from the batch's
    totals."""
    from .api import Batch
    a_nnz = sum(a.nnz for a, _ in pairs)
    rows = sum(a.nrows for a, _ in pairs)
    dev = pairs[0][0].row_ptr.device
    props = torch.cuda.get_device_properties(dev)
    key = "|".join([props.name.replace(" ", "_"), str(props.multi_processor_count), str(dtype).split(".")[-1],
                    "batch", "n%d" % _bucket(len(pairs)), "r%d" % _bucket(rows), "a%d" % _bucket(a_nnz)])
    with _lock:
        cache = _load(cache_path) if cache_path else {}
    if not refresh and key in cache:
        return dict(cache[key]["options"])
    cand = candidates or CANDIDATES
    names = sorted(cand)
    results = []
    stream = torch.cuda.current_stream()
    for values in itertools.product(*(cand[n] for n in names)):
        opts = dict(zip(names, values))
        best = float("inf")
        for _ in range(reps):
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            b = Batch(pairs, dtype=dtype, **opts)
            b.symbolic()
            b.numeric()
            e1.record(stream)
            torch.cuda.synchronize()
            best = min(best, e0.elapsed_time(e1))
            b.close()
        results.append((best, opts))
    results.sort(key=lambda t: t[0])
    if cache_path:
        with _lock:
            cache = _load(cache_path)
            cache[key] = {"options": results[0][1], "ms": results[0][0],
                          "tried": [{"options": o, "ms": t} for t, o in results]}
            _store(cache_path, cache)
    return dict(results[0][1])
