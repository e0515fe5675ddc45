"""Autotuner for the SpGEMM plan options.

It replaces the paper's analytical choice of architecture parameters
(Sec. 4.2.4, Eq. 3: SW and NUM_PE solved from the FPGA's resource limits)
with measurement on this GPU.  The options it picks, per product:

* the accumulator of the short rows, by bin: the warp hash table for rows of
  17 .. hash_max products (32, 64 or 128), with dense column windows above,
  or no hash table at all and the register sort up to sort_max products
  (128 or 256) -- the dense-versus-hash choice per bin;
* the product count above which rows take the rank-compacted accumulator
  (a presence bitmap ranks the output columns, values sit in an array of the
  row's outputs) instead of the warp's dense column windows;
* the numeric window width of a warp (columns per dense accumulator);
* the product count above which rows take the block-wide window, that
  window's width and the number of warps sharing it;
* the product count at which the symbolic pass switches from one warp to a
  whole block per row;
* optionally the split of heavy rows into window tiles.

Each candidate option set is timed on the product itself (symbolic and
numeric passes, CUDA events on the current stream, best of ``reps``).  The
search is coordinate descent: starting from the library defaults, each
option group in turn tries its candidates with the others held at the best
values found so far, for ``sweeps`` sweeps (the exhaustive product of all
candidates is available as ``strategy="grid"``).  Winners are cached in a
JSON file keyed by the GPU (name, SM count), the value type and a size class
of the product (log2 buckets of rows, nnz(A) and total and largest row
product counts), so products of the same shape reuse the choice.

The cache holds only option values and timings, never results of the
product.
"""
from __future__ import annotations

import itertools
import json
import math
import os
import threading

import torch

from .api import DeviceCSR, Plan

DEFAULT_CACHE = os.path.join(os.path.expanduser("~"), ".cache", "paper_2112_10037_gb300", "autotune.json")

# Option groups and their candidates.  A candidate is a value of the option
# named by the key, or a dict of several options set together.
SMALL_ROW_ACCUMULATORS = [
    {"hash_max": 128, "sort_max": 128},   # hash table for 17..128 products (default)
    {"hash_max": 64, "sort_max": 128},    # hash for 17..64, dense windows above
    {"hash_max": 32, "sort_max": 128},    # hash for 17..32, dense windows above
    {"hash_max": -1, "sort_max": 128},    # no hash: register sort up to 128
    {"hash_max": -1, "sort_max": 256},    # no hash: register sort up to 256
]

CANDIDATES = {
    "accumulator": SMALL_ROW_ACCUMULATORS,
    "window_warp": [1024, 2048],
    "num_block_min": [8192, 32768, 65536, 131072],
    "block_window": [{"window_block": 8192, "block_warps": 8}, {"window_block": 4096, "block_warps": 8},
                     {"window_block": 8192, "block_warps": 16}, {"window_block": 16384, "block_warps": 16}],
    "warp_max": [4096, 8192, 16384],
    "rank_min": [-1, 256, 1024, 4096],
}

# Starting point of the coordinate search: the library's defaults.
DEFAULTS = {"accumulator": SMALL_ROW_ACCUMULATORS[0], "window_warp": 1024, "num_block_min": 65536,
            "block_window": {"window_block": 8192, "block_warps": 8}, "warp_max": 8192, "rank_min": -1}

_lock = threading.Lock()


def _bucket(x: int) -> int:
    return int(math.log2(x)) if x > 0 else -1


def expand(choice: dict) -> dict:
    """Plan keyword options of a choice {group: candidate}."""
    out = {}
    for name in sorted(choice):
        v = choice[name]
        if isinstance(v, dict):
            out.update(v)
        else:
            out[name] = v
    return out


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


def search(cand: dict, timer, strategy: str = "coordinate", sweeps: int = 2, start=None):
    """Best choice {group: candidate} by ``timer(options) -> ms`` over the
    candidates ``cand`` ({group: [candidates]}).  Returns (best_ms, choice,
    tried), tried being the list of (ms, choice) timed, each distinct option
    set timed once."""
    names = sorted(cand)
    seen = {}

    def measure(choice):
        key = json.dumps(expand(choice), sort_keys=True)
        if key not in seen:
            seen[key] = (timer(expand(choice)), dict(choice))
        return seen[key][0]

    if strategy == "grid":
        for values in itertools.product(*(cand[n] for n in names)):
            measure(dict(zip(names, values)))
    elif strategy == "coordinate":
        cur = {}
        for n in names:
            s = (start or DEFAULTS).get(n)
            cur[n] = s if s in cand[n] else cand[n][0]
        best = measure(cur)
        for _ in range(max(1, sweeps)):
            changed = False
            for n in names:
                for v in cand[n]:
                    trial = dict(cur)
                    trial[n] = v
                    t = measure(trial)
                    if t < best:
                        best, cur, changed = t, trial, True
            if not changed:
                break
    else:
        raise ValueError("strategy must be 'coordinate' or 'grid'")
    tried = sorted(seen.values(), key=lambda tc: tc[0])
    return tried[0][0], tried[0][1], tried


def time_options(A: DeviceCSR, B: DeviceCSR, dtype=torch.float64, reps: int = 2, **opts) -> float:
    """Best-of-reps milliseconds of symbolic + numeric with these options."""
    best = float("inf")
    stream = torch.cuda.current_stream()
    av, bv = A.vals.to(dtype), B.vals.to(dtype)
    for _ in range(reps):
        plan = Plan(A, B, dtype=dtype, **opts)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        plan.symbolic()
        plan.numeric(av, bv)
        e1.record(stream)
        torch.cuda.synchronize()
        best = min(best, e0.elapsed_time(e1))
        plan.close()
    return best


def _tune(key, cand, timer, cache_path, refresh, strategy, sweeps):
    with _lock:
        cache = _load(cache_path) if cache_path else {}
    if not refresh and key in cache:
        return dict(cache[key]["options"])
    best_ms, best, tried = search(cand, timer, strategy=strategy, sweeps=sweeps)
    opts = expand(best)
    if cache_path:
        with _lock:
            cache = _load(cache_path)
            cache[key] = {"options": opts, "ms": best_ms, "strategy": strategy,
                          "tried": [{"options": expand(c), "ms": t} for t, c in tried]}
            _store(cache_path, cache)
    return dict(opts)


def autotune(A: DeviceCSR, B: DeviceCSR, dtype=torch.float64, candidates=None, cache_path=DEFAULT_CACHE,
             reps: int = 2, refresh: bool = False, strategy: str = "coordinate", sweeps: int = 2) -> dict:
    """Best plan options for C = A*B from ``candidates`` (a dict of option
    group -> list of candidates; defaults to CANDIDATES), using and updating
    the cache.  Returns keyword options for ``Plan`` / ``spgemm``."""
    probe = Plan(A, B, dtype=dtype)
    stats = probe.stats()
    probe.close()
    key = signature(A, B, dtype, stats)
    return _tune(key, candidates or CANDIDATES, lambda o: time_options(A, B, dtype, reps, **o), cache_path,
                 refresh, strategy, sweeps)


def time_batch(pairs, dtype=torch.float64, reps: int = 1, **opts) -> float:
    """Best-of-reps milliseconds of a batch's analysis, symbolic and numeric
    passes with these options."""
    from .api import Batch
    stream = torch.cuda.current_stream()
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
    return best


def batch_signature(pairs, dtype) -> str:
    a_nnz = sum(a.nnz for a, _ in pairs)
    rows = sum(a.nrows for a, _ in pairs)
    dev = pairs[0][0].row_ptr.device
    props = torch.cuda.get_device_properties(dev)
    return "|".join([props.name.replace(" ", "_"), str(props.multi_processor_count), str(dtype).split(".")[-1],
                     "batch", "n%d" % _bucket(len(pairs)), "r%d" % _bucket(rows), "a%d" % _bucket(a_nnz)])


def autotune_batch(pairs, dtype=torch.float64, candidates=None, cache_path=DEFAULT_CACHE, reps: int = 1,
                   refresh: bool = False, strategy: str = "coordinate", sweeps: int = 1) -> dict:
    """Best option set for a batch of products (timing the stacked batch's
    symbolic and numeric passes), cached under a key built from the batch's
    totals."""
    key = batch_signature(pairs, dtype)
    return _tune(key, candidates or CANDIDATES, lambda o: time_batch(pairs, dtype, reps, **o), cache_path,
                 refresh, strategy, sweeps)
