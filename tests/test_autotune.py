"""Autotuner: the search and cache bookkeeping on the CPU (with a synthetic
timer standing in for the GPU timings); on the GPU, that tuning over the
accumulator choice per bin (hash versus dense windows versus register sort)
and the window options picks a candidate, reuses the cache, and that the
tuned options still give the oracle's product."""
import json

import numpy as np
import pytest

from paper_2112_10037_gb300 import gen


def _at():
    pytest.importorskip("torch")
    from paper_2112_10037_gb300 import autotune as at
    return at


def test_cache_roundtrip(tmp_path):
    at = _at()
    p = str(tmp_path / "sub" / "cache.json")
    assert at._load(p) == {}
    at._store(p, {"k": {"options": {"window_warp": 1024}, "ms": 1.0}})
    assert at._load(p)["k"]["options"]["window_warp"] == 1024
    assert at._bucket(0) == -1 and at._bucket(1) == 0 and at._bucket(1024) == 10 and at._bucket(1025) == 10


def test_candidates_cover_the_accumulator_choice():
    at = _at()
    accs = at.CANDIDATES["accumulator"]
    hash_max = sorted({a["hash_max"] for a in accs if a["sort_max"] == 128 and a["hash_max"] > 0})
    assert hash_max == [32, 64, 128]
    assert {"hash_max": -1, "sort_max": 128} in accs and {"hash_max": -1, "sort_max": 256} in accs
    assert at.DEFAULTS["accumulator"] == {"hash_max": 128, "sort_max": 128}
    for group, values in at.CANDIDATES.items():
        assert at.DEFAULTS[group] in values, group
    opts = at.expand(at.DEFAULTS)
    assert opts["hash_max"] == 128 and opts["window_block"] == 8192 and opts["block_warps"] == 8


def _separable_cost(opts):
    """A cost whose minimum is known: each option contributes on its own."""
    cost = {1024: 3.0, 2048: 1.0}[opts["window_warp"]]
    cost += {128: 2.0, 64: 0.5, 32: 1.5, -1: 4.0}[opts["hash_max"]] + (0.1 if opts["sort_max"] == 256 else 0.0)
    cost += {8192: 2.0, 32768: 1.0, 65536: 0.2, 131072: 0.7}[opts["num_block_min"]]
    return cost


def test_coordinate_search_finds_separable_minimum():
    at = _at()
    cand = {k: at.CANDIDATES[k] for k in ("accumulator", "window_warp", "num_block_min")}
    calls = []

    def timer(o):
        calls.append(dict(o))
        return _separable_cost(o)

    best_ms, best, tried = at.search(cand, timer, strategy="coordinate", sweeps=2)
    opts = at.expand(best)
    assert opts["window_warp"] == 2048 and opts["hash_max"] == 64 and opts["num_block_min"] == 65536
    assert best_ms == pytest.approx(1.0 + 0.5 + 0.2)
    grid = 1
    for v in cand.values():
        grid *= len(v)
    assert len(calls) < grid  # far fewer timings than the exhaustive product
    assert len({json.dumps(c, sort_keys=True) for c in calls}) == len(calls)  # each option set timed once
    g_ms, g_best, g_tried = at.search(cand, _separable_cost, strategy="grid")
    assert len(g_tried) == grid and g_ms == pytest.approx(best_ms) and at.expand(g_best) == opts


def test_tune_uses_cache(tmp_path):
    at = _at()
    cache = str(tmp_path / "tune.json")
    cand = {"window_warp": [1024, 2048], "accumulator": at.SMALL_ROW_ACCUMULATORS}
    n = []

    def timer(o):
        n.append(1)
        return _separable_cost(dict(o, num_block_min=65536))

    first = at._tune("key", cand, timer, cache, False, "coordinate", 2)
    k = len(n)
    again = at._tune("key", cand, timer, cache, False, "coordinate", 2)
    assert again == first and len(n) == k
    data = json.load(open(cache))
    assert data["key"]["options"] == first and data["key"]["strategy"] == "coordinate"
    at._tune("key", cand, timer, cache, True, "coordinate", 2)
    assert len(n) == 2 * k


@pytest.mark.gpu
def test_autotune_picks_and_caches(tmp_path, oracle_mod):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2112_10037_gb300 import build
    build.build()
    from paper_2112_10037_gb300 import api, autotune as at
    A = gen.rmat(12, 16)
    dA = api.DeviceCSR.from_host(A)
    cache = str(tmp_path / "tune.json")
    cand = {"window_warp": [1024, 2048], "split_min": [4096, -1], "warp_max": [8192],
            "accumulator": at.SMALL_ROW_ACCUMULATORS}
    best = at.autotune(dA, dA, candidates=cand, cache_path=cache, reps=1)
    assert best["window_warp"] in (1024, 2048) and best["split_min"] in (4096, -1)
    assert {"hash_max": best["hash_max"], "sort_max": best["sort_max"]} in at.SMALL_ROW_ACCUMULATORS
    data = json.load(open(cache))
    tried = list(data.values())[0]["tried"]
    assert len(data) == 1 and 5 <= len(tried) <= 2 * 2 * 5
    again = at.autotune(dA, dA, candidates=cand, cache_path=cache, reps=1)
    assert again == best
    R = oracle_mod.spgemm(A, A)
    for acc in at.SMALL_ROW_ACCUMULATORS:  # every accumulator choice gives the same product
        C = api.spgemm(dA, dA, **dict(best, **acc)).to_host()
        assert np.array_equal(C.row_ptr.astype(np.int64), R.row_ptr)
        assert np.array_equal(C.col_idx, R.col_idx)
        assert np.allclose(C.vals, R.vals, rtol=1e-12, atol=0)
