"""Autotuner: cache bookkeeping on the CPU; on the GPU, that tuning picks a
candidate, reuses the cache, and that the tuned options still give the
oracle's product."""
import json
import os

import numpy as np
import pytest

from paper_2112_10037_gb300 import gen


def test_cache_roundtrip(tmp_path):
    pytest.importorskip("torch")
    from paper_2112_10037_gb300 import autotune as at
    p = str(tmp_path / "sub" / "cache.json")
    assert at._load(p) == {}
    at._store(p, {"k": {"options": {"window_warp": 1024}, "ms": 1.0}})
    assert at._load(p)["k"]["options"]["window_warp"] == 1024
    assert at._bucket(0) == -1 and at._bucket(1) == 0 and at._bucket(1024) == 10 and at._bucket(1025) == 10


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
    cand = {"window_warp": [1024, 2048], "split_min": [4096, -1], "warp_max": [8192]}
    best = at.autotune(dA, dA, candidates=cand, cache_path=cache, reps=1)
    assert best["window_warp"] in (1024, 2048) and best["split_min"] in (4096, -1)
    data = json.load(open(cache))
    assert len(data) == 1 and len(list(data.values())[0]["tried"]) == 4
    again = at.autotune(dA, dA, candidates=cand, cache_path=cache, reps=1)
    assert again == best
    C = api.spgemm(dA, dA, **best).to_host()
    R = oracle_mod.spgemm(A, A)
    assert np.array_equal(C.col_idx, R.col_idx)
    assert np.allclose(C.vals, R.vals, rtol=1e-12, atol=0)
