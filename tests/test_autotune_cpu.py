"""Autotuner logic on CPU: workload classes, choice of the fastest candidate,
the JSON cache, and applying cached values (fake context and timer)."""
import json

import numpy as np

from paper_1703_06680_gb300 import autotune
from paper_1703_06680_gb300._lib import (PARAM_JOIN_SHIFT, PARAM_ND_PATH, PARAM_SORT_ITEMS,
                                         PARAM_WIN_SHIFT)


class FakeCtx:
    def __init__(self, K):
        self.K = K
        self.params = {}
        self.calls = []
        self.device = 0

    def count(self, *t):
        return self.K

    def set_param(self, p, v):
        self.params[p] = v
        self.calls.append((p, v))


def tensors(d, n, m):
    return [np.zeros((d, n), np.float32), np.zeros((d, n), np.float32),
            np.zeros((d, m), np.float32), np.zeros((d, m), np.float32)]


def test_workload_key_buckets():
    assert autotune.workload_key("G", 1, 1_000_000, 50_000_000) == "G|d1|n19|k5"
    assert autotune.workload_key("G", 2, 1_000_000, 0) == "G|d2|n19|k-99"
    assert autotune.workload_key("G", 1, 1024, 1024) == autotune.workload_key("G", 1, 2047, 2047)
    assert autotune.workload_key("G", 1, 1024, 10) != autotune.workload_key("G", 1, 1024, 5000)


def test_tune_picks_fastest_and_caches(tmp_path):
    cache = tmp_path / "tune.json"
    ctx = FakeCtx(K=1000)
    fake_ms = {8: 3.0, 9: 1.0, 10: 2.0}
    items_ms = {12: 0.5, 16: 0.2, 18: 0.4}

    def timer(c, t, K, reps):   # defaults for tunables not set yet (18 items, window 10)
        return fake_ms[c.params.get(PARAM_WIN_SHIFT, 10)] + items_ms[c.params.get(PARAM_SORT_ITEMS, 18)]

    chosen = autotune.tune(ctx, tensors(1, 100, 100), cache_path=str(cache), gpu="G", timer=timer)
    assert chosen["win_shift"] == 9 and ctx.params[PARAM_WIN_SHIFT] == 9
    assert chosen["sort_items"] == 16 and ctx.params[PARAM_SORT_ITEMS] == 16
    assert PARAM_ND_PATH not in ctx.params            # d = 1: no d > 1 strategy
    assert PARAM_JOIN_SHIFT not in ctx.params
    stored = json.loads(cache.read_text())
    assert stored[chosen["key"]]["win_shift"] == 9
    assert stored[chosen["key"]]["win_shift_ms"] == {"8": 3.2, "9": 1.2, "10": 2.2}
    assert stored[chosen["key"]]["sort_items"] == 16

    fresh = FakeCtx(K=1000)
    assert autotune.apply_cached(fresh, tensors(1, 100, 100), cache_path=str(cache), gpu="G")
    assert fresh.params == {PARAM_WIN_SHIFT: 9, PARAM_SORT_ITEMS: 16}
    # another workload class or GPU: nothing cached
    assert not autotune.apply_cached(FakeCtx(K=10**6), tensors(1, 100, 100),
                                     cache_path=str(cache), gpu="G")
    assert not autotune.apply_cached(FakeCtx(K=1000), tensors(1, 100, 100),
                                     cache_path=str(cache), gpu="H")


def test_tune_d2_uses_strategy_only_and_merges_cache(tmp_path):
    cache = tmp_path / "tune.json"
    cache.write_text(json.dumps({"other": {"win_shift": 7}}))
    ctx = FakeCtx(K=500)

    def timer(c, t, K, reps):
        return ({1: 5.0, 2: 4.0}[c.params[PARAM_ND_PATH]]
                + {9: 1.0, 10: 0.5, 11: 2.0}[c.params.get(PARAM_JOIN_SHIFT, 11)])

    chosen = autotune.tune(ctx, tensors(2, 50, 60), cache_path=str(cache), gpu="G", timer=timer)
    assert chosen["nd_path"] == 2 and "win_shift" not in chosen
    assert chosen["join_shift"] == 10 and ctx.params[PARAM_JOIN_SHIFT] == 10
    assert chosen["sweep_dim"] == 0                   # equal times: the first candidate
    stored = json.loads(cache.read_text())
    assert stored["other"] == {"win_shift": 7}       # earlier entries kept
    assert stored[chosen["key"]]["nd_path"] == 2
