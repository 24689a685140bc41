"""Batched matching (one pipeline pass over many instances) against the oracle."""
import numpy as np
import pytest

import oracle
import synth
from tests.gpu_util import to_dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    import paper_1703_06680_gb300 as ddm
    ddm.build_library()
    c = ddm.Context(0)
    yield c
    c.close()


def check_batch(ctx, regs, sample=None):
    insts = [to_dev(r) for r in regs]
    pairs, offs = ctx.match_batch(insts)
    pairs = pairs.cpu().numpy()
    assert offs[0] == 0 and offs[-1] == len(pairs)
    assert np.all(np.diff(offs.astype(np.int64)) >= 0)
    idx = range(len(regs)) if sample is None else sample
    for b in idx:
        want = oracle.sbm(regs[b])
        got = pairs[int(offs[b]):int(offs[b + 1])]
        assert np.array_equal(got, want), b
    _, offs2 = ctx.match_batch(insts, count_only=True)
    assert np.array_equal(offs, offs2)
    return pairs, offs


@pytest.mark.parametrize("d", [1, 2, 3])
def test_batch_mixed_sizes(ctx, d):
    rng = np.random.default_rng(100 + d)
    regs = []
    for b in range(150):
        n, m = int(rng.integers(0, 400)), int(rng.integers(0, 400))
        N = max(n + m, 1)
        regs.append(synth.make_regions(d, n, m, synth.side_for(float(rng.choice([0.01, 1, 100])),
                                                               N, d), 1000 * d + b))
    check_batch(ctx, regs)


@pytest.mark.parametrize("d,mixed", [(2, False), (2, True), (3, False), (3, True)])
def test_batch_write_modes_agree(d, mixed):
    # The survivor path (one sort of the recorded pairs, unpacked to ids local to
    # each instance) and the write pass give the same pairs and offsets, with
    # empty instances and instances without subscriptions or updates among them.
    # At one density the survivors' room (sized from the average K / n) suffices;
    # with mixed densities dense windows may overflow it and fall back.
    import paper_1703_06680_gb300 as ddm
    rng = np.random.default_rng(300 + d + 10 * mixed)
    regs = []
    for b in range(120):
        n, m = int(rng.integers(0, 300)), int(rng.integers(0, 300))
        if b % 17 == 0:
            n = 0
        if b % 19 == 0:
            m = 0
        N = max(n + m, 1)
        alpha = float(rng.choice([0.01, 1, 100])) if mixed else 1.0
        regs.append(synth.make_regions(d, n, m, synth.side_for(alpha, N, d), 7000 * d + b))
    insts = [to_dev(r) for r in regs]
    got = {}
    with ddm.Context(0) as c:
        for mode in (1, 2):
            c.set_param(ddm._lib.PARAM_ND_WRITE, mode)
            s0 = c.stats()["survivor_calls"]
            pairs, offs = c.match_batch(insts)
            got[mode] = (pairs.cpu().numpy(), np.asarray(offs))
            used = c.stats()["survivor_calls"] > s0
            assert (not used) if mode == 1 else (used or mixed)
    assert np.array_equal(got[1][0], got[2][0]) and np.array_equal(got[1][1], got[2][1])
    offs = got[2][1]
    for b, r in enumerate(regs):
        assert np.array_equal(got[2][0][int(offs[b]):int(offs[b + 1])], oracle.sbm(r)), b


def test_batch_dense_ties(ctx):
    from tests.helpers import tiny_grid_instance
    rng = np.random.default_rng(7)
    regs = [tiny_grid_instance(rng, 1 + b % 3, int(rng.integers(0, 50)), int(rng.integers(0, 50)))
            for b in range(99)]
    # all instances of one call share d: split by d
    for d in (1, 2, 3):
        check_batch(ctx, [r for r in regs if r.d == d])


def test_batch_equals_plain_calls(ctx):
    regs = synth.batch_instances(num=64, d=2)
    pairs, offs = check_batch(ctx, regs, sample=range(0, 64, 8))
    for b in range(64):
        assert ctx.count(*to_dev(regs[b])) == int(offs[b + 1] - offs[b])


def test_batch_capacity(ctx):
    import paper_1703_06680_gb300 as ddm
    regs = [synth.small_1d(), synth.small_1d(1)]
    insts = [to_dev(r) for r in regs]
    _, offs = ctx.match_batch(insts, count_only=True)
    with pytest.raises(ddm.CapacityError) as e:
        ctx.match_batch(insts, cap=int(offs[-1]) - 1)
    assert e.value.K == int(offs[-1])


def test_batch_full_size_every_instance(ctx):
    # The 4096-instance workload (d=2, alpha=1, N_i log-uniform in [1e2, 1e5]):
    # every instance's pair list compared whole with the oracle's (oracle runs
    # spread over the host cores in a spawn pool).
    from tests.oracle_pool import check_batch as pool_check
    regs = synth.batch_instances(num=4096, d=2)
    insts = [to_dev(r) for r in regs]
    del regs
    pairs, offs = ctx.match_batch(insts)
    assert pool_check(pairs, offs.astype(np.int64), 4096, d=2, alpha=1.0) == len(pairs)
    _, offs2 = ctx.match_batch(insts, count_only=True)
    assert np.array_equal(offs, offs2)


@pytest.mark.parametrize("d", [1, 2])
def test_autotune_on_gpu_keeps_results(tmp_path, d):
    # The tuner times every candidate through the library; whatever it picks,
    # results stay identical to the oracle's, and the cache re-applies it.
    import paper_1703_06680_gb300 as ddm
    from paper_1703_06680_gb300 import autotune
    ddm.build_library()
    reg = synth.large_1d(1.0, N=100_000) if d == 1 else synth.large_nd(2, 1.0, N=60_000)
    want = oracle.sbm(reg)
    t = to_dev(reg)
    cache = str(tmp_path / "tune.json")
    with ddm.Context(0) as ctx:
        chosen = autotune.tune(ctx, t, reps=2, cache_path=cache)
        name = "win_shift" if d == 1 else "nd_path"
        assert chosen[name] in autotune.CANDIDATES[
            autotune.PARAM_WIN_SHIFT if d == 1 else autotune.PARAM_ND_PATH]
        # the tile parameters are tuned too, and cached with the rest
        assert chosen["sort_items"] in autotune.CANDIDATES[autotune.PARAM_SORT_ITEMS]
        if d > 1:
            assert chosen["join_shift"] in autotune.CANDIDATES[autotune.PARAM_JOIN_SHIFT]
        entry = autotune._load(cache)[chosen["key"]]
        assert entry["sort_items"] == chosen["sort_items"]
        assert np.array_equal(ctx.match(*t).cpu().numpy(), want)
    with ddm.Context(0) as ctx2:
        assert autotune.apply_cached(ctx2, t, cache_path=cache)
        assert np.array_equal(ctx2.match(*t).cpu().numpy(), want)
