"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle.

Results are integer pair lists, so the bar is bit-exact equality of the
sorted (sub, upd) lists.  Every workload is compared in full: where the serial
oracle takes minutes, it runs on subscription slices in a pool of host
processes (tests/oracle_pool.py), each slice checked against its rows.
"""
import numpy as np
import pytest

import oracle
import synth
from tests.gpu_util import gpu_pairs, to_dev
from tests.helpers import special_value_instance, tiny_grid_instance

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    import paper_1703_06680_gb300 as ddm
    ddm.build_library()
    c = ddm.Context(0)
    yield c
    c.close()


def assert_parity(ctx, reg, want=None):
    if want is None:
        want = oracle.sbm(reg)
    got = gpu_pairs(ctx, reg)
    assert got.shape == want.shape, (got.shape, want.shape)
    assert np.array_equal(got, want)
    assert ctx.count(*to_dev(reg)) == len(want)


# --- the workloads --------------------------------------------------------------

def test_small_1d(ctx):
    assert_parity(ctx, synth.small_1d())


@pytest.mark.parametrize("alpha", [0.01, 1.0, 100.0])
def test_large_1d_full(ctx, alpha):
    assert_parity(ctx, synth.large_1d(alpha))


@pytest.mark.parametrize("d,alpha", [(2, 1.0), (2, 100.0), (3, 1.0), (3, 100.0)])
def test_nd_reduced_full(ctx, d, alpha):
    # N = 1e5: the oracle finishes in seconds; many tiles and ragged tails
    assert_parity(ctx, synth.large_nd(d, alpha, N=100_003))


def test_d2_alpha1_full_size(ctx):
    assert_parity(ctx, synth.large_nd(2, 1.0))


@pytest.mark.parametrize("d,alpha", [(2, 100.0), (3, 1.0), (3, 100.0)])
def test_nd_full_size_complete(ctx, d, alpha):
    # N = 1e6 at d = 2 and 3: the complete sorted pair list (up to 1.9e8 pairs)
    # against the oracle, run on 64 subscription slices x all updates in a spawn
    # pool; the slices' oracle counts add up to the whole instance's K.
    import torch
    from tests.oracle_pool import check_full
    reg = synth.large_nd(d, alpha)
    t = to_dev(reg)
    K = ctx.count(*t)
    pairs = ctx.match(*t, cap=K)
    assert pairs.shape[0] == K
    assert check_full(pairs, ("large_nd", (d, alpha)), reg.n) == K
    # swapping the roles of S and U gives the same count
    assert ctx.count(t[2], t[3], t[0], t[1]) == K
    del pairs
    torch.cuda.empty_cache()


def test_d1_beyond_the_scan_counter_limits(ctx):
    # N = 9e6 (E = 1.8e7 endpoints, n = 4.5e6): more than 4096 scan tiles and more
    # than 2048 subscription-id tiles, so the sweep and the offsets scan take their
    # decoupled look-backs instead of the tile counters that the sort and the sweep
    # form below those sizes (and the sort its flat scan); the complete pair list
    # against the oracle, pooled.
    import torch
    from tests.oracle_pool import check_full
    N = 9_000_000
    reg = synth.large_1d(1.0, 0, N)
    t = to_dev(reg)
    K = ctx.count(*t)
    pairs = ctx.match(*t, cap=K)
    assert pairs.shape[0] == K
    assert check_full(pairs, ("large_1d", (1.0, 0, N)), reg.n) == K
    del pairs
    torch.cuda.empty_cache()


# --- the sweep stages (a1-a4) against the oracle's Algorithm 4 trace --------------

def test_sweep_stages_match_oracle_trace(ctx):
    reg = synth.make_regions(1, 30_011, 29_989, 40.0, 99)  # dense float32 ties near 1e6
    who, ss, us, sc, uc = [x.cpu().numpy().view(np.uint32).astype(np.int64)
                           for x in ctx.debug_sweep(*to_dev(reg))]
    kind, ids, oss, ous = oracle.sweep_trace(reg)
    assert np.array_equal(who >> 30, kind.astype(np.int64))
    assert np.array_equal(who & ((1 << 30) - 1), ids.astype(np.int64))
    assert np.array_equal(ss, oss) and np.array_equal(us, ous)
    pairs = oracle.sbm(reg)
    assert np.array_equal(sc, oracle.per_sub_counts(pairs, reg.n))
    assert np.array_equal(uc, oracle.per_upd_counts(pairs, reg.m))


# --- adversarial and edge cases ------------------------------------------------------

def test_tiny_grid_instances(ctx):
    rng = np.random.default_rng(11)
    for s in range(300):
        d = 1 + s % 3
        reg = tiny_grid_instance(rng, d, int(rng.integers(0, 70)), int(rng.integers(0, 70)))
        assert_parity(ctx, reg)


def test_special_values(ctx):
    rng = np.random.default_rng(12)
    for s in range(100):
        reg = special_value_instance(rng, 1 + s % 3, int(rng.integers(1, 300)),
                                     int(rng.integers(1, 300)))
        assert_parity(ctx, reg)


@pytest.mark.parametrize("n,m", [(0, 10), (10, 0), (0, 0), (1, 1), (4097, 1), (1, 4097),
                                 (2049, 2047)])
def test_empty_and_ragged(ctx, n, m):
    reg = synth.make_regions(1, n, m, 5000.0, 5 + n + m) if n + m else \
        synth.Regions(*(np.zeros((1, 0), np.float32) for _ in range(4)))
    assert_parity(ctx, reg)


def test_all_identical_long_segments(ctx):
    # every pair matches: 3000 x 2500 pairs, segments far above one warp's sort
    reg = synth.Regions(np.full((1, 3000), 1.0, np.float32), np.full((1, 3000), 2.0, np.float32),
                        np.full((1, 2500), 2.0, np.float32), np.full((1, 2500), 3.0, np.float32))
    assert_parity(ctx, reg)


def test_one_huge_interval(ctx):
    reg = synth.large_1d(1.0, N=200_000)
    reg.sub_lo[0, 17] = -1.0
    reg.sub_hi[0, 17] = 2.0e6
    reg.upd_lo[0, 5] = -np.inf
    reg.upd_hi[0, 5] = np.inf
    assert_parity(ctx, reg)


def test_mixed_lengths_2d(ctx):
    rng = np.random.default_rng(13)
    n, m = 20_000, 30_000
    def ext(c):
        lo = (rng.random((2, c)) * 1e5).astype(np.float32)
        side = np.exp(rng.normal(4.0, 2.0, size=(2, c))).astype(np.float32)
        return lo, (lo + side).astype(np.float32)
    reg = synth.Regions(*ext(n), *ext(m))
    assert_parity(ctx, reg)


@pytest.mark.parametrize("where", ["nan_dim0", "reversed_dim0", "nan_dim1", "reversed_dim2"])
def test_invalid_input(ctx, where):
    import paper_1703_06680_gb300 as ddm
    reg = synth.make_regions(3, 100, 100, 1e4, 3)
    if where == "nan_dim0":
        reg.upd_lo[0, 7] = np.nan
    elif where == "reversed_dim0":
        reg.sub_lo[0, 3] = reg.sub_hi[0, 3] + 1
    elif where == "nan_dim1":
        reg.sub_hi[1, 9] = np.nan
    else:
        reg.upd_lo[2, 0] = reg.upd_hi[2, 0] + 5
    t = to_dev(reg)
    with pytest.raises(ddm.DDMError) as e:
        ctx.count(*t)
    assert e.value.code == -1
    with pytest.raises(ddm.DDMError):
        ctx.match(*t, cap=10_000)
    # the context stays usable
    assert_parity(ctx, synth.make_regions(1, 50, 60, 1e4, 4))


def test_capacity_error_reports_K(ctx):
    import paper_1703_06680_gb300 as ddm
    reg = synth.small_1d()
    want = oracle.sbm(reg)
    with pytest.raises(ddm.CapacityError) as e:
        ctx.match(*to_dev(reg), cap=len(want) - 1)
    assert e.value.K == len(want)


def test_host_buffers_match_device(ctx):
    reg = synth.large_1d(1.0, N=300_000)
    want = oracle.sbm(reg)
    got = ctx.match_host(reg.sub_lo, reg.sub_hi, reg.upd_lo, reg.upd_hi, cap=len(want) + 5)
    assert np.array_equal(got, want)


def test_deterministic(ctx):
    reg = synth.large_nd(2, 100.0, N=60_000)
    a = gpu_pairs(ctx, reg)
    b = gpu_pairs(ctx, reg)
    assert np.array_equal(a, b)


# --- both d > 1 strategies (tiled join, range expansion) against the oracle -----------

@pytest.fixture(scope="module", params=[1, 2], ids=["join", "ranges"])
def ctx_path(request):
    import paper_1703_06680_gb300 as ddm
    ddm.build_library()
    c = ddm.Context(0)
    c.set_param(ddm._lib.PARAM_ND_PATH, request.param)
    yield c
    c.close()


@pytest.mark.parametrize("d,alpha", [(2, 1.0), (2, 100.0), (3, 1.0), (3, 100.0)])
def test_nd_paths_reduced(ctx_path, d, alpha):
    assert_parity(ctx_path, synth.large_nd(d, alpha, N=60_001))


def test_nd_paths_tiny_and_mixed(ctx_path):
    rng = np.random.default_rng(21)
    for s in range(120):
        d = 2 + s % 2
        reg = tiny_grid_instance(rng, d, int(rng.integers(0, 70)), int(rng.integers(0, 70)))
        assert_parity(ctx_path, reg)
    n, m = 15_000, 12_000
    def ext(c):
        lo = (rng.random((3, c)) * 1e5).astype(np.float32)
        side = np.exp(rng.normal(5.0, 2.0, size=(3, c))).astype(np.float32)
        return lo, (lo + side).astype(np.float32)
    assert_parity(ctx_path, synth.Regions(*ext(n), *ext(m)))


@pytest.mark.parametrize("d,alpha", [(1, 100.0), (1, 0.01), (2, 1.0), (3, 100.0)])
def test_pdl_off_and_profiling_modes(d, alpha):
    # Programmatic dependent launch and the stage events change only timing:
    # every combination gives the oracle's result.
    import paper_1703_06680_gb300 as ddm
    reg = synth.large_1d(alpha, N=200_001) if d == 1 else synth.large_nd(d, alpha, N=60_001)
    want = oracle.sbm(reg)
    c = ddm.Context(0)
    try:
        for pdl in (0, 1):
            c.set_param(ddm.PARAM_PDL, pdl)
            for prof in ("off", "all", "emit", "sort"):
                if prof == "off":
                    c.set_profiling(False)
                elif prof == "all":
                    c.set_profiling(True)
                else:
                    stage = "emit" if prof == "emit" else "radix_sort"
                    c.set_profiling(True, stage=ddm.STAGE_NAMES.index(stage))
                got = gpu_pairs(c, reg)
                assert np.array_equal(got, want), (pdl, prof)
                st = c.stats()["stage_ms"]
                if prof in ("emit", "sort"):
                    stage = "emit" if prof == "emit" else "radix_sort"
                    assert st[stage] > 0
                    assert all(v == 0 for k, v in st.items() if k != stage)
        with pytest.raises(ddm.DDMError):
            c.set_param(ddm.PARAM_PDL, 2)
        with pytest.raises(ddm.DDMError):
            c.set_profiling(True, stage=len(ddm.STAGE_NAMES))
    finally:
        c.set_profiling(False)
        c.close()


@pytest.mark.parametrize("sides", [(5.0e4, 20.0, 2.0e3), (500.0, 5.0e4, 5.0e3), (3.0e3, 3.0e3)])
def test_sweep_dimension_choice(sides):
    # Any dimension order gives the same pairs (Section 3); with the automatic
    # choice the library sweeps the dimension with the fewest one-dimensional
    # intersections, which the oracle's per-dimension counts predict exactly.
    import paper_1703_06680_gb300 as ddm
    reg = synth.make_regions_aniso(20_000, 25_000, sides, 4242)
    d = reg.d
    want = oracle.sbm(reg)
    one_d = [oracle.sbm_count(synth.Regions(reg.sub_lo[k:k + 1], reg.sub_hi[k:k + 1],
                                            reg.upd_lo[k:k + 1], reg.upd_hi[k:k + 1]))
             for k in range(d)]
    expected = sorted(range(d), key=lambda k: (one_d[k], k))
    c = ddm.Context(0)
    try:
        for mode in (0, 1):
            c.set_param(ddm.PARAM_SWEEP_DIM, mode)
            assert np.array_equal(gpu_pairs(c, reg), want), mode
            assert c.stats()["dim_order"][:d] == (expected if mode == 1 else list(range(d)))
            assert c.count(*to_dev(reg)) == len(want)
            host = c.match_host(reg.sub_lo, reg.sub_hi, reg.upd_lo, reg.upd_hi,
                                cap=len(want) + 1)
            assert np.array_equal(host, want)
        with pytest.raises(ddm.DDMError):
            c.set_param(ddm.PARAM_SWEEP_DIM, 2)
    finally:
        c.close()


def test_plain_sort_beyond_fused_offsets(ctx):
    # E = 6e6 endpoints: over 1024 sort tiles, so the 32-bit sort takes the flat
    # decoupled-look-back scan between upsweep and downsweep instead of the
    # in-downsweep group sums; the offsets scan over 1.5e6 subscriptions needs
    # several look-back rounds.
    assert_parity(ctx, synth.large_1d(1.0, N=3_000_000))


@pytest.mark.parametrize("d,alpha", [(1, 100.0), (2, 100.0), (3, 1.0)])
def test_swap_symmetry_and_dimension_monotonicity(ctx, d, alpha):
    # Exchanging the roles of subscriptions and updates transposes the pair set
    # (Algorithm 1 is symmetric); dropping a dimension can only add pairs
    # (Section 3's logical and).
    reg = synth.large_1d(alpha, N=100_000) if d == 1 else synth.large_nd(d, alpha, N=60_000)
    got = gpu_pairs(ctx, reg)
    sw = gpu_pairs(ctx, reg.swapped())
    assert len(sw) == len(got)
    back = sw[:, ::-1]
    order = np.lexsort((back[:, 1], back[:, 0]))
    assert np.array_equal(back[order], got)
    prev = len(got)
    for k in range(d - 1, 0, -1):
        K = ctx.count(*to_dev(reg.subset_dims(k)))
        assert K >= prev
        prev = K


def test_memory_budget_exhaustion_is_reported():
    # A context whose scratch budget is too small fails with DDM_ERR_NOMEM
    # (no device fault), and the same GPU keeps working afterwards.
    import paper_1703_06680_gb300 as ddm
    reg = synth.large_1d(1.0, N=200_000)
    small = ddm.Context(0, mem_budget=1 << 20)
    try:
        with pytest.raises(ddm.DDMError) as e:
            small.count(*to_dev(reg))
        assert e.value.code == ddm._lib.DDM_ERR_NOMEM
    finally:
        small.close()
    with ddm.Context(0) as c:
        assert c.count(*to_dev(reg)) == oracle.sbm_count(reg)


# --- window emission: long candidate lists, overflow, window sizes, alignment ---------

@pytest.mark.parametrize("num_huge", [600, 1100])
def test_window_long_candidate_lists(ctx, num_huge):
    # Short subscriptions under num_huge updates that span the whole routing space:
    # every boundary list holds them all.  600: each warp's candidate list is longer
    # than one piece (filtered piece by piece, in id order); 1100: the boundary
    # lists exceed their cap and the windows fall back to the range path.
    base = synth.make_regions(1, 20_000, 2_000, 50.0, 77)
    u_lo = np.concatenate([base.upd_lo, np.full((1, num_huge), -1.0, np.float32)], axis=1)
    u_hi = np.concatenate([base.upd_hi, np.full((1, num_huge), 2.0e6, np.float32)], axis=1)
    reg = synth.Regions(base.sub_lo, base.sub_hi, u_lo, u_hi)
    assert_parity(ctx, reg)


@pytest.mark.parametrize("shift", [6, 7, 8, 9, 10])
def test_window_sizes(shift):
    import paper_1703_06680_gb300 as ddm
    reg = synth.large_1d(100.0, N=100_000)
    want = oracle.sbm(reg)
    with ddm.Context(0) as c:
        c.set_param(ddm._lib.PARAM_WIN_SHIFT, shift)
        assert np.array_equal(gpu_pairs(c, reg), want)


def test_misaligned_pairs_rejected(ctx):
    # Pairs are written as 8-byte units: a pointer 4 bytes off is refused before
    # any launch, and the context stays usable.
    import torch
    import paper_1703_06680_gb300 as ddm
    reg = synth.small_1d()
    t = to_dev(reg)
    K = ctx.count(*t)
    buf = torch.empty(2 * K + 1, dtype=torch.int32, device=t[0].device)
    with pytest.raises(ddm.DDMError):
        ctx.match_into(buf[1:].view(K, 2), *t)
    assert_parity(ctx, reg)


# --- fault handling: a bounded device wait that runs out ------------------------------

@pytest.mark.parametrize("which", [0, 1], ids=["lookback", "mbarrier"])
def test_bounded_wait_times_out_and_context_survives(which):
    # The look-back poll and the mbarrier wait, run against a hand-off that never
    # happens with a short limit: the kernel returns, the host reads
    # DDM_ERR_DEVICE_TIMEOUT, and the same context then gives the oracle's result.
    import paper_1703_06680_gb300 as ddm
    reg = synth.small_1d()
    want = oracle.sbm(reg)
    with ddm.Context(0) as c:
        for _ in range(2):
            with pytest.raises(ddm.DDMError) as e:
                c.debug_wait_timeout(which, 4096)
            assert e.value.code == ddm._lib.DDM_ERR_DEVICE_TIMEOUT
            assert "timed out" in str(e.value)
            assert np.array_equal(gpu_pairs(c, reg), want)
        with pytest.raises(ddm.DDMError) as e:
            c.debug_wait_timeout(2, 16)
        assert e.value.code == ddm._lib.DDM_ERR_INVALID


# --- measurement aid: the emission's write pattern without its filter -----------------

def _wp_hash(x):
    # the segment-length hash of the write-pattern aid (xorshift-multiply mix, 32-bit)
    x &= 0xFFFFFFFF
    x ^= x >> 16
    x = (x * 0x7FEB352D) & 0xFFFFFFFF
    x ^= x >> 15
    x = (x * 0x846CA68B) & 0xFFFFFFFF
    x ^= x >> 16
    return x


@pytest.mark.parametrize("scattered", [False, True], ids=["id_order", "scattered"])
def test_write_pattern_aid_writes_the_stated_bytes(scattered):
    # The aid writes exactly the segments it states (lengths from its hash) and
    # reports a positive time; out-of-range arguments are rejected.
    import paper_1703_06680_gb300 as ddm
    nseg, mean = 3001, 37
    want = 8 * sum(mean // 2 + _wp_hash(s ^ 0x9E3779B9) % (mean + 1) for s in range(nseg))
    with ddm.Context(0) as c:
        ms, nbytes = c.debug_write_pattern(nseg, mean, scattered=scattered, reps=2)
        assert nbytes == want and ms > 0
        for bad in ((0, 10), (10, 0), (10, 5000)):
            with pytest.raises(ddm.DDMError) as e:
                c.debug_write_pattern(*bad)
            assert e.value.code == ddm._lib.DDM_ERR_INVALID
        reg = synth.small_1d()
        assert np.array_equal(gpu_pairs(c, reg), oracle.sbm(reg))  # context still usable


def test_tile_parameters_change_only_speed():
    # Every sort tile size (keys per thread) and every join window gives the
    # oracle's pairs, including the flat-scan sort above 1024 tiles.
    import paper_1703_06680_gb300 as ddm
    reg1 = synth.large_1d(100.0, N=200_001)
    want1 = oracle.sbm(reg1)
    big = synth.large_1d(1.0, N=2_500_000)      # > 1024 tiles at every tile size
    want_big = oracle.sbm(big)
    reg2 = synth.large_nd(3, 100.0, N=40_001)
    want2 = oracle.sbm(reg2)
    with ddm.Context(0) as c:
        for items in (12, 16, 18):
            c.set_param(ddm._lib.PARAM_SORT_ITEMS, items)
            assert np.array_equal(gpu_pairs(c, reg1), want1), items
            assert np.array_equal(gpu_pairs(c, big), want_big), items
            assert np.array_equal(gpu_pairs(c, reg2), want2), items
        for shift in (9, 10, 11):
            c.set_param(ddm._lib.PARAM_JOIN_SHIFT, shift)
            assert np.array_equal(gpu_pairs(c, reg2), want2), shift
        for bad in ((ddm._lib.PARAM_SORT_ITEMS, 20), (ddm._lib.PARAM_JOIN_SHIFT, 12)):
            with pytest.raises(ddm.DDMError):
                c.set_param(*bad)


@pytest.mark.parametrize("d,alpha", [(2, 100.0), (3, 1.0), (3, 100.0)])
def test_survivor_path_and_general_path_agree(d, alpha):
    # d > 1: the count pass records its survivors and the pairs come from one
    # sort of them once the context knows the output size (a first call without
    # that hint may run the general write pass instead).  Both give the
    # oracle's list; so does a later call on another instance.
    import paper_1703_06680_gb300 as ddm
    reg = synth.large_nd(d, alpha, N=300_000 if alpha == 100.0 else 600_000)
    from tests.oracle_pool import check_full
    with ddm.Context(0) as c:
        c.set_param(ddm._lib.PARAM_ND_WRITE, 2)
        t = to_dev(reg)
        K = c.count(*t)
        first = c.match(*t, cap=K)   # sized without a hint: may take either path
        second = c.match(*t, cap=K)
        assert c.stats()["survivor_calls"] >= 1
        assert torch_equal(first, second)
        assert check_full(second, ("large_nd", (d, alpha, 0, reg.n + reg.m)), reg.n) == K
        small = synth.large_nd(d, alpha, N=20_001)
        assert np.array_equal(gpu_pairs(c, small), oracle.sbm(small))


def torch_equal(a, b):
    import torch
    return a.shape == b.shape and bool(torch.equal(a, b))


@pytest.mark.parametrize("d,alpha", [(2, 1.0), (3, 100.0)])
def test_nd_write_modes_agree(d, alpha):
    # Both ways of writing the d > 1 pairs, and the automatic choice, give the
    # oracle's list on the same context (two calls each, the second sized).
    import paper_1703_06680_gb300 as ddm
    reg = synth.large_nd(d, alpha, N=80_001)
    want = oracle.sbm(reg)
    with ddm.Context(0) as c:
        for mode in (1, 2, 0):
            c.set_param(ddm._lib.PARAM_ND_WRITE, mode)
            for _ in range(2):
                assert np.array_equal(gpu_pairs(c, reg), want), mode
        with pytest.raises(ddm.DDMError):
            c.set_param(ddm._lib.PARAM_ND_WRITE, 3)
