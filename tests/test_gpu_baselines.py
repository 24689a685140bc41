"""The paper's comparison matchers on the GPU: Brute-Force (Algorithm 2),
Interval-Tree matching (Algorithm 3) and Grid-Based matching (Section 2),
through the C ABI, against the CPU oracle; and brute force as a second, independent GPU-side check of the
sort-based path at moderate sizes.  Results are integer pair lists: the bar is
bit-exact equality of the sorted lists.
"""
import numpy as np
import pytest

import oracle
import synth
from tests.gpu_util import to_dev
from tests.helpers import special_value_instance, tiny_grid_instance

pytestmark = pytest.mark.gpu

METHODS = ["bruteforce", "itm", "grid"]


@pytest.fixture(scope="module")
def ctx():
    import paper_1703_06680_gb300 as ddm
    ddm.build_library()
    c = ddm.Context(0)
    yield c
    c.close()


def method_fn(ctx, method):
    return {"bruteforce": ctx.match_bruteforce, "itm": ctx.match_itm,
            "grid": ctx.match_grid}[method]


def run(ctx, method, reg, count_only=False):
    r = method_fn(ctx, method)(*to_dev(reg), count_only=count_only)
    return r if count_only else r.cpu().numpy()


def check(ctx, method, reg, want=None):
    if want is None:
        want = oracle.sbm(reg)
    got = run(ctx, method, reg)
    assert got.shape == want.shape, (got.shape, want.shape)
    assert np.array_equal(got, want)
    assert run(ctx, method, reg, count_only=True) == len(want)


@pytest.mark.parametrize("method", METHODS)
def test_small_and_reduced_workloads(ctx, method):
    check(ctx, method, synth.small_1d())
    check(ctx, method, synth.large_1d(100.0, N=60_000))
    check(ctx, method, synth.large_1d(0.01, N=60_000))
    check(ctx, method, synth.large_nd(2, 100.0, N=40_001))
    check(ctx, method, synth.large_nd(3, 1.0, N=40_001))


@pytest.mark.parametrize("method", METHODS)
def test_dense_ties_special_values_and_edges(ctx, method):
    rng = np.random.default_rng(31)
    for s in range(120):
        d = 1 + s % 3
        check(ctx, method, tiny_grid_instance(rng, d, int(rng.integers(0, 70)),
                                              int(rng.integers(0, 70))))
    for s in range(40):
        check(ctx, method, special_value_instance(rng, 1 + s % 3, int(rng.integers(1, 200)),
                                                  int(rng.integers(1, 200))))
    # every pair matches; one extent; empty sets; the most dimensions
    check(ctx, method, synth.Regions(np.full((1, 700), 1.0, np.float32),
                                     np.full((1, 700), 2.0, np.float32),
                                     np.full((1, 900), 2.0, np.float32),
                                     np.full((1, 900), 3.0, np.float32)))
    for n, m in [(1, 1), (0, 50), (50, 0), (1, 3000), (3000, 1), (1025, 1023)]:
        check(ctx, method, synth.make_regions(1, n, m, 5000.0, 7 + n + m))
    check(ctx, method, synth.make_regions_aniso(3000, 2500, (2.0e4,) + (4.0e5,) * 7, 88))


@pytest.mark.parametrize("method", METHODS)
def test_invalid_input_and_capacity(ctx, method):
    import paper_1703_06680_gb300 as ddm
    for where in range(3):
        reg = synth.make_regions(3, 200, 150, 1e4, 3)
        if where == 0:
            reg.upd_lo[0, 7] = np.nan
        elif where == 1:
            reg.sub_lo[2, 3] = reg.sub_hi[2, 3] + 1
        else:
            reg.upd_lo[1, 0] = reg.upd_hi[1, 0] + 5
        with pytest.raises(ddm.DDMError) as e:
            run(ctx, method, reg, count_only=True)
        assert e.value.code == ddm._lib.DDM_ERR_INVALID
    reg = synth.small_1d()
    want = oracle.sbm(reg)
    with pytest.raises(ddm.CapacityError) as e:
        method_fn(ctx, method)(*to_dev(reg), cap=len(want) - 1)
    assert e.value.K == len(want)
    check(ctx, method, reg, want)   # the context stays usable


@pytest.mark.parametrize("d,alpha", [(1, 100.0), (2, 100.0), (3, 1.0)])
def test_bruteforce_checks_sort_based_path(ctx, d, alpha):
    # Two independent GPU methods on N = 1e5 (plus the oracle's count): the
    # sort-based list equals brute force's, pair for pair.
    reg = synth.large_1d(alpha, N=100_000) if d == 1 else synth.large_nd(d, alpha, N=100_000)
    t = to_dev(reg)
    sbm = ctx.match(*t).cpu().numpy()
    bf = ctx.match_bruteforce(*t).cpu().numpy()
    assert np.array_equal(sbm, bf)
    assert len(bf) == oracle.sbm_count(reg)
    itm = ctx.match_itm(*t).cpu().numpy()
    assert np.array_equal(itm, bf)


@pytest.mark.parametrize("d,alpha", [(1, 100.0), (2, 1.0), (3, 100.0)])
def test_grid_size_changes_only_speed(ctx, d, alpha):
    # Any mesh gives the same pairs: one cell (brute force), a few, the
    # library's choice, and more cells than extents per dimension (clamped).
    reg = synth.large_1d(alpha, N=40_000) if d == 1 else synth.large_nd(d, alpha, N=30_000)
    want = oracle.sbm(reg)
    t = to_dev(reg)
    for cells in (1, 3, 0, 64, 1 << 20):
        got = ctx.match_grid(*t, cells_per_dim=cells).cpu().numpy()
        assert np.array_equal(got, want), cells
        grid = ctx.last_grid
        assert all(1 <= g for g in grid) and grid[min(d, 3):] == [1] * (3 - min(d, 3))
        if cells == 1:
            assert grid == [1, 1, 1]


def test_grid_huge_extents_and_infinities(ctx):
    # Extents spanning the whole space fall into every cell; an infinite bound
    # makes that dimension one cell; pairs stay exact and unique.
    reg = synth.large_nd(2, 1.0, N=20_000)
    reg.sub_lo[:, 5] = -1.0
    reg.sub_hi[:, 5] = 2.0e6
    reg.upd_lo[0, 9] = -np.inf
    reg.upd_hi[1, 9] = np.inf
    want = oracle.sbm(reg)
    assert np.array_equal(ctx.match_grid(*to_dev(reg)).cpu().numpy(), want)
    assert ctx.last_grid[0] == 1
