"""Served mode: resident sessions, device drift, count/admit/emit, continuous batching.

The drift kernel is checked bit for bit against the workload generator's own
implementation of the same counter-based definition; matching results after
drift are checked against the oracle run on the generator's drifted
coordinates (never on coordinates read back from the GPU); and every result
computed inside the concurrent mix must equal the one computed alone.
"""
import numpy as np
import pytest

import oracle
import synth
from tests.gpu_util import to_dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ddm():
    import paper_1703_06680_gb300 as ddm
    ddm.build_library()
    return ddm


def small_sims(count=8, seed=77):
    rng = np.random.default_rng(seed)
    sims = []
    for k in range(count):
        N = int(rng.integers(2_000, 60_000))
        d = 1 + k % 3
        alpha = (0.01, 1.0, 100.0)[k % 3] if d == 1 else (1.0, 100.0)[k % 2]
        side = synth.side_for(alpha, N, d)
        sims.append({"reg": synth.make_regions(d, N // 2, N - N // 2, side, 9000 + k),
                     "seed": 1234 + k, "sigma": 0.1 * side})
    return sims


@pytest.mark.parametrize("d", [1, 2, 3])
def test_drift_kernel_matches_generator(ddm, d):
    reg = synth.make_regions(d, 3001, 2999, 2000.0, 31 + d)
    sess = ddm.Session(*to_dev(reg))
    host = reg
    for step in range(3):
        sess.drift(555, step, 200.0)
        host = synth.drift(host, 555, step, 200.0)
        got = [t.cpu().numpy() for t in sess.coords()]
        for g, w in zip(got, (host.sub_lo, host.sub_hi, host.upd_lo, host.upd_hi)):
            assert np.array_equal(g.view(np.uint32), w.view(np.uint32))
    sess.close()


def test_session_count_emit_matches_oracle(ddm):
    import torch
    for sim in small_sims(4, seed=5):
        sess = ddm.Session(*to_dev(sim["reg"]))
        host = sim["reg"]
        for step in range(2):
            sess.drift(sim["seed"], step, sim["sigma"])
            host = synth.drift(host, sim["seed"], step, sim["sigma"])
            want = oracle.sbm(host)
            K = sess.count()
            assert K == len(want)
            out = torch.empty((K + 3, 2), dtype=torch.int32, device="cuda:0")
            assert sess.emit(out) == K
            assert np.array_equal(out[:K].cpu().numpy(), want)
        sess.close()


def test_emit_needs_count_and_capacity(ddm):
    import torch
    reg = synth.small_1d()
    sess = ddm.Session(*to_dev(reg))
    out = torch.empty((10, 2), dtype=torch.int32, device="cuda:0")
    with pytest.raises(ddm.DDMError):
        sess.emit(out)
    K = sess.count()
    with pytest.raises(ddm.CapacityError) as e:
        sess.emit(out[:K - 1] if K > 1 else out[:0])
    assert e.value.K == K
    sess.close()


def run_alone(ddm, sims, steps):
    import torch
    res = {}
    for k, sim in enumerate(sims):
        sess = ddm.Session(*to_dev(sim["reg"]))
        for step in range(steps):
            sess.drift(sim["seed"], step, sim["sigma"])
            K = sess.count()
            out = torch.empty((max(K, 1), 2), dtype=torch.int32, device="cuda:0")
            sess.emit(out[:K])
            res[(k, step)] = out[:K].cpu().numpy()
        sess.close()
    return res


@pytest.mark.parametrize("budget", [4 << 30, None])
def test_mix_equals_alone(ddm, budget):
    from paper_1703_06680_gb300.serve import Server, Simulation
    sims = small_sims(8)
    steps = 3
    alone = run_alone(ddm, sims, steps)
    if budget is None:  # tight budget: admission must make requests wait
        budget = 8 * max(len(v) for v in alone.values())
    objs = [Simulation(k, to_dev(s["reg"]), s["seed"], s["sigma"]) for k, s in enumerate(sims)]
    server = Server(objs, slots=4, out_budget_bytes=budget)
    reqs = [server.submit(k, keep_pairs=True) for step in range(steps) for k in range(len(sims))]
    for r in reqs:
        assert r.done.wait(120)
    server.close()
    for r in reqs:
        assert r.error is None, r.error
        assert np.array_equal(r.pairs, alone[(r.sim, r.step)]), (r.sim, r.step)
    for o in objs:
        o.close()


def test_mix_matches_oracle(ddm):
    from paper_1703_06680_gb300.serve import Server, Simulation
    sims = small_sims(6, seed=3)
    objs = [Simulation(k, to_dev(s["reg"]), s["seed"], s["sigma"]) for k, s in enumerate(sims)]
    server = Server(objs, slots=3)
    reqs = [server.submit(k, keep_pairs=True) for _ in range(2) for k in range(len(sims))]
    for r in reqs:
        assert r.done.wait(120)
    server.close()
    hosts = {}
    for r in sorted(reqs, key=lambda q: (q.sim, q.step)):
        s = sims[r.sim]
        prev = hosts.get(r.sim, s["reg"])
        hosts[r.sim] = synth.drift(prev, s["seed"], r.step, s["sigma"])
        assert np.array_equal(r.pairs, oracle.sbm(hosts[r.sim])), (r.sim, r.step)
    for o in objs:
        o.close()


def _rows_minus(a: np.ndarray, b: np.ndarray) -> np.ndarray:
    """Rows of the (k, 2) int32 array a that are not rows of b, sorted."""
    ka = (a[:, 0].astype(np.int64) << 32) | a[:, 1].astype(np.int64)
    kb = (b[:, 0].astype(np.int64) << 32) | b[:, 1].astype(np.int64)
    k = np.setdiff1d(ka, kb)
    return np.stack([(k >> 32).astype(np.int32), (k & 0xFFFFFFFF).astype(np.int32)], axis=1)


def test_emit_delta_matches_oracle_differences(ddm):
    # Every report equals the set differences of the oracle's pair lists of two
    # consecutive timesteps (first report: everything is added).
    for sim in small_sims(6, seed=11):
        sess = ddm.Session(*to_dev(sim["reg"]))
        host = sim["reg"]
        prev = np.zeros((0, 2), np.int32)
        for step in range(4):
            sess.drift(sim["seed"], step, sim["sigma"])
            host = synth.drift(host, sim["seed"], step, sim["sigma"])
            want = oracle.sbm(host)
            assert sess.count() == len(want)
            added, removed = sess.emit_delta()
            assert np.array_equal(added.cpu().numpy(), _rows_minus(want, prev)), step
            assert np.array_equal(removed.cpu().numpy(), _rows_minus(prev, want)), step
            prev = want
        sess.close()


def test_emit_delta_no_motion_and_capacity_retry(ddm):
    import torch
    reg = synth.make_regions(2, 3000, 3500, 3000.0, 5151)
    sess = ddm.Session(*to_dev(reg))
    buf = torch.empty((16, 2), dtype=torch.int32, device="cuda:0")
    with pytest.raises(ddm.DDMError):
        sess.emit_delta(buf, buf)                  # the first report needs a count first
    K = sess.count()
    added, removed = sess.emit_delta()
    assert len(added) == K and len(removed) == 0
    sess.drift(1, 0, 0.0)                          # no motion: nothing changes
    sess.count()
    added, removed = sess.emit_delta()
    assert len(added) == 0 and len(removed) == 0
    host = synth.drift(reg, 9, 1, 400.0)
    sess.drift(9, 1, 400.0)
    sess.count()
    small = torch.empty((1, 2), dtype=torch.int32, device="cuda:0")
    with pytest.raises(ddm.CapacityError):
        sess.emit_delta(small, small)
    added, removed = sess.emit_delta()             # the pending report, into larger buffers
    want_prev, want = oracle.sbm(reg), oracle.sbm(host)
    assert np.array_equal(added.cpu().numpy(), _rows_minus(want, want_prev))
    assert np.array_equal(removed.cpu().numpy(), _rows_minus(want_prev, want))
    sess.close()


@pytest.mark.parametrize("d", [1, 2])
def test_emit_delta_counts_its_own_timestep(ddm, d):
    # After the first report, a report of a timestep nobody counted runs the
    # count phase itself (one library call): the same differences, and the
    # session's K is that timestep's.
    import torch
    N = 40_000
    side = synth.side_for(100.0 if d == 1 else 10.0, N, d)
    reg = synth.make_regions(d, N // 2, N - N // 2, side, 5200 + d)
    sess = ddm.Session(*to_dev(reg))
    host = reg
    prev = oracle.sbm(host)
    assert sess.count() == len(prev)
    sess.emit_delta()
    cap = max(len(prev), 16)
    add_b = torch.empty((cap, 2), dtype=torch.int32, device="cuda:0")
    rem_b = torch.empty((cap, 2), dtype=torch.int32, device="cuda:0")
    for step in range(3):
        sess.drift(33, step, 0.02 * side)
        host = synth.drift(host, 33, step, 0.02 * side)
        want = oracle.sbm(host)
        added, removed = sess.emit_delta(add_b, rem_b)
        assert sess.K == len(want)
        assert np.array_equal(added.cpu().numpy(), _rows_minus(want, prev)), step
        assert np.array_equal(removed.cpu().numpy(), _rows_minus(prev, want)), step
        prev = want
    sess.close()


def test_session_budget_covers_change_report_buffers(ddm):
    # A session's budget caps everything it holds on the device: the resident
    # coordinates, the pipeline workspace, the reference coordinates and the
    # buffers of a change report (16 bytes per changed pair).  A report with
    # more changes than the budget allows fails with DDM_ERR_NOMEM before it
    # writes anything; count and emit still work; an oversized coordinate set
    # is refused at creation.
    import torch
    reg = synth.large_1d(100.0, N=200_000)          # K ~ 1e7
    side = synth.side_for(100.0, 200_000, 1)
    sess = ddm.Session(*to_dev(reg), mem_budget=64 << 20)
    try:
        K = sess.count()
        assert K == oracle.sbm_count(reg)
        added, removed = sess.emit_delta()          # first report: into the caller's buffers
        assert len(added) == K and len(removed) == 0
        sess.drift(77, 0, 0.5 * side)               # millions of pairs change
        host = synth.drift(reg, 77, 0, 0.5 * side)
        want = oracle.sbm(host)
        assert sess.count() == len(want)
        with pytest.raises(ddm.DDMError) as e:
            sess.emit_delta()
        assert e.value.code == ddm._lib.DDM_ERR_NOMEM
        sess.count()
        out = torch.empty((len(want), 2), dtype=torch.int32, device="cuda:0")
        assert sess.emit(out) == len(want)
        assert np.array_equal(out.cpu().numpy(), want)
    finally:
        sess.close()
    with pytest.raises(ddm.DDMError) as e:
        ddm.Session(*to_dev(reg), mem_budget=1 << 20)  # 1.6 MB of coordinates
    assert e.value.code == ddm._lib.DDM_ERR_NOMEM


@pytest.mark.parametrize("d,alpha", [(1, 100.0), (1, 0.01), (2, 100.0), (3, 1.0)])
def test_emit_delta_against_last_delivered_report(ddm, d, alpha):
    # Reports at steps 0, 1, 3 and 6 of a drifting workload (served drift,
    # 0.1 side per step, and a slower one): each report is the difference from
    # the last DELIVERED report, whatever happened in between.
    N = 60_000 if d == 1 else 30_000
    side = synth.side_for(alpha, N, d)
    reg = synth.make_regions(d, N // 2, N - N // 2, side, 4400 + d)
    for sigma in (0.1 * side, 0.01 * side):
        sess = ddm.Session(*to_dev(reg))
        host, prev = reg, None
        for step in range(7):
            sess.drift(91, step, sigma)
            host = synth.drift(host, 91, step, sigma)
            K = sess.count()
            if step not in (0, 1, 3, 6):
                continue
            want = oracle.sbm(host)
            assert K == len(want)
            added, removed = sess.emit_delta()
            base = np.zeros((0, 2), np.int32) if prev is None else prev
            assert np.array_equal(added.cpu().numpy(), _rows_minus(want, base)), (sigma, step)
            assert np.array_equal(removed.cpu().numpy(), _rows_minus(base, want)), (sigma, step)
            prev = want
        sess.close()


def test_emit_delta_infinite_and_degenerate_bounds(ddm):
    # Extents with infinite bounds (they stay infinite under drift), points,
    # and touching extents: the report stays the exact set difference.
    rng = np.random.default_rng(5)
    from tests.helpers import tiny_grid_instance
    reg = tiny_grid_instance(rng, 2, 300, 280, grid=16)
    reg.sub_lo[0, :5] = -np.inf
    reg.upd_hi[1, :7] = np.inf
    sess = ddm.Session(*to_dev(reg))
    host, prev = reg, np.zeros((0, 2), np.int32)
    for step in range(4):
        sess.drift(3, step, 0.7)
        host = synth.drift(host, 3, step, 0.7)
        want = oracle.sbm(host)
        assert sess.count() == len(want)
        added, removed = sess.emit_delta()
        assert np.array_equal(added.cpu().numpy(), _rows_minus(want, prev)), step
        assert np.array_equal(removed.cpu().numpy(), _rows_minus(prev, want)), step
        prev = want
    sess.close()
