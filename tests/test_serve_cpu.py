"""Host logic of the continuous-batching server, on CPU with fake sessions.

The fakes stand in for the native sessions and the CUDA side (streams, output
buffers); what is tested is the server's own logic: timesteps of one
simulation in order and never concurrent, different simulations overlapping,
admission by the output-memory budget, errors reported per request, and
draining on close.
"""
import threading
import time

import numpy as np
import pytest

from paper_1703_06680_gb300 import DDMError
from paper_1703_06680_gb300.serve import Request, Server, latency_summary


class Tracker:
    def __init__(self):
        self.lock = threading.Lock()
        self.inflight_bytes = 0
        self.max_inflight_bytes = 0
        self.running = 0
        self.max_running = 0
        self.events = []  # (sim, step, t_start, t_end)


class FakeSession:
    """K(sim, step) pairs per timestep; emit fills (sim, step*1000 + r)."""

    def __init__(self, sim, tracker, K=5, delay=0.01, fail_steps=()):
        self.sim, self.t, self.K, self.delay = sim, tracker, K, delay
        self.fail_steps = set(fail_steps)
        self.step = None
        self.t0 = None

    def drift(self, seed, step, sigma, stream=None):
        self.step = step
        self.t0 = time.perf_counter()
        with self.t.lock:
            self.t.running += 1
            self.t.max_running = max(self.t.max_running, self.t.running)

    def count(self, stream=None):
        return self.K(self.step) if callable(self.K) else self.K

    def emit(self, out, stream=None):
        K = len(out)
        with self.t.lock:
            self.t.inflight_bytes += 8 * K
            self.t.max_inflight_bytes = max(self.t.max_inflight_bytes, self.t.inflight_bytes)
        try:
            time.sleep(self.delay)
            if self.step in self.fail_steps:
                raise DDMError(-6, "planted failure")
            out[:, 0] = self.sim
            out[:, 1] = self.step * 1000 + np.arange(K)
            return K
        finally:
            with self.t.lock:
                self.t.inflight_bytes -= 8 * K
                self.t.running -= 1
                self.t.events.append((self.sim, self.step, self.t0, time.perf_counter()))


class FakeSim:
    def __init__(self, sim_id, session):
        self.sim_id, self.session = sim_id, session
        self.seed, self.sigma = 1, 0.1
        self.next_step = 0
        self.busy = False


class FakeBackend:
    def stream(self):
        return object()

    def bind(self):
        pass

    def alloc_pairs(self, K, stream):
        return np.zeros((max(K, 1), 2), dtype=np.int32)

    def to_host(self, pairs):
        return np.array(pairs)

    def synchronize(self, stream):
        pass


def make(num_sims, tracker, slots=4, budget=1 << 30, **kw):
    sims = [FakeSim(k, FakeSession(k, tracker, **kw)) for k in range(num_sims)]
    return sims, Server(sims, slots=slots, out_budget_bytes=budget, backend=FakeBackend())


def wait_all(reqs, timeout=30):
    for r in reqs:
        assert r.done.wait(timeout)


def test_steps_in_order_never_concurrent_and_sims_overlap():
    t = Tracker()
    sims, server = make(3, t, slots=4, delay=0.02)
    reqs = [server.submit(k % 3, keep_pairs=True) for k in range(15)]
    wait_all(reqs)
    server.close()
    for r in reqs:
        assert r.error is None
        assert np.array_equal(r.pairs[:, 0], np.full(5, r.sim))
        assert np.array_equal(r.pairs[:, 1], r.step * 1000 + np.arange(5))
    for s in range(3):
        ev = sorted((e for e in t.events if e[0] == s), key=lambda e: e[2])
        assert [e[1] for e in ev] == list(range(5))          # submission order
        for a, b in zip(ev, ev[1:]):
            assert a[3] <= b[2]                               # never concurrent
        assert sorted(r.step for r in reqs if r.sim == s) == list(range(5))
    assert t.max_running >= 2                                 # different sims overlap


def test_admission_keeps_output_within_budget():
    t = Tracker()
    K = 1000
    sims, server = make(6, t, slots=6, budget=2 * 8 * K, K=K, delay=0.03)
    reqs = [server.submit(k) for k in range(6)]
    wait_all(reqs)
    server.close()
    assert all(r.error is None and r.K == K for r in reqs)
    assert t.max_inflight_bytes <= 2 * 8 * K
    assert t.max_inflight_bytes == 2 * 8 * K                  # and it does run two at once
    assert server.free == server.budget


def test_request_above_budget_fails_alone():
    t = Tracker()
    sims, server = make(2, t, slots=2, budget=8 * 100,
                        K=lambda step: 10_000 if step == 1 else 10)
    reqs = [server.submit(0) for _ in range(3)] + [server.submit(1)]
    wait_all(reqs)
    server.close()
    by_step = {(r.sim, r.step): r for r in reqs}
    assert isinstance(by_step[(0, 1)].error, DDMError)
    assert all(r.error is None for key, r in by_step.items() if key != (0, 1))
    assert server.free == server.budget                      # nothing released twice


def test_session_error_reported_and_slot_survives():
    t = Tracker()
    sims, server = make(1, t, slots=1, fail_steps=(2,))
    reqs = [server.submit(0) for _ in range(5)]
    wait_all(reqs)
    server.close()
    errs = [r.step for r in reqs if r.error is not None]
    assert errs == [2]
    assert [r.K for r in reqs if r.error is None] == [5, 5, 5, 5]
    assert server.free == server.budget


def test_close_drains_queue():
    t = Tracker()
    sims, server = make(4, t, slots=2, delay=0.005)
    reqs = [server.submit(k % 4) for k in range(24)]
    server.close()
    assert all(r.done.is_set() and r.error is None for r in reqs)
    assert len(server.completed) == 24


def test_latency_summary():
    reqs = []
    for k in range(100):
        r = Request(sim=0, arrival=0.0)
        r.finish = (k + 1) * 1e-3
        r.K = 10
        reqs.append(r)
    s = latency_summary(reqs, wall=2.0)
    assert s["requests"] == 100 and s["pairs"] == 1000 and s["pairs_per_s"] == 500.0
    assert s["p50_ms"] == pytest.approx(50.5)
    assert s["p99_ms"] == pytest.approx(99.01)
    assert s["errors"] == 0
