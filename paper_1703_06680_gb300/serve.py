"""Served mode: continuous batching of matching requests over resident simulations.

A request asks for the next timestep of one simulation: its extents drift
(device-side, deterministic draws), then all intersecting (sub, upd) pairs of
the new state are reported.  Each simulation is a native session
(ddm_session_*) that keeps its coordinates and pipeline workspace on the GPU
across timesteps.

The server runs `slots` workers, each with its own CUDA stream.  A worker
takes the oldest queued request whose simulation is idle (timesteps of one
simulation stay in order), runs drift + count, then ADMITS the request by
device memory: the count gives the exact output size 8*K, which is reserved
from the output budget before the pairs are emitted; a request that does not
fit waits until running requests release memory.  Requests that arrive while
others run are admitted as soon as a slot and memory free up, and their
kernels overlap on the device through the slots' streams (ctypes releases the
GIL during library calls).  Latency is measured from arrival to completion.
"""
from __future__ import annotations

import collections
import dataclasses
import threading
import time

import numpy as np

from ._lib import DDMError, Session


@dataclasses.dataclass
class Request:
    sim: int
    arrival: float
    keep_pairs: bool = False
    step: int = -1
    K: int = -1
    pairs: np.ndarray | None = None
    start: float = 0.0
    finish: float = 0.0
    error: Exception | None = None
    done: threading.Event = dataclasses.field(default_factory=threading.Event)

    @property
    def latency(self) -> float:
        return self.finish - self.arrival


class Simulation:
    """One simulation: resident extents plus its drift parameters."""

    def __init__(self, sim_id: int, tensors, seed: int, sigma: float, device: int = 0):
        self.sim_id = sim_id
        self.seed = seed
        self.sigma = sigma
        self.session = Session(*tensors, device=device)
        self.next_step = 0
        self.busy = False

    def close(self):
        self.session.close()


class CudaBackend:
    """Device side of a server slot: its stream and the output buffers."""

    def __init__(self, device: int = 0):
        import torch
        self.torch = torch
        self.device = device

    def stream(self):
        return self.torch.cuda.Stream(device=self.device)

    def bind(self):
        self.torch.cuda.set_device(self.device)

    def alloc_pairs(self, K: int, stream):
        with self.torch.cuda.stream(stream):
            return self.torch.empty((max(K, 1), 2), dtype=self.torch.int32, device=self.device)

    def to_host(self, pairs):
        return pairs.cpu().numpy()

    def synchronize(self, stream):
        stream.synchronize()


class Server:
    def __init__(self, sims: list[Simulation], slots: int = 4, out_budget_bytes: int = 4 << 30,
                 device: int = 0, backend=None):
        self.backend = backend if backend is not None else CudaBackend(device)
        self.sims = sims
        self.device = device
        self.budget = out_budget_bytes
        self.free = out_budget_bytes
        self.queue: collections.deque[Request] = collections.deque()
        self.cv = threading.Condition()
        self.stop = False
        self.completed: list[Request] = []
        self.streams = [self.backend.stream() for _ in range(slots)]
        self.workers = [threading.Thread(target=self._work, args=(k,), daemon=True)
                        for k in range(slots)]
        for w in self.workers:
            w.start()

    # -- client side --------------------------------------------------------------
    def submit(self, sim: int, keep_pairs: bool = False, arrival: float | None = None) -> Request:
        req = Request(sim=sim, arrival=time.perf_counter() if arrival is None else arrival,
                      keep_pairs=keep_pairs)
        with self.cv:
            self.queue.append(req)
            self.cv.notify_all()
        return req

    def close(self):
        with self.cv:
            self.stop = True
            self.cv.notify_all()
        for w in self.workers:
            w.join()

    # -- workers -----------------------------------------------------------------
    def _take(self) -> Request | None:
        with self.cv:
            while True:
                for k, req in enumerate(self.queue):
                    if not self.sims[req.sim].busy:
                        del self.queue[k]
                        sim = self.sims[req.sim]
                        sim.busy = True
                        req.step = sim.next_step
                        sim.next_step += 1
                        return req
                if self.stop and not self.queue:
                    return None
                self.cv.wait(0.05)

    def _admit(self, nbytes: int):
        with self.cv:
            if nbytes > self.budget:
                raise DDMError(-3, f"request needs {nbytes} output bytes, above the budget")
            while self.free < nbytes:
                self.cv.wait()
            self.free -= nbytes

    def _release(self, nbytes: int):
        with self.cv:
            self.free += nbytes
            self.cv.notify_all()

    def _work(self, slot: int):
        be = self.backend
        stream = self.streams[slot]
        be.bind()
        while True:
            req = self._take()
            if req is None:
                return
            sim = self.sims[req.sim]
            req.start = time.perf_counter()
            reserved = 0
            try:
                sess = sim.session
                sess.drift(sim.seed, req.step, sim.sigma, stream=stream)
                K = sess.count(stream=stream)
                self._admit(8 * K)
                reserved = 8 * K  # only what was admitted is released
                out = be.alloc_pairs(K, stream)
                req.K = sess.emit(out[:K], stream=stream)
                if req.keep_pairs:
                    req.pairs = be.to_host(out[:K])
                be.synchronize(stream)
                del out
            except Exception as exc:  # reported through the request
                req.error = exc
            finally:
                if reserved:
                    self._release(reserved)
                req.finish = time.perf_counter()
                with self.cv:
                    sim.busy = False
                    self.completed.append(req)
                    self.cv.notify_all()
                req.done.set()


def run_plain(sims: list[Simulation], requests: list[Request], device: int = 0):
    """Baseline: the same requests one at a time on one stream, each ONE plain
    ddm_match call on the simulation's resident coordinates (no copy), into a
    buffer sized by that simulation's previous K (plus 10%); only when the
    pairs do not fit is a larger buffer taken and the call repeated.  Nothing
    overlaps.  Requests start no earlier than their arrival time."""
    import torch

    from ._lib import CapacityError, Context
    ctx = Context(device)
    cap_of: dict[int, int] = {}
    out = torch.empty((1, 2), dtype=torch.int32, device=device)
    t0 = time.perf_counter()
    for req in requests:
        now = time.perf_counter()
        if req.arrival > now:
            time.sleep(req.arrival - now)
        sim = sims[req.sim]
        req.step = sim.next_step
        sim.next_step += 1
        req.start = time.perf_counter()
        sim.session.drift(sim.seed, req.step, sim.sigma)
        packed = sim.session.packed()
        cap = cap_of.get(req.sim, 1 << 16)
        if out.shape[0] < cap:
            out = torch.empty((cap, 2), dtype=torch.int32, device=device)
        try:
            K = ctx.match_packed(packed, out[:cap])
        except CapacityError as e:
            cap = e.K + e.K // 10 + 1024
            out = torch.empty((cap, 2), dtype=torch.int32, device=device)
            K = ctx.match_packed(packed, out[:cap])
        cap_of[req.sim] = K + K // 10 + 1024
        req.K = K
        if req.keep_pairs:
            req.pairs = out[:K].cpu().numpy()
        torch.cuda.synchronize()
        req.finish = time.perf_counter()
        req.done.set()
    ctx.close()
    return time.perf_counter() - t0


def latency_summary(reqs: list[Request], wall: float) -> dict:
    lat = np.array([r.latency for r in reqs]) * 1e3
    pairs = sum(max(r.K, 0) for r in reqs)
    return {"requests": len(reqs), "p50_ms": float(np.percentile(lat, 50)),
            "p99_ms": float(np.percentile(lat, 99)), "mean_ms": float(lat.mean()),
            "pairs": int(pairs), "pairs_per_s": pairs / wall, "wall_s": wall,
            "errors": sum(1 for r in reqs if r.error is not None)}
