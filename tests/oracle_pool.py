"""Full-size parity at oracle speed: the CPU oracle run slice by slice in a pool.

The pairs of subscription S_i depend only on S_i and the updates, so the
oracle's answer for the subscriptions [a, b) is the oracle run on those
subscriptions alone against all updates, with a added to the subscription
ids.  The GPU's sorted list is written once to a memory-mapped file; each
worker process regenerates the seeded workload itself (synth, no GPU), runs
the oracle on its slice and compares its rows of the GPU list element by
element.  Batched instances are checked the same way, instance by instance.

The pool is started with the "spawn" method (never "fork": a child forked
from a process that has used CUDA can hang), and the workers import neither
torch nor the CUDA library.
"""
from __future__ import annotations

import multiprocessing as mp
import os
import shutil
import tempfile

import numpy as np

import oracle
import synth

_CACHE: dict = {}


def _workload(spec):
    """spec = (name of a synth function, args tuple); cached per worker process."""
    if spec not in _CACHE:
        name, args = spec
        _CACHE.clear()
        _CACHE[spec] = getattr(synth, name)(*args)
    return _CACHE[spec]


def _pairs_file(K: int) -> str:
    need = 8 * max(K, 1) + (64 << 20)
    for d in ("/dev/shm", tempfile.gettempdir()):
        try:
            if os.path.isdir(d) and shutil.disk_usage(d).free > need:
                fd, path = tempfile.mkstemp(prefix="ddm_pairs_", suffix=".i32", dir=d)
                os.close(fd)
                return path
        except OSError:
            continue
    raise RuntimeError("no room for the GPU pair list on disk")


def _store(pairs_dev, K: int) -> str:
    """Copies a (K, 2) int32 CUDA tensor into a memory-mapped file; returns its path."""
    path = _pairs_file(K)
    mm = np.memmap(path, dtype=np.int32, mode="w+", shape=(max(K, 1), 2))
    step = 1 << 24
    for a in range(0, K, step):
        b = min(K, a + step)
        mm[a:b] = pairs_dev[a:b].cpu().numpy()
    mm.flush()
    del mm
    return path


def _open(path: str, K: int):
    return np.memmap(path, dtype=np.int32, mode="r", shape=(max(K, 1), 2))


def _check_subs(job):
    spec, a, b, lo, hi, path, K = job
    reg = _workload(spec)
    sl = synth.Regions(reg.sub_lo[:, a:b].copy(), reg.sub_hi[:, a:b].copy(), reg.upd_lo,
                       reg.upd_hi)
    want = oracle.sbm(sl)
    want[:, 0] += a
    got = np.asarray(_open(path, K)[lo:hi])
    if got.shape != want.shape:
        return (a, b, len(want), False, f"rows {len(got)} vs oracle {len(want)}")
    if not np.array_equal(got, want):
        k = int(np.argmax(np.any(got != want, axis=1)))
        return (a, b, len(want), False, f"row {lo + k}: {got[k].tolist()} vs {want[k].tolist()}")
    return (a, b, len(want), True, "")


def _check_instances(job):
    spec, b0, b1, offs, path, K = job
    _, (num, replica, d, alpha) = spec
    sizes = synth.batch_sizes(num, replica)
    mm = _open(path, K)
    total = 0
    for b in range(b0, b1):
        reg = synth.batch_instance(b, sizes, replica, d, alpha)
        want = oracle.sbm(reg)
        total += len(want)
        got = np.asarray(mm[offs[b - b0]:offs[b - b0 + 1]])
        if got.shape != want.shape or not np.array_equal(got, want):
            return (b0, b1, total, False, f"instance {b}: {len(got)} rows vs oracle {len(want)}")
    return (b0, b1, total, True, "")


def _pool(nproc: int | None):
    oracle.build()
    n = nproc or max(1, min(16, os.cpu_count() or 1))
    return mp.get_context("spawn").Pool(n)


def check_full(pairs_dev, spec, n: int, slices: int = 64, nproc: int | None = None):
    """Compares the complete sorted GPU list of the workload `spec` (n subscriptions)
    with the oracle, slice by slice; returns the oracle's total K.  Raises
    AssertionError on the first mismatch."""
    import torch
    K = int(pairs_dev.shape[0])
    bounds = np.linspace(0, n, slices + 1).astype(np.int64)
    col = pairs_dev[:, 0].contiguous()
    pos = torch.searchsorted(col, torch.from_numpy(bounds.astype(np.int32)).to(col.device))
    pos = pos.cpu().numpy().astype(np.int64)
    assert pos[0] == 0 and pos[-1] == K, "pairs with a subscription id out of range"
    path = _store(pairs_dev, K)
    try:
        jobs = [(spec, int(bounds[s]), int(bounds[s + 1]), int(pos[s]), int(pos[s + 1]), path, K)
                for s in range(slices) if bounds[s + 1] > bounds[s]]
        with _pool(nproc) as pool:
            res = pool.map(_check_subs, jobs, chunksize=1)
    finally:
        os.unlink(path)
    bad = [r for r in res if not r[3]]
    assert not bad, f"subscriptions [{bad[0][0]}, {bad[0][1]}): {bad[0][4]}"
    total = sum(r[2] for r in res)
    assert total == K, (total, K)
    return total


def check_batch(pairs_dev, offs, num: int, replica: int = 0, d: int = 2, alpha: float = 1.0,
                chunk: int = 64, nproc: int | None = None):
    """Compares every instance of synth.batch_instances(num, replica, d, alpha) with
    the oracle; pairs_dev rows offs[b]:offs[b+1] are instance b's (local ids)."""
    K = int(pairs_dev.shape[0])
    offs = np.asarray(offs, dtype=np.int64)
    assert offs[0] == 0 and offs[-1] == K and np.all(np.diff(offs) >= 0)
    path = _store(pairs_dev, K)
    spec = ("batch", (num, replica, d, alpha))
    try:
        jobs = [(spec, b0, min(num, b0 + chunk), offs[b0:min(num, b0 + chunk) + 1].tolist(),
                 path, K) for b0 in range(0, num, chunk)]
        with _pool(nproc) as pool:
            res = pool.map(_check_instances, jobs, chunksize=1)
    finally:
        os.unlink(path)
    bad = [r for r in res if not r[3]]
    assert not bad, bad[0][4]
    assert sum(r[2] for r in res) == K
    return K
