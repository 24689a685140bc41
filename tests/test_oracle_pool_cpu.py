"""The pooled full-size parity helper (tests/oracle_pool.py), on the CPU.

The helper splits the oracle's work into subscription slices (or batches of
instances) run in spawn-started worker processes and compares each slice with
its rows of a given pair list.  Here the "GPU" list is the oracle's own answer
held in a CPU tensor: the helper must accept it, and must reject it after one
planted change, a dropped row, or an out-of-range id.
"""
import numpy as np
import pytest

import oracle
import synth
from tests.oracle_pool import check_batch, check_full


@pytest.fixture(scope="module")
def one_d():
    spec = ("large_1d", (1.0, 0, 20_000))
    reg = synth.large_1d(1.0, 0, 20_000)
    return spec, reg, oracle.sbm(reg)


def test_full_accepts_the_oracle_list(one_d):
    import torch
    spec, reg, want = one_d
    assert check_full(torch.from_numpy(want), spec, reg.n, slices=8, nproc=2) == len(want)


@pytest.mark.parametrize("plant", ["changed", "dropped", "out_of_range"])
def test_full_rejects_a_planted_mistake(one_d, plant):
    import torch
    spec, reg, want = one_d
    bad = want.copy()
    if plant == "changed":
        bad[len(bad) // 2, 1] += 1
    elif plant == "dropped":
        bad = np.delete(bad, len(bad) // 3, axis=0)
    else:
        bad[-1, 0] = reg.n
    with pytest.raises(AssertionError):
        check_full(torch.from_numpy(bad), spec, reg.n, slices=8, nproc=2)


def test_batch_accepts_and_rejects():
    import torch
    regs = synth.batch_instances(num=12, d=2)
    lists = [oracle.sbm(r) for r in regs]
    offs = np.concatenate([[0], np.cumsum([len(x) for x in lists])]).astype(np.int64)
    allp = np.concatenate(lists)
    assert check_batch(torch.from_numpy(allp), offs, 12, chunk=5, nproc=2) == len(allp)
    allp[offs[7] + 1, 1] ^= 1
    with pytest.raises(AssertionError):
        check_batch(torch.from_numpy(allp), offs, 12, chunk=5, nproc=2)
