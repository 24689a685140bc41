"""The no-allocation count entry point (ddm_count_noalloc) against the oracle.

Some callers cannot allocate device memory (code running where cudaMalloc is
unavailable or forbidden); ddm_count_noalloc serves them from a fixed scratch
array inside the library.  Its K is checked against the CPU oracle's count
(and against ddm_count, the entry point that allocates), on two calls in a
row that share the same scratch.  This file is collected last so that a run
stopping at the first failure has already run every other test; it must pass
both alone in a fresh process and after the other tests.
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


def _case(name):
    if name == "d1":
        return synth.large_1d(100.0, N=120_000)
    if name == "d2":
        return synth.large_nd(2, 100.0, N=100_001)
    if name == "d3_tiny":
        return synth.make_regions(3, 37, 41, 3.0e5, 21)
    if name == "d8_at_limit":
        # n + m exactly at the limit with the most dimensions: the largest
        # scratch layout the entry point accepts.  A short side along dim 0
        # keeps the dim-0 candidates few; long sides elsewhere let pairs survive.
        half = (1 << 17) // 2
        return synth.make_regions_aniso(half, half, (2.0e3,) + (5.0e5,) * 7, 8181)
    return synth.Regions(*(np.zeros((1, 0), np.float32) for _ in range(4)))


@pytest.mark.parametrize("case", ["d1", "d2", "d3_tiny", "d8_at_limit", "empty"])
def test_count_noalloc_equals_oracle_twice(ddm, case):
    reg = _case(case)
    if case == "d8_at_limit":
        assert reg.n + reg.m == ddm.NOALLOC_MAX_REGIONS and reg.d == 8
    want = oracle.sbm_count(reg)
    t = to_dev(reg)
    # two calls in a row share the same scratch; both must give the oracle's K
    assert ddm.count_noalloc(*t) == want
    assert ddm.count_noalloc(*t) == want
    with ddm.Context(0) as ctx:
        assert ctx.count(*t) == want


def test_count_noalloc_rejects_oversize(ddm):
    import ctypes

    from paper_1703_06680_gb300._lib import _pack_device
    n = ddm.NOALLOC_MAX_REGIONS
    reg = synth.make_regions(1, n // 2 + 1, n // 2, 10.0, 5)
    t = to_dev(reg)
    with pytest.raises(ddm.DDMError) as e:
        ddm.count_noalloc(*t)
    assert e.value.code == -1
    # the C entry point itself rejects the size (DDM_ERR_INVALID)
    K = ctypes.c_uint64(123)
    rc = ddm.load_library().ddm_count_noalloc(_pack_device(*t).ref, None, ctypes.byref(K))
    assert rc == -1 and K.value == 123
