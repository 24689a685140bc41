"""The no-allocation count entry point (ddm_count_noalloc) against ddm_count.

Some callers cannot allocate device memory (code running where cudaMalloc is
unavailable or forbidden); ddm_count_noalloc serves them from a fixed scratch
array inside the library.  This file is collected last so that a run stopping
at the first failure has already run every other test; it must pass both alone
in a fresh process and after the other tests.
"""
import numpy as np
import pytest

import synth
from tests.gpu_util import to_dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ddm():
    import paper_1703_06680_gb300 as ddm
    ddm.build_library()
    return ddm


@pytest.mark.parametrize("case", ["d1", "d2", "d3_tiny", "empty"])
def test_count_noalloc_equals_count_twice(ddm, case):
    if case == "d1":
        reg = synth.large_1d(100.0, N=120_000)
    elif case == "d2":
        reg = synth.large_nd(2, 100.0, N=100_001)
    elif case == "d3_tiny":
        reg = synth.make_regions(3, 37, 41, 3.0e5, 21)
    else:
        reg = synth.Regions(*(np.zeros((1, 0), np.float32) for _ in range(4)))
    t = to_dev(reg)
    with ddm.Context(0) as ctx:
        want = ctx.count(*t)
    # two calls in a row share the same scratch; both must agree exactly
    assert ddm.count_noalloc(*t) == want
    assert ddm.count_noalloc(*t) == want


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
