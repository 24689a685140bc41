"""GB300 (sm_103a) Sort-Based Matching for Data Distribution Management.

Exact matching of subscription and update extents (d-dimensional
axis-parallel rectangles) after Marzolla and D'Angelo, "Parallel Sort-Based
Matching for Data Distribution Management on Shared-Memory Multiprocessors"
(DS-RT 2017).  The computation lives in the CUDA library declared by
include/ddm.h; this package is its thin Python binding.
"""
from ._lib import (CapacityError, Context, DDMError, LIB_PATH, NOALLOC_MAX_REGIONS,  # noqa: F401
                   Session, SIGNATURES, count_noalloc, load_library, STAGE_NAMES, PARAM_PDL, PARAM_SWEEP_DIM)
from .build import build as build_library  # noqa: F401
