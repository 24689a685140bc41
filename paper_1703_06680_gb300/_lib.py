"""ctypes binding of the C ABI in include/ddm.h (argument marshalling only).

Every computation runs in the CUDA library; this module only turns torch
tensors (device memory) and numpy arrays (host memory) into the pointers and
sizes the C functions take.  If the library is missing the import of a
Context fails loudly: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

from . import build as _build

LIB_PATH = _build.LIB

DDM_OK = 0
DDM_ERR_INVALID = -1
DDM_ERR_CAPACITY = -2
DDM_ERR_NOMEM = -3
DDM_ERR_DEVICE_TIMEOUT = -4
DDM_ERR_CUDA = -5
DDM_ERR_INTERNAL = -6
MAX_DIMS = 8
PARAM_WIN_SHIFT = 1
PARAM_ND_PATH = 2
PARAM_PDL = 3
PARAM_SWEEP_DIM = 4
PARAM_SORT_ITEMS = 5
PARAM_JOIN_SHIFT = 6
PARAM_ND_WRITE = 7


class DDMError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{msg} (code {code})")
        self.code = code


class CapacityError(DDMError):
    def __init__(self, code: int, msg: str, K: int):
        super().__init__(code, msg)
        self.K = K


class Stats(ctypes.Structure):
    _fields_ = [("launches", ctypes.c_uint64), ("calls", ctypes.c_uint64),
                ("stage_ms", ctypes.c_float * 8), ("dim_order", ctypes.c_uint32 * 8),
                ("survivor_calls", ctypes.c_uint64)]


STAGE_NAMES = ["keybuild", "radix_sort", "sweep_scan", "counts", "offsets", "emit_setup", "emit",
               "segsort"]


class _Regions(ctypes.Structure):
    _fields_ = [("d", ctypes.c_int), ("n", ctypes.c_int64), ("m", ctypes.c_int64),
                ("sub_lo", ctypes.POINTER(ctypes.c_void_p)),
                ("sub_hi", ctypes.POINTER(ctypes.c_void_p)),
                ("upd_lo", ctypes.POINTER(ctypes.c_void_p)),
                ("upd_hi", ctypes.POINTER(ctypes.c_void_p))]


_lib = None
_lock = threading.Lock()
_P = ctypes.c_void_p
_U64P = ctypes.POINTER(ctypes.c_uint64)
_RP = ctypes.POINTER(_Regions)

# name -> (restype, argtypes) for every entry point of include/ddm.h
SIGNATURES = {
    "ddm_create": (ctypes.c_int, [ctypes.POINTER(_P), ctypes.c_int, _P, ctypes.c_size_t]),
    "ddm_destroy": (ctypes.c_int, [_P]),
    "ddm_last_error": (ctypes.c_char_p, [_P]),
    "ddm_count": (ctypes.c_int, [_P, _RP, _U64P]),
    "ddm_match": (ctypes.c_int, [_P, _RP, _P, ctypes.c_uint64, _U64P]),
    "ddm_match_host": (ctypes.c_int, [_P, _RP, _P, ctypes.c_uint64, _U64P]),
    "ddm_match_bruteforce": (ctypes.c_int, [_P, _RP, _P, ctypes.c_uint64, _U64P]),
    "ddm_match_itm": (ctypes.c_int, [_P, _RP, _P, ctypes.c_uint64, _U64P]),
    "ddm_match_grid": (ctypes.c_int, [_P, _RP, ctypes.c_uint32, _P, ctypes.c_uint64, _U64P, _P]),
    "ddm_debug_sweep": (ctypes.c_int, [_P, _RP, _P, _P, _P, _P, _P]),
    "ddm_set_profiling": (ctypes.c_int, [_P, ctypes.c_int]),
    "ddm_set_param": (ctypes.c_int, [_P, ctypes.c_int, ctypes.c_int64]),
    "ddm_count_noalloc": (ctypes.c_int, [_RP, _P, _U64P]),
    "ddm_match_batch": (ctypes.c_int, [_P, ctypes.c_int, _P, _P, ctypes.c_uint64, _P, _U64P]),
    "ddm_session_create": (ctypes.c_int, [ctypes.POINTER(_P), ctypes.c_int, _RP, ctypes.c_size_t]),
    "ddm_session_destroy": (ctypes.c_int, [_P]),
    "ddm_session_regions": (_RP, [_P]),
    "ddm_session_last_error": (ctypes.c_char_p, [_P]),
    "ddm_session_drift": (ctypes.c_int, [_P, _P, ctypes.c_uint64, ctypes.c_uint64, ctypes.c_double]),
    "ddm_session_count": (ctypes.c_int, [_P, _P, _U64P]),
    "ddm_session_emit": (ctypes.c_int, [_P, _P, _P, ctypes.c_uint64, _U64P]),
    "ddm_session_emit_delta": (ctypes.c_int, [_P, _P, _P, ctypes.c_uint64, _P, ctypes.c_uint64,
                                              _U64P, _U64P]),
    "ddm_session_K": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_uint64)]),
    "ddm_get_stats": (ctypes.c_int, [_P, ctypes.POINTER(Stats)]),
    "ddm_debug_wait_timeout": (ctypes.c_int, [_P, ctypes.c_int, ctypes.c_uint32]),
    "ddm_debug_write_pattern": (ctypes.c_int, [_P, ctypes.c_uint32, ctypes.c_uint32, ctypes.c_int,
                                               ctypes.c_int, ctypes.POINTER(ctypes.c_double),
                                               ctypes.POINTER(ctypes.c_uint64)]),
}


def load_library(path: str | None = None):
    """Loads libddm.so (built by build.build()); raises if it is missing."""
    global _lib
    with _lock:
        if _lib is not None and path is None:
            return _lib
        p = path or LIB_PATH
        if not os.path.exists(p):
            raise ImportError(f"CUDA library {p} is missing: run paper_1703_06680_gb300.build."
                              "build() (no CPU fallback exists)")
        lib = ctypes.CDLL(p)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        if path is None:
            _lib = lib
        return lib


def _torch():
    import torch
    return torch


class _Packed:
    """Keeps the pointer arrays of one ddm_regions alive."""

    def __init__(self, d, n, m, ptrs):
        self.arrays = [(ctypes.c_void_p * d)(*p) for p in ptrs]
        self.s = _Regions(d, n, m, *[ctypes.cast(a, ctypes.POINTER(ctypes.c_void_p))
                                     for a in self.arrays])

    @property
    def ref(self):
        return ctypes.byref(self.s)


def _pack_device(sub_lo, sub_hi, upd_lo, upd_hi):
    torch = _torch()
    ts = [sub_lo, sub_hi, upd_lo, upd_hi]
    for t in ts:
        if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.float32):
            raise TypeError("coordinates must be float32 CUDA tensors of shape (d, count)")
        if t.dim() != 2 or not t.is_contiguous():
            raise TypeError("coordinates must be contiguous (d, count) tensors")
    d, n = sub_lo.shape
    m = upd_lo.shape[1]
    if sub_hi.shape != (d, n) or upd_lo.shape[0] != d or upd_hi.shape != (d, m):
        raise ValueError("inconsistent coordinate shapes")
    ptrs = [[t.data_ptr() + 4 * k * t.shape[1] for k in range(d)] for t in ts]
    return _Packed(d, n, m, ptrs)


def _pack_host(sub_lo, sub_hi, upd_lo, upd_hi):
    arrs = [np.ascontiguousarray(a, dtype=np.float32) for a in (sub_lo, sub_hi, upd_lo, upd_hi)]
    d, n = arrs[0].shape
    m = arrs[2].shape[1]
    ptrs = [[a.ctypes.data + 4 * k * a.shape[1] for k in range(d)] for a in arrs]
    p = _Packed(d, n, m, ptrs)
    p.keep = arrs
    return p


NOALLOC_MAX_REGIONS = 1 << 17


def count_noalloc(sub_lo, sub_hi, upd_lo, upd_hi, stream=None) -> int:
    """ddm_count_noalloc: exact K without any allocation (no context needed).

    For callers that cannot allocate device memory.  Runs on the current CUDA
    device; n + m must not exceed NOALLOC_MAX_REGIONS.  Calls that overlap on
    the GPU share the library's fixed scratch and race: serialise them.
    """
    lib = load_library()
    torch = _torch()
    p = _pack_device(sub_lo, sub_hi, upd_lo, upd_hi)
    if p.s.n + p.s.m > NOALLOC_MAX_REGIONS:
        raise DDMError(DDM_ERR_INVALID, f"n + m = {p.s.n + p.s.m} exceeds the no-allocation "
                                        f"limit of {NOALLOC_MAX_REGIONS} regions")
    if stream is None:
        stream = torch.cuda.current_stream(sub_lo.device)
    K = ctypes.c_uint64(0)
    rc = lib.ddm_count_noalloc(p.ref, ctypes.c_void_p(stream.cuda_stream), ctypes.byref(K))
    if rc != DDM_OK:
        raise DDMError(rc, "ddm_count_noalloc failed")
    return int(K.value)


class Context:
    """A library context bound to one device and one CUDA stream."""

    def __init__(self, device: int = 0, stream=None, mem_budget: int = 0):
        self._lib = load_library()
        torch = _torch()
        if stream is None:
            stream = torch.cuda.current_stream(device)
        self.device = device
        self.stream = stream
        handle = ctypes.c_void_p()
        rc = self._lib.ddm_create(ctypes.byref(handle), device, ctypes.c_void_p(stream.cuda_stream),
                                  mem_budget)
        if rc != DDM_OK:
            raise DDMError(rc, "ddm_create failed")
        self._h = handle

    def close(self):
        if getattr(self, "_h", None):
            self._lib.ddm_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def _check(self, rc: int, K: int | None = None):
        if rc == DDM_OK:
            return
        msg = self._lib.ddm_last_error(self._h).decode(errors="replace")
        if rc == DDM_ERR_CAPACITY:
            raise CapacityError(rc, msg, int(K or 0))
        raise DDMError(rc, msg)

    def set_param(self, param: int, value: int):
        self._check(self._lib.ddm_set_param(self._h, param, value))

    def set_profiling(self, on: bool, stage: int | None = None):
        """Per-stage CUDA events: on=True records every stage boundary; with `stage`
        (an index into STAGE_NAMES) only that stage is bracketed."""
        mode = 0 if not on else (1 if stage is None else 2 + int(stage))
        self._check(self._lib.ddm_set_profiling(self._h, mode))

    def stats(self) -> dict:
        s = Stats()
        self._check(self._lib.ddm_get_stats(self._h, ctypes.byref(s)))
        return {"launches": int(s.launches), "calls": int(s.calls),
                "stage_ms": dict(zip(STAGE_NAMES, [float(x) for x in s.stage_ms])),
                "dim_order": [int(x) for x in s.dim_order],
                "survivor_calls": int(s.survivor_calls)}

    # -- entry points ----------------------------------------------------------
    def count(self, sub_lo, sub_hi, upd_lo, upd_hi) -> int:
        """ddm_count: exact number of intersecting pairs (device tensors)."""
        p = _pack_device(sub_lo, sub_hi, upd_lo, upd_hi)
        K = ctypes.c_uint64(0)
        self._check(self._lib.ddm_count(self._h, p.ref, ctypes.byref(K)))
        return int(K.value)

    def match_packed(self, packed, out) -> int:
        """ddm_match with descriptors packed once by pack(); out is a (cap, 2) int32 tensor."""
        K = ctypes.c_uint64(0)
        cap = out.shape[0]
        rc = self._lib.ddm_match(self._h, packed.ref, ctypes.c_void_p(out.data_ptr() if cap else 0),
                                 cap, ctypes.byref(K))
        self._check(rc, K.value)
        return int(K.value)

    @staticmethod
    def pack(sub_lo, sub_hi, upd_lo, upd_hi):
        return _pack_device(sub_lo, sub_hi, upd_lo, upd_hi)

    def match_into(self, out, sub_lo, sub_hi, upd_lo, upd_hi) -> int:
        """ddm_match into a preallocated (cap, 2) int32 CUDA tensor; returns K."""
        torch = _torch()
        if not (out.is_cuda and out.dtype == torch.int32 and out.is_contiguous()):
            raise TypeError("out must be a contiguous int32 CUDA tensor")
        p = _pack_device(sub_lo, sub_hi, upd_lo, upd_hi)
        K = ctypes.c_uint64(0)
        cap = out.numel() // 2
        rc = self._lib.ddm_match(self._h, p.ref, ctypes.c_void_p(out.data_ptr() if cap else 0),
                                 cap, ctypes.byref(K))
        self._check(rc, K.value)
        return int(K.value)

    def match(self, sub_lo, sub_hi, upd_lo, upd_hi, cap: int | None = None):
        """ddm_match; returns the sorted (K, 2) int32 pairs as a CUDA tensor."""
        torch = _torch()
        if cap is None:
            cap = self.count(sub_lo, sub_hi, upd_lo, upd_hi)
        out = torch.empty((max(cap, 1), 2), dtype=torch.int32, device=sub_lo.device)
        K = self.match_into(out[:cap] if cap else out[:0], sub_lo, sub_hi, upd_lo, upd_hi)
        return out[:K]

    def _baseline(self, fn, tensors, cap, count_only):
        torch = _torch()
        p = _pack_device(*tensors)
        K = ctypes.c_uint64(0)
        if count_only:
            self._check(fn(self._h, p.ref, None, 0, ctypes.byref(K)), K.value)
            return int(K.value)
        if cap is None:
            cap = self._baseline(fn, tensors, None, True)
        out = torch.empty((max(cap, 1), 2), dtype=torch.int32, device=tensors[0].device)
        rc = fn(self._h, p.ref, ctypes.c_void_p(out.data_ptr()), cap, ctypes.byref(K))
        self._check(rc, K.value)
        return out[:K.value]

    def match_bruteforce(self, sub_lo, sub_hi, upd_lo, upd_hi, cap: int | None = None,
                         count_only: bool = False):
        """ddm_match_bruteforce (Algorithm 2 on the GPU): sorted (K, 2) int32 pairs,
        or K with count_only=True."""
        return self._baseline(self._lib.ddm_match_bruteforce, (sub_lo, sub_hi, upd_lo, upd_hi),
                              cap, count_only)

    def match_itm(self, sub_lo, sub_hi, upd_lo, upd_hi, cap: int | None = None,
                  count_only: bool = False):
        """ddm_match_itm (Algorithm 3, interval tree, on the GPU): sorted (K, 2) int32
        pairs, or K with count_only=True."""
        return self._baseline(self._lib.ddm_match_itm, (sub_lo, sub_hi, upd_lo, upd_hi), cap,
                              count_only)

    def match_grid(self, sub_lo, sub_hi, upd_lo, upd_hi, cells_per_dim: int = 0,
                   cap: int | None = None, count_only: bool = False):
        """ddm_match_grid (grid-based matching on the GPU): sorted (K, 2) int32 pairs, or
        K with count_only=True.  The cells used per gridded dimension are kept in
        self.last_grid."""
        torch = _torch()
        p = _pack_device(sub_lo, sub_hi, upd_lo, upd_hi)
        K = ctypes.c_uint64(0)
        grid = (ctypes.c_uint32 * 3)()
        fn = self._lib.ddm_match_grid
        if count_only or cap is None:
            self._check(fn(self._h, p.ref, cells_per_dim, None, 0, ctypes.byref(K), grid), K.value)
            self.last_grid = list(grid)
            if count_only:
                return int(K.value)
            cap = int(K.value)
        out = torch.empty((max(cap, 1), 2), dtype=torch.int32, device=sub_lo.device)
        rc = fn(self._h, p.ref, cells_per_dim, ctypes.c_void_p(out.data_ptr()), cap,
                ctypes.byref(K), grid)
        self._check(rc, K.value)
        self.last_grid = list(grid)
        return out[:K.value]

    def match_host(self, sub_lo, sub_hi, upd_lo, upd_hi, cap: int | None = None,
                   out: np.ndarray | None = None):
        """ddm_match_host: numpy (d, count) float32 inputs, numpy (K, 2) int32 output."""
        p = _pack_host(sub_lo, sub_hi, upd_lo, upd_hi)
        if out is None:
            if cap is None:
                raise ValueError("give cap or a preallocated out array")
            out = np.empty((cap, 2), np.int32)
        cap = out.shape[0]
        K = ctypes.c_uint64(0)
        rc = self._lib.ddm_match_host(self._h, p.ref, ctypes.c_void_p(out.ctypes.data), cap,
                                      ctypes.byref(K))
        self._check(rc, K.value)
        return out[:K.value]

    @staticmethod
    def pack_batch(instances):
        """Packs the descriptors of a list of instances once, for repeated match_batch calls."""
        packs = [_pack_device(*inst) for inst in instances]
        arr = (_Regions * max(len(packs), 1))(*[p.s for p in packs])
        return {"packs": packs, "arr": arr, "num": len(packs),
                "device": instances[0][0].device if instances else None}

    def match_batch_packed(self, pack, out=None, offs=None):
        """ddm_match_batch on a pack_batch() result; out: (cap, 2) int32 CUDA tensor or None
        (count only).  Returns (K, inst_offsets)."""
        num = pack["num"]
        if offs is None:
            offs = np.zeros(num + 1, np.uint64)
        K = ctypes.c_uint64(0)
        cap = 0 if out is None else out.shape[0]
        rc = self._lib.ddm_match_batch(self._h, num, ctypes.cast(pack["arr"], ctypes.c_void_p),
                                       ctypes.c_void_p(out.data_ptr() if out is not None else 0),
                                       cap, ctypes.c_void_p(offs.ctypes.data), ctypes.byref(K))
        self._check(rc, K.value)
        return int(K.value), offs

    def match_batch(self, instances, cap: int | None = None, count_only: bool = False):
        """ddm_match_batch over a list of (sub_lo, sub_hi, upd_lo, upd_hi) CUDA tensors.

        Returns (pairs, inst_offsets): pairs is a (K, 2) int32 CUDA tensor whose rows
        inst_offsets[b]:inst_offsets[b+1] are instance b's sorted pairs (local ids);
        inst_offsets is a numpy uint64 array of len(instances) + 1.  With
        count_only=True no pairs are written and pairs is None.
        """
        torch = _torch()
        packs = [_pack_device(*inst) for inst in instances]
        num = len(packs)
        arr = (_Regions * max(num, 1))(*[p.s for p in packs])
        offs = np.zeros(num + 1, np.uint64)
        K = ctypes.c_uint64(0)
        if count_only:
            rc = self._lib.ddm_match_batch(self._h, num, ctypes.cast(arr, ctypes.c_void_p), None, 0,
                                           ctypes.c_void_p(offs.ctypes.data), ctypes.byref(K))
            self._check(rc, K.value)
            return None, offs
        if cap is None:
            _, o = self.match_batch(instances, count_only=True)
            cap = int(o[-1])
        dev = instances[0][0].device if num else torch.device("cuda", self.device)
        out = torch.empty((max(cap, 1), 2), dtype=torch.int32, device=dev)
        rc = self._lib.ddm_match_batch(self._h, num, ctypes.cast(arr, ctypes.c_void_p),
                                       ctypes.c_void_p(out.data_ptr()), cap,
                                       ctypes.c_void_p(offs.ctypes.data), ctypes.byref(K))
        self._check(rc, K.value)
        return out[:K.value], offs

    def debug_wait_timeout(self, which: int, spin_limit: int = 4096):
        """ddm_debug_wait_timeout: runs a bounded device wait against a hand-off that
        never comes (0 = look-back, 1 = mbarrier); raises DDMError (expected code
        DDM_ERR_DEVICE_TIMEOUT)."""
        self._check(self._lib.ddm_debug_wait_timeout(self._h, int(which), int(spin_limit)))

    def debug_write_pattern(self, nseg: int, mean_len: int, scattered: bool = True,
                            reps: int = 5):
        """ddm_debug_write_pattern: the emission's store pattern without its filter.
        Returns (fastest ms, bytes written per run)."""
        ms = ctypes.c_double(0.0)
        nbytes = ctypes.c_uint64(0)
        self._check(self._lib.ddm_debug_write_pattern(self._h, int(nseg), int(mean_len),
                                                      1 if scattered else 0, int(reps),
                                                      ctypes.byref(ms), ctypes.byref(nbytes)))
        return ms.value, nbytes.value
    def debug_sweep(self, sub_lo, sub_hi, upd_lo, upd_hi):
        """ddm_debug_sweep: (sorted_who, subset_size, updset_size, sub_count, upd_count)."""
        torch = _torch()
        p = _pack_device(sub_lo, sub_hi, upd_lo, upd_hi)
        n, m = p.s.n, p.s.m
        E = 2 * (n + m)
        dev = sub_lo.device
        outs = [torch.zeros(max(k, 1), dtype=torch.int32, device=dev) for k in (E, E, E, n, m)]
        rc = self._lib.ddm_debug_sweep(self._h, p.ref, *[ctypes.c_void_p(o.data_ptr()) for o in outs])
        self._check(rc)
        self.stream.synchronize()
        return tuple(o[:k] for o, k in zip(outs, (E, E, E, n, m)))


class Session:
    """Resident state of one simulation (ddm_session_*): coordinates and pipeline
    workspace stay on the device across timesteps."""

    def __init__(self, sub_lo, sub_hi, upd_lo, upd_hi, device: int = 0, mem_budget: int = 0):
        self._lib = load_library()
        p = _pack_device(sub_lo, sub_hi, upd_lo, upd_hi)
        self.d, self.n, self.m = p.s.d, p.s.n, p.s.m
        self.device = device
        h = ctypes.c_void_p()
        rc = self._lib.ddm_session_create(ctypes.byref(h), device, p.ref, mem_budget)
        if rc != DDM_OK:
            raise DDMError(rc, "ddm_session_create failed")
        self._h = h
        self._K_last = 0   # K of the last count phase
        self._K_ref = 0    # K of the reference list of emit_delta()
        self._counted = False  # a count phase is held (count() since the last drift/emit)

    def close(self):
        if getattr(self, "_h", None):
            self._lib.ddm_session_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, rc, K=0):
        if rc == DDM_OK:
            return
        msg = self._lib.ddm_session_last_error(self._h).decode(errors="replace")
        if rc == DDM_ERR_CAPACITY:
            raise CapacityError(rc, msg, int(K))
        raise DDMError(rc, msg)

    @staticmethod
    def _stream(stream):
        return ctypes.c_void_p(stream.cuda_stream if stream is not None else 0)

    @property
    def K(self) -> int:
        """K of the last count phase (count(), or a report that counted itself)."""
        return self._K_last

    def drift(self, seed: int, step: int, sigma: float, stream=None):
        self._check(self._lib.ddm_session_drift(self._h, self._stream(stream), seed & (2**64 - 1),
                                                step, float(sigma)))
        self._counted = False

    def count(self, stream=None) -> int:
        K = ctypes.c_uint64(0)
        self._check(self._lib.ddm_session_count(self._h, self._stream(stream), ctypes.byref(K)))
        self._K_last = int(K.value)
        self._counted = True
        return int(K.value)

    def emit(self, out, stream=None) -> int:
        """Writes the pairs of the last count() into `out` ((cap, 2) int32 CUDA tensor)."""
        K = ctypes.c_uint64(0)
        cap = out.shape[0]
        rc = self._lib.ddm_session_emit(self._h, self._stream(stream),
                                        ctypes.c_void_p(out.data_ptr() if cap else 0), cap,
                                        ctypes.byref(K))
        self._check(rc, K.value)
        self._counted = False
        return int(K.value)

    def emit_delta(self, added=None, removed=None, stream=None):
        """Change report of this timestep against the previous emit_delta():
        returns (added, removed) as (rows, 2) int32 CUDA tensors, each sorted.  Given
        output tensors are filled and sliced; otherwise they are allocated at the
        bounds (this timestep's K and the previous report's K), for which the
        timestep is counted first.  With given tensors, a timestep not counted
        yet is counted by the report itself (one library call)."""
        import torch
        dev = torch.device("cuda", self.device)
        if (added is None or removed is None) and not self._counted:
            self.count(stream)
        if added is None:
            added = torch.empty((max(self._K_last, 1), 2), dtype=torch.int32, device=dev)
        if removed is None:
            removed = torch.empty((max(self._K_ref, 1), 2), dtype=torch.int32, device=dev)
        na, nr = ctypes.c_uint64(0), ctypes.c_uint64(0)
        rc = self._lib.ddm_session_emit_delta(
            self._h, self._stream(stream), ctypes.c_void_p(added.data_ptr()), added.shape[0],
            ctypes.c_void_p(removed.data_ptr()), removed.shape[0], ctypes.byref(na),
            ctypes.byref(nr))
        self._check(rc, max(na.value, nr.value))
        K = ctypes.c_uint64(0)
        self._check(self._lib.ddm_session_K(self._h, ctypes.byref(K)))
        self._K_last = self._K_ref = int(K.value)
        self._counted = False
        return added[:na.value], removed[:nr.value]

    def packed(self):
        """The resident coordinates as a packed descriptor for Context.match_packed
        (device pointers into the session's memory, no copy; valid while the
        session lives)."""
        r = self._lib.ddm_session_regions(self._h).contents
        ptrs = [[arr[k] for k in range(self.d)] for arr in (r.sub_lo, r.sub_hi, r.upd_lo,
                                                             r.upd_hi)]
        p = _Packed(self.d, self.n, self.m, ptrs)
        p.owner = self
        return p

    def coords(self):
        """Copies of the resident coordinates as (d, count) float32 CUDA tensors."""
        import torch
        r = self._lib.ddm_session_regions(self._h).contents
        out = []
        for arr, count in ((r.sub_lo, self.n), (r.sub_hi, self.n), (r.upd_lo, self.m),
                           (r.upd_hi, self.m)):
            t = torch.empty((self.d, count), dtype=torch.float32, device=f"cuda:{self.device}")
            for k in range(self.d):
                if count:
                    src = _DeviceView(arr[k], count)
                    t[k].copy_(torch.as_tensor(src, device=f"cuda:{self.device}"))
            out.append(t)
        return out


class _DeviceView:
    """Minimal __cuda_array_interface__ over a device float32 pointer."""

    def __init__(self, ptr, count):
        self.__cuda_array_interface__ = {"shape": (count,), "typestr": "<f4",
                                         "data": (int(ptr), False), "version": 3}
