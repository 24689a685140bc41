"""CPU oracle for exact DDM matching (test infrastructure only).

Only the tests, the package smoke check and the benchmark's CPU-baseline leg
may import this package.  It wraps `sbm_oracle.c` (serial Sort-Based Matching,
Algorithm 4, and Brute-Force matching, Algorithm 2, of the paper) with ctypes,
and shares no code with the CUDA library.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "sbm_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
EINVAL = -1
ENOMEM = -2

_lock = threading.Lock()
_libs: dict = {}


class OracleError(RuntimeError):
    pass


def build(mutant: int = 0, force: bool = False) -> str:
    """Compile the oracle with gcc (plain -O2, no architecture flags); return the .so path.

    `mutant` > 0 compiles a copy with a planted mistake (see ORACLE_MUTANT in the
    C source); the pin tests use those copies to show that they catch mistakes.
    """
    os.makedirs(_BUILD, exist_ok=True)
    name = "liboracle.so" if mutant == 0 else f"liboracle_mutant{mutant}.so"
    out = os.path.join(_BUILD, name)
    if force or not os.path.exists(out) or os.path.getmtime(out) < os.path.getmtime(_SRC):
        tmp = out + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=c11", "-shared", "-fPIC", f"-DORACLE_MUTANT={mutant}",
               _SRC, "-o", tmp]
        subprocess.run(cmd, check=True)
        os.replace(tmp, out)
    return out


def _lib(mutant: int = 0):
    with _lock:
        if mutant not in _libs:
            lib = ctypes.CDLL(build(mutant))
            f32p = ctypes.POINTER(ctypes.c_float)
            for fn in (lib.oracle_sbm, lib.oracle_bruteforce):
                fn.restype = ctypes.c_int64
                fn.argtypes = [ctypes.c_int, ctypes.c_int64, ctypes.c_int64, f32p, f32p, f32p,
                               f32p, ctypes.POINTER(ctypes.POINTER(ctypes.c_int32))]
            lib.oracle_sweep_trace.restype = ctypes.c_int64
            lib.oracle_sweep_trace.argtypes = [ctypes.c_int64, ctypes.c_int64, f32p, f32p, f32p,
                                               f32p, ctypes.c_void_p, ctypes.c_void_p,
                                               ctypes.c_void_p, ctypes.c_void_p]
            lib.oracle_free.restype = None
            lib.oracle_free.argtypes = [ctypes.c_void_p]
            _libs[mutant] = lib
        return _libs[mutant]


def _arrays(reg):
    d, n, m = reg.d, reg.n, reg.m
    arrs = [np.ascontiguousarray(a, dtype=np.float32).reshape(d, -1)
            for a in (reg.sub_lo, reg.sub_hi, reg.upd_lo, reg.upd_hi)]
    return d, n, m, arrs


def _ptr(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_float))


def _run(fn_name: str, reg, store: bool, mutant: int):
    lib = _lib(mutant)
    d, n, m, arrs = _arrays(reg)
    out = ctypes.POINTER(ctypes.c_int32)()
    K = getattr(lib, fn_name)(d, n, m, *[_ptr(a) for a in arrs],
                              ctypes.byref(out) if store else None)
    if K == EINVAL:
        raise OracleError("invalid input (NaN or lo > hi)")
    if K < 0:
        raise OracleError(f"oracle failed ({K})")
    if not store:
        return int(K)
    if K == 0:
        if out:
            lib.oracle_free(out)
        return np.zeros((0, 2), np.int32)
    res = np.ctypeslib.as_array(out, shape=(K, 2)).copy()
    lib.oracle_free(out)
    return res


def sbm(reg, mutant: int = 0) -> np.ndarray:
    """Algorithm 4 (dimension 0) + filter on dims 1..d-1; sorted (K, 2) int32 pairs."""
    return _run("oracle_sbm", reg, True, mutant)


def sbm_count(reg, mutant: int = 0) -> int:
    """K from Algorithm 4 without storing the pairs (the paper's measured mode)."""
    return _run("oracle_sbm", reg, False, mutant)


def bruteforce(reg, mutant: int = 0) -> np.ndarray:
    """Algorithm 2 over all n*m pairs and all dimensions; sorted (K, 2) int32 pairs."""
    return _run("oracle_bruteforce", reg, True, mutant)


def bruteforce_count(reg, mutant: int = 0) -> int:
    return _run("oracle_bruteforce", reg, False, mutant)


def sweep_trace(reg, mutant: int = 0):
    """Sorted endpoint order of dimension 0 and the active-set sizes after each endpoint.

    Returns (kind, id, subset_size, updset_size); kind is 0 S lower, 1 U lower,
    2 S upper, 3 U upper.
    """
    lib = _lib(mutant)
    _, n, m, arrs = _arrays(reg.subset_dims(1))
    E = 2 * (n + m)
    kind = np.empty(E, np.uint8)
    ids = np.empty(E, np.int32)
    ss = np.empty(E, np.int64)
    us = np.empty(E, np.int64)
    rc = lib.oracle_sweep_trace(n, m, *[_ptr(a) for a in arrs], kind.ctypes.data,
                                ids.ctypes.data, ss.ctypes.data, us.ctypes.data)
    if rc != 0:
        raise OracleError(f"oracle sweep failed ({rc})")
    return kind, ids, ss, us


def per_sub_counts(pairs: np.ndarray, n: int) -> np.ndarray:
    return np.bincount(pairs[:, 0], minlength=n).astype(np.int64) if len(pairs) else \
        np.zeros(n, np.int64)


def per_upd_counts(pairs: np.ndarray, m: int) -> np.ndarray:
    return np.bincount(pairs[:, 1], minlength=m).astype(np.int64) if len(pairs) else \
        np.zeros(m, np.int64)
