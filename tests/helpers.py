"""Shared test helpers: golden fixtures and small adversarial instances."""
from __future__ import annotations

import os

import numpy as np

import synth

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def regions(sub_lo, sub_hi, upd_lo, upd_hi) -> synth.Regions:
    f = lambda a: np.asarray(a, np.float32).reshape(len(a) if np.ndim(a) > 1 else 1, -1)
    return synth.Regions(f(sub_lo), f(sub_hi), f(upd_lo), f(upd_hi))


def load_intersect_table():
    rows = []
    with open(os.path.join(GOLDEN, "intersect_1d.txt")) as fh:
        for line in fh:
            line = line.split("#", 1)[0].strip()
            if not line:
                continue
            a, b, c, d, e = line.split()
            rows.append((float(a), float(b), float(c), float(d), int(e)))
    return rows


def load_fig1():
    subs, upds, pairs = {}, {}, []
    with open(os.path.join(GOLDEN, "fig1.txt")) as fh:
        for line in fh:
            line = line.split("#", 1)[0].strip()
            if not line:
                continue
            tok = line.split()
            if tok[0] == "P":
                pairs.append((int(tok[1]), int(tok[2])))
            else:
                (subs if tok[0] == "S" else upds)[int(tok[1])] = [float(t) for t in tok[2:]]

    def arr(dct, col):
        return [[dct[i][2 * k + col] for i in sorted(dct)] for k in range(2)]

    reg = synth.Regions(*(np.asarray(x, np.float32) for x in
                          (arr(subs, 0), arr(subs, 1), arr(upds, 0), arr(upds, 1))))
    return reg, np.asarray(pairs, np.int32).reshape(-1, 2)


def tiny_grid_instance(rng: np.random.Generator, d: int, n: int, m: int, grid: int = 8):
    """Integer coordinates in {0..grid-1}: dense ties and degenerate intervals."""
    def ext(count):
        a = rng.integers(0, grid, size=(d, count))
        b = rng.integers(0, grid, size=(d, count))
        return np.minimum(a, b).astype(np.float32), np.maximum(a, b).astype(np.float32)
    s_lo, s_hi = ext(n)
    u_lo, u_hi = ext(m)
    return synth.Regions(s_lo, s_hi, u_lo, u_hi)


SPECIALS = np.array([-np.inf, -1.0, -0.0, 0.0, 1e-45, 1.0, 1.0000001, 2.0, np.inf], np.float32)


def special_value_instance(rng: np.random.Generator, d: int, n: int, m: int):
    """Coordinates drawn from signed zeros, infinities, a denormal and adjacent ulps."""
    def ext(count):
        a = SPECIALS[rng.integers(0, len(SPECIALS), size=(d, count))]
        b = SPECIALS[rng.integers(0, len(SPECIALS), size=(d, count))]
        lo = np.where(a <= b, a, b).astype(np.float32)
        hi = np.where(a <= b, b, a).astype(np.float32)
        return lo, hi
    s_lo, s_hi = ext(n)
    u_lo, u_hi = ext(m)
    return synth.Regions(s_lo, s_hi, u_lo, u_hi)


def grid_point_pairs(reg: synth.Regions, grid: int = 8) -> np.ndarray:
    """Pairs whose extents share a point of the integer grid in every dimension.

    For integer endpoints, two closed intervals intersect iff they share an
    integer point (the larger lower bound is one).  This enumerates points, so
    it does not use the Intersect-1D formula.
    """
    t = np.arange(grid, dtype=np.float32)
    both = np.ones((reg.n, reg.m), bool)
    for k in range(reg.d):
        ms = (reg.sub_lo[k][:, None] <= t) & (t <= reg.sub_hi[k][:, None])
        mu = (reg.upd_lo[k][:, None] <= t) & (t <= reg.upd_hi[k][:, None])
        both &= (ms.astype(np.int32) @ mu.T.astype(np.int32)) > 0
    i, j = np.nonzero(both)
    return np.stack([i, j], axis=1).astype(np.int32) if len(i) else np.zeros((0, 2), np.int32)


def as_set(pairs: np.ndarray) -> set:
    return set(map(tuple, np.asarray(pairs).reshape(-1, 2).tolist()))


def is_lex_sorted(pairs: np.ndarray) -> bool:
    if len(pairs) < 2:
        return True
    key = pairs[:, 0].astype(np.int64) << 32 | pairs[:, 1].astype(np.int64)
    return bool(np.all(np.diff(key) > 0))
