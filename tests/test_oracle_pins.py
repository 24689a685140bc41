"""Pins for the CPU oracle: checks against what the paper and mathematics fix.

None of these tests retypes the oracle's formulas.  Expected values come from
hand-written set semantics (golden tables), point enumeration on integer
grids, closed forms, invariants of the problem, and the agreement of two
independent algorithms (Algorithm 2 and Algorithm 4).  The mutation test at
the end shows that a planted mistake anywhere in the oracle fails a pin.
"""
import math

import numpy as np
import pytest

import oracle
import synth
from tests.helpers import (as_set, grid_point_pairs, is_lex_sorted, load_fig1,
                           load_intersect_table, regions, special_value_instance,
                           tiny_grid_instance)


# --- Algorithm 1 against hand-written set semantics ---------------------------

def check_intersect_table(mutant=0):
    bad = []
    for s_lo, s_hi, u_lo, u_hi, want in load_intersect_table():
        reg = regions([s_lo], [s_hi], [u_lo], [u_hi])
        for fn in (oracle.bruteforce, oracle.sbm):
            got = len(fn(reg, mutant=mutant))
            if got != want:
                bad.append((fn.__name__, s_lo, s_hi, u_lo, u_hi, want, got))
    return bad


def test_intersect_1d_table():
    assert check_intersect_table() == []


# --- Figure 1 pattern ------------------------------------------------------------

def check_fig1(mutant=0):
    reg, want = load_fig1()
    return [fn.__name__ for fn in (oracle.bruteforce, oracle.sbm)
            if not np.array_equal(fn(reg, mutant=mutant), want)]


def test_fig1_pattern():
    assert check_fig1() == []


# --- Brute force against point enumeration (integer grids) -----------------------

def check_grid_enumeration(mutant=0, seeds=200):
    rng = np.random.default_rng(1)
    for s in range(seeds):
        d = 1 + s % 3
        reg = tiny_grid_instance(rng, d, int(rng.integers(0, 24)), int(rng.integers(0, 24)))
        want = grid_point_pairs(reg)
        if not np.array_equal(oracle.bruteforce(reg, mutant=mutant), want):
            return ("bruteforce", s)
        if not np.array_equal(oracle.sbm(reg, mutant=mutant), want):
            return ("sbm", s)
    return None


def test_bruteforce_equals_grid_enumeration():
    assert check_grid_enumeration(seeds=600) is None


# --- SBM against brute force on many tiny instances --------------------------------

def test_sbm_equals_bruteforce_tiny_grid():
    rng = np.random.default_rng(2)
    for s in range(10_000):
        d = 1 + s % 3
        reg = tiny_grid_instance(rng, d, int(rng.integers(0, 65)), int(rng.integers(0, 65)))
        a = oracle.sbm(reg)
        b = oracle.bruteforce(reg)
        assert np.array_equal(a, b), s
        assert is_lex_sorted(a)


def test_sbm_equals_bruteforce_special_values():
    rng = np.random.default_rng(3)
    for s in range(2_000):
        d = 1 + s % 3
        reg = special_value_instance(rng, d, int(rng.integers(0, 40)), int(rng.integers(0, 40)))
        assert np.array_equal(oracle.sbm(reg), oracle.bruteforce(reg)), s


def test_sbm_equals_bruteforce_float_workload():
    # the small 1-D workload (N = 1e4, alpha = 1): float32 ties near 1e6 included
    reg = synth.small_1d()
    assert np.array_equal(oracle.sbm(reg), oracle.bruteforce(reg))


# --- Closed forms ----------------------------------------------------------------------

def closed_form_points_vs_windows(n, m, w):
    """S_i = [i, i] and U_j = [j, j + w]: U_j contains i iff i - w <= j <= i."""
    reg = regions(np.arange(n), np.arange(n), np.arange(m), np.arange(m) + w)
    want = [(i, j) for i in range(n) for j in range(max(0, i - w), min(m - 1, i) + 1)]
    return reg, np.asarray(want, np.int32).reshape(-1, 2)


def check_closed_forms(mutant=0):
    bad = []
    for n, m, w in [(50, 40, 0), (50, 40, 3), (7, 30, 10), (30, 7, 2)]:
        reg, want = closed_form_points_vs_windows(n, m, w)
        for fn in (oracle.bruteforce, oracle.sbm):
            if not np.array_equal(fn(reg, mutant=mutant), want):
                bad.append((fn.__name__, n, m, w))
    # every subscription equals every update: K = n * m
    reg = regions(np.full(9, 2.0), np.full(9, 3.0), np.full(7, 2.0), np.full(7, 3.0))
    for fn in (oracle.bruteforce, oracle.sbm):
        if len(fn(reg, mutant=mutant)) != 63:
            bad.append((fn.__name__, "all-equal"))
    # a 2-D lattice: unit boxes [a, a+1] x [b, b+1] against points (x, y): a box
    # holds the point iff a <= x <= a+1 and b <= y <= b+1
    pts = [(x, y) for x in range(4) for y in range(4)]
    boxes = [(a, b) for a in range(3) for b in range(3)]
    reg = synth.Regions(
        np.asarray([[a for a, b in boxes], [b for a, b in boxes]], np.float32),
        np.asarray([[a + 1 for a, b in boxes], [b + 1 for a, b in boxes]], np.float32),
        np.asarray([[x for x, y in pts], [y for x, y in pts]], np.float32),
        np.asarray([[x for x, y in pts], [y for x, y in pts]], np.float32))
    want = [(i, j) for i, (a, b) in enumerate(boxes) for j, (x, y) in enumerate(pts)
            if x in (a, a + 1) and y in (b, b + 1)]
    for fn in (oracle.bruteforce, oracle.sbm):
        if not np.array_equal(fn(reg, mutant=mutant), np.asarray(want, np.int32)):
            bad.append((fn.__name__, "lattice"))
    return bad


def test_closed_forms():
    assert check_closed_forms() == []


# --- Invariants of the problem ---------------------------------------------------------

def check_invariants(mutant=0, seeds=60):
    rng = np.random.default_rng(4)
    for s in range(seeds):
        d = 1 + s % 3
        reg = tiny_grid_instance(rng, d, int(rng.integers(1, 50)), int(rng.integers(1, 50)))
        p = oracle.sbm(reg, mutant=mutant)
        # swapping the roles of S and U transposes the list
        q = oracle.sbm(reg.swapped(), mutant=mutant)
        if as_set(p) != {(j, i) for i, j in as_set(q)}:
            return ("swap", s)
        # dropping a dimension can only add pairs
        if d > 1 and not as_set(p) <= as_set(oracle.sbm(reg.subset_dims(d - 1), mutant=mutant)):
            return ("monotone-d", s)
        # growing every extent can only add pairs
        grown = synth.Regions(reg.sub_lo - 1, reg.sub_hi + 1, reg.upd_lo, reg.upd_hi)
        if not as_set(p) <= as_set(oracle.sbm(grown, mutant=mutant)):
            return ("monotone-grow", s)
        # the count-only mode reports the length of the list
        if oracle.sbm_count(reg, mutant=mutant) != len(p):
            return ("count", s)
    return None


def test_invariants():
    assert check_invariants(seeds=300) is None


def test_empty_sets():
    reg = regions(np.zeros((1, 0)), np.zeros((1, 0)), [1.0], [2.0])
    assert len(oracle.sbm(reg)) == 0 and len(oracle.bruteforce(reg)) == 0
    reg = regions([1.0], [2.0], np.zeros((1, 0)), np.zeros((1, 0)))
    assert len(oracle.sbm(reg)) == 0 and len(oracle.bruteforce(reg)) == 0


@pytest.mark.parametrize("bad", ["nan", "reversed"])
def test_invalid_input_rejected(bad):
    lo, hi = [0.0, 1.0], [1.0, 2.0]
    if bad == "nan":
        lo[1] = float("nan")
    else:
        lo[1], hi[1] = 3.0, 2.0
    reg = regions(lo, hi, [0.5], [0.7])
    for fn in (oracle.sbm, oracle.bruteforce, oracle.sbm_count):
        with pytest.raises(oracle.OracleError):
            fn(reg)


# --- The sweep's active sets, against their definition ----------------------------------

def test_sweep_trace_against_definition():
    rng = np.random.default_rng(5)
    for s in range(200):
        reg = tiny_grid_instance(rng, 1, int(rng.integers(0, 30)), int(rng.integers(0, 30)))
        kind, ids, ss, us = oracle.sweep_trace(reg)
        E = len(kind)
        coord = np.where(kind == 0, reg.sub_lo[0][ids.clip(0, max(reg.n - 1, 0))] if reg.n else 0,
                         0).astype(np.float64)
        x = np.empty(E)
        for t in range(E):
            src = (reg.sub_lo, reg.upd_lo, reg.sub_hi, reg.upd_hi)[kind[t]]
            x[t] = src[0][ids[t]]
        # non-decreasing, and lowers before uppers at equal coordinates
        assert np.all(np.diff(x) >= 0)
        for t in range(E - 1):
            if x[t] == x[t + 1]:
                assert not (kind[t] >= 2 and kind[t + 1] < 2)
        # every endpoint appears exactly once
        for k, cnt in ((0, reg.n), (1, reg.m), (2, reg.n), (3, reg.m)):
            assert sorted(ids[kind == k].tolist()) == list(range(cnt))
        # |SubSet| after t = extents whose lower is at or before t and upper after t
        pos = {}
        for t in range(E):
            pos[(int(kind[t]) % 2, int(kind[t]) // 2, int(ids[t]))] = t
        for t in range(E):
            act_s = sum(1 for i in range(reg.n) if pos[(0, 0, i)] <= t < pos[(0, 1, i)])
            act_u = sum(1 for j in range(reg.m) if pos[(1, 0, j)] <= t < pos[(1, 1, j)])
            assert ss[t] == act_s and us[t] == act_u
        if E:
            assert ss[-1] == 0 and us[-1] == 0


# --- Statistical sanity (not an exactness pin) ---------------------------------------------

def test_expected_count_sanity():
    # E[K] = n m (2 l / L - (l / L)^2) for uniform starts in [0, L), no clipping
    N, alpha = 40_000, 1.0
    reg = synth.make_regions(1, N // 2, N // 2, synth.side_for(alpha, N, 1), 12345)
    l, L = synth.side_for(alpha, N, 1), synth.ROUTING_SPACE
    expect = (N // 2) ** 2 * (2 * l / L - (l / L) ** 2)
    K = oracle.sbm_count(reg)
    assert abs(K - expect) < 6 * math.sqrt(3 * expect), (K, expect)


# --- Mutation test: each planted mistake fails at least one pin ----------------------------

@pytest.mark.parametrize("mutant", [1, 2, 3, 4, 5])
def test_planted_mistakes_are_caught(mutant):
    caught = (check_intersect_table(mutant) != [] or check_fig1(mutant) != []
              or check_grid_enumeration(mutant, seeds=100) is not None
              or check_closed_forms(mutant) != [] or check_invariants(mutant, seeds=30) is not None)
    assert caught, f"mutant {mutant} passed every pin"
