"""Seeded synthetic DDM workloads (subscription and update extents).

This module only draws inputs.  It holds none of the matching arithmetic, and
both the CPU oracle and the CUDA path consume what it returns.

Random numbers come from SplitMix64 (Steele, Lea and Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014), used as a counter-based
generator: draw number c of stream `seed` is mix(seed + (c + 1) * GAMMA).
A uniform double in [0, 1) is (x >> 11) * 2^-53.

The workload follows the paper's experimental methodology (Section 5,
"Experimental setup"): extents are placed uniformly at random on a routing
space of length L = 1e6, all with the same side length, and the overlapping
degree alpha = N * l / L fixes that length (l = alpha * L / N in one
dimension).  For d > 1 the side is L * (alpha / N) ** (1 / d), so that the
total volume of the extents is alpha times that of the routing space.

Coordinates are float32: lo = f32(L * u) and hi = f32(f64(lo) + side), both
rounded to nearest.  Because float32 is coarse near 1e6 (ulp 0.0625 above
2^19), equal coordinates occur in every configuration, and at alpha = 0.01
most extents collapse to points (hi == lo).
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)
ROUTING_SPACE = 1.0e6          # L in the paper's Section 5
SEED_BASE = 1703066800


def splitmix64(seed: int, count: int, offset: int = 0) -> np.ndarray:
    """Draws offset .. offset+count-1 of the SplitMix64 stream `seed` (uint64)."""
    c = np.arange(offset + 1, offset + count + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + c * GAMMA
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def uniform01(seed: int, count: int, offset: int = 0) -> np.ndarray:
    """Uniform float64 in [0, 1): (x >> 11) * 2^-53."""
    x = splitmix64(seed, count, offset) >> np.uint64(11)
    return x.astype(np.float64) * (2.0 ** -53)


@dataclasses.dataclass
class Regions:
    """d-dimensional extents, dimension-major float32 arrays of shape (d, count).

    sub_lo[k, i] is the lower bound of subscription S_i along dimension k;
    ids are 0-based positions in these arrays.
    """
    sub_lo: np.ndarray
    sub_hi: np.ndarray
    upd_lo: np.ndarray
    upd_hi: np.ndarray

    @property
    def d(self) -> int:
        return int(self.sub_lo.shape[0])

    @property
    def n(self) -> int:
        return int(self.sub_lo.shape[1])

    @property
    def m(self) -> int:
        return int(self.upd_lo.shape[1])

    def swapped(self) -> "Regions":
        """The same instance with the roles of subscriptions and updates exchanged."""
        return Regions(self.upd_lo, self.upd_hi, self.sub_lo, self.sub_hi)

    def subset_dims(self, d: int) -> "Regions":
        return Regions(self.sub_lo[:d], self.sub_hi[:d], self.upd_lo[:d], self.upd_hi[:d])


def _extents(seed: int, d: int, count: int, side: float, offset: int, L: float):
    lo = np.empty((d, count), np.float32)
    hi = np.empty((d, count), np.float32)
    for k in range(d):
        u = uniform01(seed, count, offset + k * count)
        lo[k] = (L * u).astype(np.float32)
        hi[k] = (lo[k].astype(np.float64) + side).astype(np.float32)
    return lo, hi


def make_regions(d: int, n: int, m: int, side: float, seed: int,
                 L: float = ROUTING_SPACE) -> Regions:
    """Uniform placement on [0, L)^d, equal sides; subscriptions drawn first."""
    s_lo, s_hi = _extents(seed, d, n, side, 0, L)
    u_lo, u_hi = _extents(seed, d, m, side, d * n, L)
    return Regions(s_lo, s_hi, u_lo, u_hi)


def make_regions_aniso(n: int, m: int, sides, seed: int, L: float = ROUTING_SPACE) -> Regions:
    """Uniform placement on [0, L)^d with a side of its own per dimension
    (dimension k drawn as a one-dimensional instance with side sides[k] and
    seed + k): extents that are long along some dimensions and short along
    others, for the choice of the swept dimension."""
    parts = [make_regions(1, n, m, float(sd), seed + k, L) for k, sd in enumerate(sides)]
    return Regions(*(np.concatenate([getattr(p, f) for p in parts], axis=0)
                     for f in ("sub_lo", "sub_hi", "upd_lo", "upd_hi")))


def side_for(alpha: float, N: int, d: int, L: float = ROUTING_SPACE) -> float:
    """Side length giving overlapping degree alpha for N extents in d dimensions."""
    if d == 1:
        return alpha * L / N
    if d == 2:
        return L * math.sqrt(alpha / N)
    return L * (alpha / N) ** (1.0 / d)


def seed_for(config_index: int, replica: int = 0) -> int:
    return SEED_BASE + 1000 * config_index + replica


# ----------------------------------------------------------------------------
# The five workload families (index 0..4 in the order they are listed).
# ----------------------------------------------------------------------------

def small_1d(replica: int = 0) -> Regions:
    """d=1, N=1e4 (5000 + 5000), alpha=1."""
    N = 10_000
    return make_regions(1, N // 2, N // 2, side_for(1.0, N, 1), seed_for(0, replica))


def large_1d(alpha: float, replica: int = 0, N: int = 1_000_000) -> Regions:
    """d=1, N=1e6 (500k + 500k), alpha in {0.01, 1, 100}."""
    return make_regions(1, N // 2, N - N // 2, side_for(alpha, N, 1), seed_for(1, replica))


def large_nd(d: int, alpha: float, replica: int = 0, N: int = 1_000_000) -> Regions:
    """d in {2, 3}, N=1e6, corners uniform in [0, L)^d, side L (alpha/N)^(1/d)."""
    return make_regions(d, N // 2, N - N // 2, side_for(alpha, N, d), seed_for(2, replica))


def batch_sizes(num: int = 4096, replica: int = 0, lo: float = 100.0,
                hi: float = 1.0e5) -> np.ndarray:
    """Per-instance region counts N_i = round(exp(U[ln lo, ln hi]))."""
    u = uniform01(seed_for(3, replica) ^ 0x5EED, num)
    N = np.rint(np.exp(math.log(lo) + u * (math.log(hi) - math.log(lo)))).astype(np.int64)
    return np.maximum(N, 2)


def batch_instance(k: int, sizes: np.ndarray, replica: int = 0, d: int = 2,
                   alpha: float = 1.0) -> Regions:
    """Instance k of the batch: n_k = floor(N_k / 2) subs, m_k = N_k - n_k updates."""
    N = int(sizes[k])
    n = N // 2
    return make_regions(d, n, N - n, side_for(alpha, N, d), seed_for(3, replica) + 7919 * (k + 1))


def batch_instances(num: int = 4096, replica: int = 0, d: int = 2, alpha: float = 1.0,
                    sizes: np.ndarray | None = None) -> list[Regions]:
    """Independent instances: n_i = floor(N_i / 2) subs, m_i = N_i - n_i updates."""
    if sizes is None:
        sizes = batch_sizes(num, replica)
    return [batch_instance(k, sizes, replica, d, alpha) for k in range(len(sizes))]


# ----------------------------------------------------------------------------
# Served workload: drift between timesteps.
# ----------------------------------------------------------------------------

def normal_draws(seed: int, step: int, count: int) -> np.ndarray:
    """Approximately standard-normal float64 draws, exact in integer arithmetic.

    Each draw is the Irwin-Hall sum of 12 uniforms: S = sum of twelve (x >> 11)
    values (an exact uint64 sum), z = (S - 6 * 2^53) * 2^-53, which has mean 0
    and variance 1.  Draw e of timestep `step` uses stream draws
    (step * count + e) * 12 .. +11.  The int64 -> float64 conversion rounds to
    nearest, so any IEEE implementation reproduces z bit for bit.
    """
    x = splitmix64(seed, 12 * count, 12 * count * step) >> np.uint64(11)
    s = x.reshape(count, 12).sum(axis=1, dtype=np.uint64)
    z = (s.astype(np.int64) - np.int64(6 << 53)).astype(np.float64) * (2.0 ** -53)
    return z


def drift(reg: Regions, seed: int, step: int, sigma: float) -> Regions:
    """Move every extent by delta ~ N(0, sigma) per dimension (same delta for lo and hi).

    delta = f32(z * sigma); lo' = fl32(lo + delta); hi' = fl32(hi + delta).  Rounding
    is monotone, so lo' <= hi' still holds.  Element e of a step is the region-
    dimension index: k * n + i for S_i, d * n + k * m + j for U_j.
    """
    d, n, m = reg.d, reg.n, reg.m
    z = normal_draws(seed, step, d * (n + m))
    delta = (z * sigma).astype(np.float32)
    ds = delta[: d * n].reshape(d, n)
    du = delta[d * n:].reshape(d, m)
    return Regions((reg.sub_lo + ds).astype(np.float32), (reg.sub_hi + ds).astype(np.float32),
                   (reg.upd_lo + du).astype(np.float32), (reg.upd_hi + du).astype(np.float32))


def served_simulations(num: int = 64, replica: int = 0, lo: float = 1.0e3,
                       hi: float = 1.0e6) -> list[dict]:
    """Per-simulation (N, d, alpha, seed): N log-uniform, d and alpha uniform."""
    base = seed_for(4, replica)
    u = uniform01(base, 3 * num).reshape(num, 3)
    sims = []
    for k in range(num):
        N = int(round(math.exp(math.log(lo) + u[k, 0] * (math.log(hi) - math.log(lo)))))
        d = 1 + min(2, int(u[k, 1] * 3))
        alpha = (0.01, 1.0, 100.0)[min(2, int(u[k, 2] * 3))]
        sims.append({"N": N, "d": d, "alpha": alpha, "seed": base + 104729 * (k + 1)})
    return sims


def simulation_regions(sim: dict) -> Regions:
    N, d = sim["N"], sim["d"]
    return make_regions(d, N // 2, N - N // 2, side_for(sim["alpha"], N, d), sim["seed"])
