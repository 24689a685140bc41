"""Helpers for the GPU tests (CUDA path through the C ABI vs the CPU oracle)."""
from __future__ import annotations

import numpy as np

import oracle


def to_dev(reg, device="cuda:0"):
    import torch
    return [torch.from_numpy(np.ascontiguousarray(a)).to(device)
            for a in (reg.sub_lo, reg.sub_hi, reg.upd_lo, reg.upd_hi)]


def gpu_pairs(ctx, reg) -> np.ndarray:
    return ctx.match(*to_dev(reg)).cpu().numpy()


def segment_of(pairs_dev, i: int):
    """Rows of sub i in a sorted (K, 2) CUDA tensor, as numpy."""
    import torch
    col = pairs_dev[:, 0].contiguous()
    key = torch.tensor([i, i + 1], dtype=torch.int32, device=col.device)
    a, b = torch.searchsorted(col, key).tolist()
    return pairs_dev[a:b].cpu().numpy()


def oracle_row(reg, i: int) -> np.ndarray:
    """Matches of S_i alone, by brute force (Algorithm 2) over all updates."""
    one = type(reg)(reg.sub_lo[:, i:i + 1].copy(), reg.sub_hi[:, i:i + 1].copy(),
                    reg.upd_lo, reg.upd_hi)
    p = oracle.bruteforce(one)
    p[:, 0] = i
    return p
