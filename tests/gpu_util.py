"""Helpers for the GPU tests (CUDA path through the C ABI vs the CPU oracle)."""
from __future__ import annotations

import numpy as np


def to_dev(reg, device="cuda:0"):
    import torch
    return [torch.from_numpy(np.ascontiguousarray(a)).to(device)
            for a in (reg.sub_lo, reg.sub_hi, reg.upd_lo, reg.upd_hi)]


def gpu_pairs(ctx, reg) -> np.ndarray:
    return ctx.match(*to_dev(reg)).cpu().numpy()
