"""Replicas over disjoint shift batches: the multi-GPU form of the QMC estimate.

Every shift batch of the randomised lattice is an independent estimate
(Section 2.1), so N GPUs run N replicas of the same problem with disjoint
shifts and only the per-shift log means are gathered: log p_hat is the
log-sum-exp over all shifts of all ranks, and the error is the standard error
of that mean, exactly as one solve over the union of the shifts would give.
The gather is one all_gather of M doubles per rank (any torch.distributed
backend; gloo on CPU in the tests).
"""
from __future__ import annotations

import numpy as np


def rank_seed(seed: int, rank: int, n_shifts: int) -> int:
    """Seed of a rank's shift batches: the library draws shift s of a call seeded
    `q` as splitmix64 outputs q-relative; ranks use disjoint seeds."""
    return int(seed) + int(rank) * (1 << 32)


def combine(per_shift_logs) -> tuple[float, float]:
    """(log p_hat, err) from per-shift log means, pooled over replicas: the replicas'
    values are concatenated here and the estimate is the library's
    (tlrmvn_estimate_pooled, float64 on the host)."""
    from .api import tlrmvn_estimate_pooled
    ell = np.concatenate([np.asarray(x, dtype=np.float64).ravel() for x in per_shift_logs])
    return tlrmvn_estimate_pooled(ell)


def gather_and_combine(per_shift_log, group=None) -> tuple[float, float]:
    """all_gather each rank's per-shift log means, then combine (every rank gets the result)."""
    import torch
    import torch.distributed as dist
    local = torch.as_tensor(np.asarray(per_shift_log, dtype=np.float64))
    sizes = [torch.zeros(1, dtype=torch.int64) for _ in range(dist.get_world_size(group))]
    dist.all_gather(sizes, torch.tensor([local.numel()], dtype=torch.int64), group=group)
    width = int(max(s.item() for s in sizes))
    padded = torch.full((width,), float("nan"), dtype=torch.float64)
    padded[:local.numel()] = local
    parts = [torch.empty(width, dtype=torch.float64) for _ in sizes]
    dist.all_gather(parts, padded, group=group)
    return combine([p[:int(s.item())].numpy() for p, s in zip(parts, sizes)])
