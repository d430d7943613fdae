"""Several GPUs or processes: each integrates its own independent shift set of
the same lattice (no exchange on the data path); the one exchange is the
gather of the per-shift values Q^(k) (m x 2 doubles per rank), after which
every rank forms the same Eq. (3) estimate over all m x world shifts through
qmc_combine_shifts.  Works with any torch.distributed backend (gloo on CPU,
nccl on GPUs)."""
from __future__ import annotations

import numpy as np

from . import qmc


def combine_across_ranks(per_shift, group=None) -> qmc.qmc_result:
    """All-gather per_shift [m, 2] from every rank (rank order) and return the
    combined estimate; identical on every rank."""
    import torch
    import torch.distributed as dist
    local = torch.as_tensor(np.ascontiguousarray(per_shift, dtype=np.float64).reshape(-1, 2))
    if dist.get_backend(group) == "nccl":
        local = local.cuda()
    sizes = [torch.zeros(1, dtype=torch.int64, device=local.device) for _ in range(dist.get_world_size(group))]
    dist.all_gather(sizes, torch.tensor([local.shape[0]], dtype=torch.int64, device=local.device), group=group)
    mmax = int(max(s.item() for s in sizes))
    padded = torch.zeros((mmax, 2), dtype=torch.float64, device=local.device)
    padded[: local.shape[0]] = local
    bufs = [torch.zeros_like(padded) for _ in sizes]
    dist.all_gather(bufs, padded, group=group)
    rows = np.concatenate([b[: int(s.item())].cpu().numpy() for b, s in zip(bufs, sizes)], axis=0)
    return qmc.qmc_combine_shifts(rows)
