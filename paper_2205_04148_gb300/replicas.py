"""Independent replicas on several GPUs of one node (one process per GPU).

The acoustic substep of one member needs no data from another member, so the
multi-GPU form here is replicas: every rank advances its own members (seeded
by its rank) and nothing is exchanged on the data path.  The only
collectives are the host-side barrier around the timed region and the
maximum of the per-rank times.  Ranks read RANK / LOCAL_RANK / WORLD_SIZE /
MASTER_ADDR / MASTER_PORT from the environment (torchrun).
"""
from __future__ import annotations

import os


def world():
    """(world size, rank, local rank) from the launcher's environment"""
    return (int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("RANK", "0")),
            int(os.environ.get("LOCAL_RANK", "0")))


def init(backend="nccl"):
    """Bind the rank to its GPU (nccl) and join the process group when the
    world has more than one rank; returns (world size, rank, local rank)."""
    ws, rank, local = world()
    if ws > 1:
        import torch
        import torch.distributed as D
        if backend == "nccl":
            torch.cuda.set_device(local)
        D.init_process_group(backend, init_method="env://")
    return ws, rank, local


def barrier():
    import torch.distributed as D
    if D.is_available() and D.is_initialized():
        D.barrier()


def max_over_ranks(x, device="cuda"):
    """the largest value of x over all ranks (x itself on a single rank)"""
    import torch.distributed as D
    if not (D.is_available() and D.is_initialized()):
        return x
    import torch
    t = torch.tensor([float(x)], device=device, dtype=torch.float64)
    D.all_reduce(t, op=D.ReduceOp.MAX)
    return float(t.item())


def member_seed(rank, member, stride=100):
    """seed of a rank's member: ranks draw disjoint members"""
    return stride * rank + member


def finish():
    import torch.distributed as D
    if D.is_available() and D.is_initialized():
        D.destroy_process_group()
