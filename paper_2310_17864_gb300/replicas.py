"""Replicas across GPUs: how a multi-GPU run of the benchmark combines ranks.

Alignments of different utterances are independent (no exchange step), and a
single utterance does not split across GPUs (its state axis would need a
cross-GPU hand-off every frame). So N GPUs run N replicas, each aligning its
own batch: the work per GPU is fixed (weak scaling), there is no data-path
collective, and the only communication is the timing: the job's time is the
slowest rank's, and its throughput is the units of all ranks over that time.
"""
from __future__ import annotations


def slowest(ms: float, dist=None, device=None) -> float:
    """The largest `ms` over the ranks of the default process group (the
    value itself without one). `device`: where the reduction tensor lives
    (a CUDA device for NCCL, None / "cpu" for gloo)."""
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return float(ms)
    import torch
    t = torch.tensor([float(ms)], dtype=torch.float64, device=device if device is not None else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(units_per_rank: float, world: int, ms: float) -> float:
    """Units per second of the whole job: every rank's units over the slowest rank's time."""
    if ms <= 0:
        raise ValueError("non-positive time")
    return world * units_per_rank / (ms / 1e3)


def prints(rank: int) -> bool:
    """Only rank 0 prints the result line (and runs the host-side baselines)."""
    return rank == 0
