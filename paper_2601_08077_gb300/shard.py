"""Multi-rank helpers: the auxiliary-index sharding of the J/K build and the
bench's max-over-ranks timing.

The path shards over the auxiliary index P: rank r takes a contiguous run of
128-function blocks, computes rho_P for its P (rho_P needs only B_P), its
partial J = sum_{P in r} B_P rho_P and its partial K = sum over its blocks of
K_b (Eqs. df-j-2, df-k-2), and one sum all-reduce of J and one of K complete
the build.  Every machine this library runs on here has one GPU, so the GPU
path runs replicas; these helpers are the sharded design's host side, tested
with gloo ranks on the CPU.
"""
from __future__ import annotations

import torch
import torch.distributed as dist

AUX_BLOCK = 128


def aux_block_ranges(naux: int, world: int) -> list[tuple[int, int]]:
    """Contiguous [p0, p1) runs of whole 128-function blocks, one per rank,
    block counts differing by at most one (earlier ranks take the extra)."""
    if world < 1:
        raise ValueError("world must be >= 1")
    nblk = (naux + AUX_BLOCK - 1) // AUX_BLOCK
    base, extra = divmod(nblk, world)
    out, b0 = [], 0
    for r in range(world):
        nb = base + (1 if r < extra else 0)
        p0 = min(naux, b0 * AUX_BLOCK)
        p1 = min(naux, (b0 + nb) * AUX_BLOCK)
        out.append((p0, p1))
        b0 += nb
    return out


def allreduce_sum_(t: torch.Tensor) -> torch.Tensor:
    """In-place sum over the ranks of the default process group (no-op alone)."""
    if dist.is_available() and dist.is_initialized() and dist.get_world_size() > 1:
        dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return t


def max_over_ranks(value: float, device="cpu") -> float:
    """The largest of the ranks' values (the job's time is its slowest rank's)."""
    if dist.is_available() and dist.is_initialized() and dist.get_world_size() > 1:
        t = torch.tensor([float(value)], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        return float(t.item())
    return float(value)
