"""Energy sharding across GPUs (one process per GPU).

Energies are independent: rank r of R solves the energies k with k % R == r of a common grid (or
its own interleaved sub-grid for weak scaling) with no exchange during the solve. The only
collective is one sum of integrated observables at the end (and, in the benchmark, a max of the
timings). Integrals over a grid that is split between ranks are assembled from per-rank partial
trapezoid sums, so the result equals the single-process integral.
"""
from __future__ import annotations

import numpy as np


def shard(n_E: int, rank: int, world: int) -> np.ndarray:
    """Indices of the energies owned by `rank` (round robin)."""
    if not (0 <= rank < world):
        raise ValueError("rank out of range")
    return np.arange(rank, n_E, world)


def interleaved_grid(E: np.ndarray, rank: int, world: int) -> np.ndarray:
    """Weak-scaling grid of one rank: the common grid shifted by rank/world of a spacing (a grid of
    one energy has no spacing and is returned as is)."""
    if world == 1 or len(E) < 2:
        return E
    return E + (E[1] - E[0]) * rank / world


def trapezoid_weights(E: np.ndarray) -> np.ndarray:
    """w such that sum(w * f(E)) is the trapezoid rule on the (sorted) grid E."""
    w = np.zeros_like(E, dtype=np.float64)
    d = np.diff(E)
    w[:-1] += 0.5 * d
    w[1:] += 0.5 * d
    return w


def partial_integral(E: np.ndarray, values: np.ndarray, owned: np.ndarray) -> np.ndarray:
    """This rank's share of the trapezoid integral of `values` (rows = owned energies)."""
    w = trapezoid_weights(E)[owned]
    return np.tensordot(w, values, axes=(0, 0))


def allreduce_sum(x: np.ndarray, group=None) -> np.ndarray:
    """Sum a host array over all ranks (torch.distributed). NCCL reduces device tensors only, so
    under that backend the array makes a round trip through the current CUDA device."""
    import torch
    import torch.distributed as dist
    t = torch.from_numpy(np.ascontiguousarray(x, dtype=np.float64))
    if dist.is_initialized() and dist.get_world_size(group) > 1:
        if dist.get_backend(group) == "nccl":
            d = t.to(torch.device("cuda", torch.cuda.current_device()))
            dist.all_reduce(d, op=dist.ReduceOp.SUM, group=group)
            return d.cpu().numpy()
        dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)
    return t.numpy()
