"""Independent B-scans across GPUs: every rank reconstructs its own scans and no
data crosses ranks (the reconstruction of one B-scan couples all its A-scans
through the lateral FFT, so a scan never spans ranks).

`assign` splits a list of scans over ranks by a greedy byte-balanced rule (the
largest remaining scan goes to the least-loaded rank), `max_over_ranks` is the
host-side reduction of a timing that the benchmark reports.
"""
from __future__ import annotations

from typing import Sequence


def scan_bytes(nx: int, nz: int, m: int) -> int:
    """Device bytes that one FP32 solve streams per iteration: four images and
    five measurement arrays (z^k, z^{k-1}, z^{k-2} / v, the adjoint output; y,
    Phi z, r and the two operator intermediates)."""
    return 4 * 8 * nx * nz + 5 * 4 * nx * m


def assign(sizes: Sequence[int], world_size: int) -> list[list[int]]:
    """Indices of `sizes` per rank: greedy longest-first onto the least-loaded rank
    (ties to the lower rank); deterministic for a given input."""
    if world_size < 1:
        raise ValueError("world_size must be >= 1")
    order = sorted(range(len(sizes)), key=lambda i: (-sizes[i], i))
    load = [0] * world_size
    out: list[list[int]] = [[] for _ in range(world_size)]
    for i in order:
        r = min(range(world_size), key=lambda k: (load[k], k))
        out[r].append(i)
        load[r] += sizes[i]
    for lst in out:
        lst.sort()
    return out


def max_over_ranks(value: float, group=None) -> float:
    """Maximum of a host float over the ranks of the default process group (or
    the value itself when torch.distributed is not initialised)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return float(value)
    backend = dist.get_backend(group)
    dev = torch.device("cuda", torch.cuda.current_device()) if backend == "nccl" else torch.device("cpu")
    t = torch.tensor([float(value)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX, group=group)
    return float(t.item())
