"""Replica sharding of the Lanczos GW path over several GPUs.

Every (t, m) start vector is an independent recurrence, so the path shards
without any exchange during the k Lanczos steps.  Two layouts:

* whole targets per rank (weak scaling): no communication at all;
* the summed set of one target split over ranks: each rank runs the
  recurrences of its share of m, the ranks gather their tridiagonals
  (B x k x 16 bytes -- the only exchange), and one rank evaluates the
  spectral map, the continued fractions summed over all m (Eq. 10) and the
  QP equation from the gathered coefficients (lgw_sigma_from_coeffs).

This module is torch.distributed plumbing only; the arithmetic is in the
library.
"""
from __future__ import annotations

from typing import Sequence, Tuple

import torch
import torch.distributed as dist


def shard_range(n: int, rank: int, world: int) -> Tuple[int, int]:
    """Contiguous [lo, hi) share of n items for `rank` of `world` (sizes
    differ by at most one)."""
    base, extra = divmod(n, world)
    lo = rank * base + min(rank, extra)
    return lo, lo + base + (1 if rank < extra else 0)


def gather_coefficients(alpha: torch.Tensor, beta: torch.Tensor, beta0: torch.Tensor,
                        k_eff: torch.Tensor, n_m_total: int, group=None):
    """All-gather per-rank tridiagonals of one target set whose summed
    orbitals were sharded with `shard_range`.

    Each rank passes its [n_t, n_m_local, k] / [n_t, n_m_local] arrays;
    returns the full [n_t * n_m_total, k] / [n_t * n_m_total] arrays in the
    vector order t_index * n_m_total + m_index that lgw_sigma_from_coeffs
    expects (on every rank)."""
    world = dist.get_world_size(group)
    n_t, _, k = alpha.shape

    def pad_gather(x):
        # ranks may hold different shares: pad to the largest share
        parts_n = [shard_range(n_m_total, r, world) for r in range(world)]
        width = max(hi - lo for lo, hi in parts_n)
        shape = list(x.shape)
        shape[1] = width
        buf = torch.zeros(shape, dtype=x.dtype, device=x.device)
        buf[:, : x.shape[1]] = x
        out = [torch.empty_like(buf) for _ in range(world)]
        dist.all_gather(out, buf, group=group)
        return torch.cat([o[:, : hi - lo] for o, (lo, hi) in zip(out, parts_n)], dim=1)

    a = pad_gather(alpha).reshape(n_t * n_m_total, k)
    b = pad_gather(beta).reshape(n_t * n_m_total, k)
    b0 = pad_gather(beta0).reshape(n_t * n_m_total)
    ke = pad_gather(k_eff).reshape(n_t * n_m_total)
    return a.contiguous(), b.contiguous(), b0.contiguous(), ke.contiguous()


def max_over_ranks(value: float, device=None, group=None) -> float:
    """Largest value over all ranks (the slowest rank's time)."""
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX, group=group)
    return float(t.item())


def targets_for_step(step: int, rank: int, world: int, per_step: int,
                     n_targets: int) -> Sequence[int]:
    """Targets rank `rank` processes in benchmark step `step`: consecutive
    blocks of `per_step`, interleaved over ranks, cycling over n_targets."""
    off = ((step * world + rank) * per_step) % n_targets
    return [(off + i) % n_targets for i in range(per_step)]
