"""Host-side logic of a sharded half (Eq. 3: the subproblems of a half are
independent, so the units can be split across processes).

Each rank takes a contiguous range of units (columns for the F half, rows
for the W half) holding about the same number of nonzeros, updates those
units, and the updated factor is reassembled by an all-gather of the
ranks' unit-major row blocks. Because every unit's coordinate order is keyed
by (seed, sweep, side, unit), the result does not depend on the partition.

Only the partition and the exchange live here; the per-unit work is the
CUDA library's (or, in the CPU tests, the oracle's).

One sharded step (sharded_step) is the whole hot path on P ranks: the F half
on each rank's columns, an all-gather of F's unit-major rows, the W half on
each rank's rows, an all-gather of W's rows, and Eq. 1 as the all-reduced sum
of the ranks' data terms plus the linear term sum_k sumW_k sumF_k.
"""
from __future__ import annotations

import numpy as np


def partition(ptr, world: int) -> list[tuple[int, int]]:
    """Contiguous unit ranges [lo, hi) for `world` ranks, split where the
    running nonzero count crosses k * nnz / world (ties to the left). Every
    unit belongs to exactly one range; ranges may be empty."""
    if world < 1:
        raise ValueError("world must be >= 1")
    ptr = np.asarray(ptr, dtype=np.int64)
    units = ptr.size - 1
    nnz = int(ptr[-1])
    cuts = [0]
    for k in range(1, world):
        target = (nnz * k) // world
        # first unit whose start offset reaches the target
        cut = int(np.searchsorted(ptr[:-1], target, side="left")) if units else 0
        cuts.append(max(cuts[-1], min(cut, units)))
    cuts.append(units)
    return [(cuts[k], cuts[k + 1]) for k in range(world)]


def gather_units(local, ranges, rank: int, group=None):
    """All-gather of unit-major blocks: `local` is this rank's (hi - lo) x ldr
    block of a factor (torch tensor); returns the full (units x ldr) factor on
    every rank, blocks in rank order. Uses torch.distributed (any backend)."""
    import torch
    import torch.distributed as dist

    world = len(ranges)
    lo, hi = ranges[rank]
    if local.shape[0] != hi - lo:
        raise ValueError("local block has %d rows, range holds %d" % (local.shape[0], hi - lo))
    ldr = local.shape[1]
    width = max(h - l for l, h in ranges)
    # equal-size buffers for all_gather; padded rows are dropped afterwards
    buf = torch.zeros((width, ldr), dtype=local.dtype, device=local.device)
    buf[: hi - lo] = local
    out = [torch.empty_like(buf) for _ in range(world)]
    dist.all_gather(out, buf, group=group)
    return torch.cat([out[k][: h - l] for k, (l, h) in enumerate(ranges)], dim=0)


def exchange_units(view, ranges, rank: int, group=None):
    """In-place all-gather of a factor's unit-major rows: `view` (units x ldr
    tensor) holds this rank's updated rows in its range; afterwards it holds
    every rank's."""
    lo, hi = ranges[rank]
    full = gather_units(view[lo:hi], ranges, rank, group)
    view.copy_(full)


def sharded_step(model, sweep: int, parts, rank: int, group=None) -> float:
    """One step of Algorithm 1 sharded over the ranks of `group`: parts[0] are
    the column ranges of the F half, parts[1] the row ranges of the W half (one
    per rank, from `partition`). `model` offers sweep_range(side, sweep, lo,
    hi) -> data term, factor_unit_major(side) -> tensor view and linear_term().
    Returns Eq. 1 at the new W and F (FP64), the same on every rank."""
    import torch
    import torch.distributed as dist

    lo, hi = parts[0][rank]
    model.sweep_range(0, sweep, lo, hi)
    view = model.factor_unit_major(0)
    exchange_units(view, parts[0], rank, group)
    if view.is_cuda:
        torch.cuda.synchronize(view.device)
    lo, hi = parts[1][rank]
    data = model.sweep_range(1, sweep, lo, hi)
    view = model.factor_unit_major(1)
    exchange_units(view, parts[1], rank, group)
    t = torch.tensor([data], dtype=torch.float64, device=view.device)
    dist.all_reduce(t, group=group)
    if view.is_cuda:
        torch.cuda.synchronize(view.device)
    return float(t.item()) + model.linear_term()
