"""Splitting one source across ranks (one process per GPU).

The offsets of a source are independent, so the path partitions into
horizontal bands of offset rows: rank r owns offset rows [v0, v1) and needs
source rows [v0, v1 + H - 1) (an H - 1 row halo).  Sum tables of the band
alone give the same box sums as the full table, because every box sum is a
difference of table entries, so each rank runs the unchanged single-GPU path
on its band and no data-path collective is needed.  The only exchange is
the final gather of the (few) match records to one rank.
"""
from __future__ import annotations

from dataclasses import dataclass
from typing import List, Optional, Sequence

import numpy as np


@dataclass(frozen=True)
class Band:
    rank: int
    v0: int            # first offset row owned
    v1: int            # one past the last offset row owned
    src_y0: int        # first source row needed
    src_y1: int        # one past the last source row needed

    @property
    def empty(self) -> bool:
        return self.v1 <= self.v0


def bands(N: int, H: int, world: int) -> List[Band]:
    """Balanced bands of offset rows for `world` ranks (V = N - H + 1 rows;
    the first V % world ranks get one extra row)."""
    if world < 1 or H < 1 or H > N:
        raise ValueError("need 1 <= H <= N and world >= 1")
    V = N - H + 1
    base, extra = divmod(V, world)
    out, v = [], 0
    for r in range(world):
        n = base + (1 if r < extra else 0)
        out.append(Band(r, v, v + n, v, v + n + H - 1 if n > 0 else v))
        v += n
    return out


def to_global(band: Band, U: int, u: np.ndarray, v_local: np.ndarray) -> np.ndarray:
    """Linear offset indices v*U + u of the full source for a band's matches."""
    return (np.asarray(v_local, np.int64) + band.v0) * U + np.asarray(u, np.int64)


def merge(parts: Sequence[tuple]) -> tuple:
    """Merges per-rank (index, rho) arrays into one list sorted by index."""
    if not parts:
        return np.zeros(0, np.int64), np.zeros(0, np.float32)
    idx = np.concatenate([np.asarray(p[0], np.int64) for p in parts])
    rho = np.concatenate([np.asarray(p[1]) for p in parts])
    order = np.argsort(idx, kind="stable")
    if idx.size and np.any(np.diff(idx[order]) == 0):
        raise ValueError("two ranks reported the same offset")
    return idx[order], rho[order]


def gather_matches(idx: np.ndarray, rho: np.ndarray, dst: int = 0, group=None) -> Optional[tuple]:
    """Gathers every rank's (index, rho) arrays on rank `dst` with
    torch.distributed (any backend); returns the merged lists on `dst` and
    None elsewhere."""
    import torch.distributed as dist
    world = dist.get_world_size(group)
    rank = dist.get_rank(group)
    payload = (np.asarray(idx, np.int64), np.asarray(rho, np.float32))
    objs = [None] * world if rank == dst else None
    dist.gather_object(payload, objs, dst=dst, group=group)
    if rank != dst:
        return None
    return merge(objs)
