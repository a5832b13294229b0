"""Partition of a collision batch across ranks (one process per GPU).

Every evaluation Q(g, f) of a batch is independent (the operator is local in
x, paper Sec. 2.1), so a batch of pairs or cells shards into contiguous,
balanced slices with no exchange on the data path: each rank evaluates its
slice with its own grid handle and writes its own outputs.  A rank needs the
spectra of the inputs its slice uses; the r^3 projection of a slice is the
corresponding slice of T along (j, l).
"""
from __future__ import annotations


def shard_range(n_units: int, world: int, rank: int) -> range:
    """Contiguous slice of [0, n_units) owned by `rank`; sizes differ by at most 1."""
    if world < 1 or not 0 <= rank < world or n_units < 0:
        raise ValueError("need world >= 1, 0 <= rank < world, n_units >= 0")
    base, extra = divmod(n_units, world)
    start = rank * base + min(rank, extra)
    return range(start, start + base + (1 if rank < extra else 0))


def shard_pairs(pairs, world: int, rank: int):
    """The rank's slice of an ordered pair (or cell) list, with the global indices."""
    r = shard_range(len(pairs), world, rank)
    return [pairs[e] for e in r], r


def inputs_used(pairs) -> list[int]:
    """Distinct input indices a slice of pairs reads (what the rank must hold)."""
    return sorted({i for pr in pairs for i in pr})
