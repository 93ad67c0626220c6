"""Batched self-search of many independent genomes in one pass.

The genomes are concatenated into one input (each genome one sequence) and
the whole path runs once with self_mode = 2: every stage is one launch over
the batch, the filter and refine kernels are persistent and take windows and
runs from device work counters, and no work is spent between genomes (the
filter narrows each posting list to the query's own genome).  `plain` is the
one-genome-per-pass form the batch is compared with; both give identical
candidates.
"""
from __future__ import annotations

import numpy as np

from . import binding


def shard(items: list, rank: int, world: int) -> list:
    """The items rank `rank` of `world` processes: a contiguous block, sizes
    balanced by total length when items have `.length` (greedy by prefix)."""
    if world <= 1:
        return list(items)
    lengths = [getattr(x, "length", 1) for x in items]
    total = float(sum(lengths)) or 1.0
    out, acc = [], 0.0
    for x, ln in zip(items, lengths):
        mid = acc + ln / 2.0
        if int(mid * world / total) == rank or (rank == world - 1 and mid * world / total >= world):
            out.append(x)
        acc += ln
    return out


def concatenate(genomes) -> tuple:
    """(seq, offsets) of the genomes, one sequence per genome."""
    parts = [np.ascontiguousarray(g.seq, dtype=np.uint8) for g in genomes]
    offs = np.zeros(len(parts) + 1, dtype=np.int64)
    offs[1:] = np.cumsum([len(x) for x in parts])
    seq = np.concatenate(parts) if parts else np.zeros(0, dtype=np.uint8)
    return seq, offs


def split_candidates(cands: np.ndarray, ngenomes: int) -> list:
    """Per-genome candidate arrays (qseq/tseq reset to 0)."""
    out = []
    for gi in range(ngenomes):
        c = cands[cands["qseq"] == gi].copy()
        c["qseq"] = 0
        c["tseq"] = 0
        out.append(c)
    return out


def batched(ctx: "binding.Context", d_seq, offsets, p: "binding.Params") -> dict:
    """One pass over a device-resident batch (self_mode 2)."""
    q = binding.params_from_struct(p, self_mode=2)
    return ctx.selfsearch(d_seq, offsets, q)


def plain(ctx: "binding.Context", d_seqs, offsets_list, p: "binding.Params") -> list:
    """One pass per genome (self_mode 1)."""
    q = binding.params_from_struct(p, self_mode=1)
    return [ctx.selfsearch(d, off, q) for d, off in zip(d_seqs, offsets_list)]
