"""The identity behind the batch posting ranges (host logic, no GPU).

In a batch self-search every query record's posting list is narrowed to the
record's own genome.  The library finds these ranges by walking the index:
the entries with one hash in one genome form a run, and that run is the
narrowed range of each of its records; each range is stored at its record
through the rank of the record's position among all record positions (a
bitmap with a count of set bits before each 32-bit word).  Both facts are
checked here against their definitions on the oracle's sketch and index of a
small batch, with numpy standing in for the device code."""
import numpy as np

import oracle
from paper_1807_00205_gb300 import synth


def _batch():
    gs = [synth.small_case(s, lengths=(L,), n_sd=3, mask_frac=0.25) for s, L in
          ((11, 40_000), (12, 9_000), (13, 25_000), (14, 700), (15, 31_000))]
    seq = np.concatenate([g.seq for g in gs])
    off = np.concatenate([[0], np.cumsum([len(g.seq) for g in gs])]).astype(np.int64)
    return seq, off


def test_runs_of_equal_hash_and_genome_are_the_narrowed_ranges():
    seq, off = _batch()
    pd = oracle.params(self_mode=2)
    recs = oracle.sketch(seq, off, pd)
    idx, toff = oracle.index(recs, pd["k"])
    genome = np.searchsorted(off, idx[:, 1], side="right") - 1
    # definition: the postings of the record's hash with positions in its genome
    want = {}
    for h, p in recs[:, :2]:
        st, en = int(toff[h]), int(toff[h + 1])
        g = np.searchsorted(off, p, side="right") - 1
        pos = idx[st:en, 1]
        a = st + int(np.searchsorted(pos, off[g], side="left"))
        b = st + int(np.searchsorted(pos, off[g + 1], side="left"))
        want[int(p)] = (a, b - a)
    # the walk: runs of equal (hash, genome) over the index
    key = idx[:, 0].astype(np.int64) * (len(off) + 1) + genome
    start = np.r_[True, key[1:] != key[:-1]]
    first = np.maximum.accumulate(np.where(start, np.arange(len(idx)), 0))
    end = np.r_[key[1:] != key[:-1], True]
    last = np.minimum.accumulate(np.where(end, np.arange(len(idx)), len(idx))[::-1])[::-1]
    got = {int(p): (int(f), int(l - f + 1)) for p, f, l in zip(idx[:, 1], first, last)}
    assert got == want
    assert len(got) == len(recs)  # positions are unique: one record per position


def test_position_rank_is_the_record_index():
    seq, off = _batch()
    recs = oracle.sketch(seq, off, oracle.params(self_mode=2))
    pos = recs[:, 1].astype(np.int64)
    nw = (int(off[-1]) + 31) // 32
    bits = np.zeros(nw, dtype=np.uint32)
    np.bitwise_or.at(bits, pos >> 5, (np.uint32(1) << (pos & 31).astype(np.uint32)))
    pop = np.array([bin(int(w)).count("1") for w in bits], dtype=np.int64)
    before = np.r_[0, np.cumsum(pop)[:-1]]
    below = (np.uint32(1) << (pos & 31).astype(np.uint32)) - np.uint32(1)
    rank = before[pos >> 5] + np.array([bin(int(v)).count("1") for v in bits[pos >> 5] & below])
    assert np.array_equal(rank, np.arange(len(recs)))
