"""Seeded synthetic genomes with planted segmental duplications.

This module only produces inputs.  It holds none of the seeding filter's
arithmetic (no k-mer codes, hashes, winnowing, counting or chaining), so both
the CUDA path and the CPU oracle may draw their inputs from it.

The shapes follow the workloads used to evaluate SEDEF: random sequences with
planted duplications (Section 4.1.1: copies mutated by point substitutions and
small indels, identity drawn per duplication, both orientations), soft-masked
interspersed repeats (Section 3.2 uses only k-mers with an unmasked base while
seeding) and runs of N, standing in for assembly gaps.

Every generator takes an explicit seed and uses numpy's PCG64, so a workload
is a pure function of its arguments.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

_ACGT = np.frombuffer(b"ACGT", dtype=np.uint8)
_COMP = np.zeros(256, dtype=np.uint8)
for _a, _b in zip(b"ACGTNacgtn", b"TGCANtgcan"):
    _COMP[_a] = _b


@dataclasses.dataclass
class PlantedSD:
    """One planted duplication: source [src, src+length) copied to dst."""

    src: int
    length: int
    dst: int
    copy_length: int
    reverse: bool
    identity: float


@dataclasses.dataclass
class Genome:
    """Concatenated ASCII sequences plus their boundaries.

    ``seq`` is uint8 ASCII; sequence ``s`` is ``seq[offsets[s]:offsets[s+1]]``.
    ``planted`` lists duplications in global coordinates.
    """

    seq: np.ndarray
    offsets: np.ndarray
    planted: list
    name: str = ""

    @property
    def length(self) -> int:
        return int(self.offsets[-1])

    @property
    def nseq(self) -> int:
        return len(self.offsets) - 1


def random_bases(rng: np.random.Generator, length: int, gc: float = 0.5) -> np.ndarray:
    """i.i.d. uppercase bases with the given GC fraction."""
    at = (1.0 - gc) / 2.0
    cg = gc / 2.0
    idx = rng.choice(4, size=length, p=[at, cg, cg, at]).astype(np.uint8)
    return _ACGT[idx]


def random_bases_chunked(rng: np.random.Generator, out: np.ndarray, gc: float = 0.5,
                         chunk: int = 1 << 24) -> None:
    """Fill ``out`` with i.i.d. uppercase bases, drawn in chunks so that
    gigabase sequences need no 8-byte-per-base temporaries."""
    c0, c1, c2 = (1.0 - gc) / 2.0, 0.5, 0.5 + gc / 2.0
    for a in range(0, len(out), chunk):
        u = rng.random(min(chunk, len(out) - a), dtype=np.float32)
        idx = (u >= c0).astype(np.uint8)
        idx += u >= c1
        idx += u >= c2
        out[a:a + len(u)] = _ACGT[idx]


def reverse_complement(seq: np.ndarray) -> np.ndarray:
    """Case-preserving reverse complement (N stays N)."""
    return _COMP[seq[::-1]]


def mutate(rng: np.random.Generator, seq: np.ndarray, identity: float,
           sub_frac: float = 0.8, indel_max: int = 5) -> np.ndarray:
    """Apply round((1-identity)*len) edit events to a copy of ``seq``.

    A fraction ``sub_frac`` of the events are substitutions to a different
    base; the rest are insertions or deletions (equally likely) of 1..indel_max
    bases.  Case is preserved: substituted and inserted bases take the case of
    the base at the event position.
    """
    seq = np.array(seq, dtype=np.uint8, copy=True)
    L = len(seq)
    n_ev = int(round((1.0 - identity) * L))
    if L == 0 or n_ev <= 0:
        return seq
    n_ev = min(n_ev, L)
    pos = np.sort(rng.choice(L, size=n_ev, replace=False))
    is_sub = rng.random(n_ev) < sub_frac
    lower = (seq >= ord("a")) & (seq <= ord("z"))

    sp = pos[is_sub]
    if len(sp):
        up = seq[sp] & 0xDF
        code = np.searchsorted(_ACGT, up)
        code = np.where(code < 4, code, 0)
        new = _ACGT[(code + rng.integers(1, 4, size=len(sp))) % 4]
        seq[sp] = np.where(lower[sp], new | 0x20, new)

    ip = pos[~is_sub]
    if len(ip) == 0:
        return seq
    ins = rng.random(len(ip)) < 0.5
    lens = rng.integers(1, indel_max + 1, size=len(ip))
    keep = np.ones(L, dtype=bool)
    for p, ln in zip(ip[~ins], lens[~ins]):
        keep[p:p + ln] = False
    ins_pos = ip[ins]
    ins_len = lens[ins]
    if len(ins_pos):
        where = np.repeat(ins_pos, ins_len)
        vals = _ACGT[rng.integers(0, 4, size=len(where))]
        vals = np.where(lower[where], vals | 0x20, vals)
        # insert before each position, then drop deleted bases
        tagged = np.insert(np.arange(L), where, -1)
        out = np.insert(seq, where, vals)
        ok = np.ones(len(out), dtype=bool)
        src_idx = tagged >= 0
        ok[src_idx] = keep[tagged[src_idx]]
        return out[ok]
    return seq[keep]


def log_uniform_int(rng, lo: int, hi: int, size=None):
    return np.exp(rng.uniform(math.log(lo), math.log(hi), size=size)).astype(np.int64)


def plant_duplications(rng, seq: np.ndarray, count: int, len_lo: int, len_hi: int,
                       id_lo: float, id_hi: float, rc_frac: float = 0.5,
                       offsets: np.ndarray | None = None,
                       inter_frac: float = 0.0, exact_half_rc: bool = False,
                       disjoint: bool = False) -> list:
    """Copy ``count`` random segments to random places (overwriting).

    Lengths are log-uniform in [len_lo, len_hi], identities uniform in
    [id_lo, id_hi].  Copies keep the case (mask) of their source.  With
    several sequences, a copy stays within its source's sequence unless it is
    drawn as inter-sequence (probability ``inter_frac``).  With ``disjoint``
    a duplication whose mates would overlap an earlier one's is redrawn (up
    to 50 times), so that every planted pair survives intact.  Returns the
    list of planted duplications in global coordinates.
    """
    total = len(seq)
    if offsets is None:
        offsets = np.array([0, total], dtype=np.int64)
    seq_len = np.diff(offsets)
    planted = []
    lengths = log_uniform_int(rng, len_lo, len_hi + 1, size=count)
    ids = rng.uniform(id_lo, id_hi, size=count)
    if exact_half_rc:
        rcs = np.zeros(count, dtype=bool)
        rcs[rng.permutation(count)[: count // 2]] = True
    else:
        rcs = rng.random(count) < rc_frac
    weights = seq_len / seq_len.sum()
    taken = []

    def clash(a, b):
        return any(a < y and x < b for x, y in taken)

    for L, ident, rc in zip(lengths, ids, rcs):
        L = int(L)
        for _attempt in range(50 if disjoint else 1):
            got = _draw_pair(rng, seq, offsets, seq_len, weights, L, float(ident), bool(rc),
                             inter_frac)
            if got is None:
                continue
            src, piece, dst = got
            if disjoint and (clash(src, src + L) or clash(dst, dst + len(piece))):
                continue
            seq[dst:dst + len(piece)] = piece
            taken.extend([(src, src + L), (dst, dst + len(piece))])
            planted.append(PlantedSD(src, L, dst, len(piece), bool(rc), float(ident)))
            break
    return planted


def _draw_pair(rng, seq, offsets, seq_len, weights, L, ident, rc, inter_frac):
    """Draw a source, mutate it, and draw a destination; None if it does not fit."""
    s_src = int(rng.choice(len(seq_len), p=weights))
    if seq_len[s_src] <= 2 * L:
        return None
    s_dst = s_src
    if len(seq_len) > 1 and rng.random() < inter_frac:
        s_dst = int(rng.choice(len(seq_len), p=weights))
        if seq_len[s_dst] <= 2 * L:
            s_dst = s_src
    src = int(offsets[s_src] + rng.integers(0, seq_len[s_src] - L))
    piece = mutate(rng, seq[src:src + L], ident)
    if rc:
        piece = reverse_complement(piece)
    room = int(seq_len[s_dst] - len(piece))
    if room <= 0:
        return None
    dst = int(offsets[s_dst] + rng.integers(0, room))
    if s_dst == s_src and abs(dst - src) < L + len(piece):
        # keep the two mates apart so that the pair is a duplication
        # rather than an overlapping overwrite
        return None
    return src, piece, dst


def add_masked_repeats(rng, seq: np.ndarray, frac: float, family_lengths=(300, 6000),
                       id_lo: float = 0.80, id_hi: float = 0.95, gc: float = 0.41) -> None:
    """Overwrite ``seq`` with lowercase (soft-masked) repeat copies.

    One random consensus per family length; copies carry substitutions only,
    at an identity drawn per copy in [id_lo, id_hi].  Enough copies are placed
    that the expected covered fraction is ``frac``; each family covers about
    the same number of bases.
    """
    total = len(seq)
    if frac <= 0 or total == 0:
        return
    placed_bases = -math.log(1.0 - frac) * total
    per_family = placed_bases / len(family_lengths)
    for flen in family_lengths:
        if flen >= total:
            continue
        cons = random_bases(rng, flen, gc)
        ncopy = max(1, int(per_family / flen))
        done = 0
        while done < ncopy:
            batch = min(ncopy - done, max(1, (1 << 24) // flen))
            ident = rng.uniform(id_lo, id_hi, size=(batch, 1))
            sub = rng.random((batch, flen)) >= ident
            codes = np.searchsorted(_ACGT, cons)
            rows = np.broadcast_to(codes, (batch, flen)).copy()
            rows[sub] = (rows[sub] + rng.integers(1, 4, size=int(sub.sum()))) % 4
            vals = _ACGT[rows] | 0x20
            starts = rng.integers(0, total - flen, size=batch)
            idx = (starts[:, None] + np.arange(flen)[None, :]).ravel()
            seq[idx] = vals.ravel()
            done += batch


def add_n_gaps(rng, seq: np.ndarray, every: int, len_lo: int, len_hi: int) -> list:
    """Overwrite a run of 'N' of length U[len_lo, len_hi] in every ``every`` bases."""
    gaps = []
    total = len(seq)
    for block in range(0, total, every):
        end = min(block + every, total)
        glen = int(rng.integers(len_lo, len_hi + 1))
        if end - block <= glen:
            continue
        g = int(block + rng.integers(0, end - block - glen))
        seq[g:g + glen] = ord("N")
        gaps.append((g, glen))
    return gaps


def genome_from_parts(parts: list, planted=None, name="") -> Genome:
    offs = np.zeros(len(parts) + 1, dtype=np.int64)
    offs[1:] = np.cumsum([len(p) for p in parts])
    seq = np.concatenate(parts) if parts else np.zeros(0, dtype=np.uint8)
    return Genome(np.ascontiguousarray(seq, dtype=np.uint8), offs, planted or [], name)


# ---------------------------------------------------------------------------
# Named workloads.  Seeds are 0x5EDEF000 + workload number.
# ---------------------------------------------------------------------------

def plain_2mbp(seed: int = 0x5EDEF001, length: int = 2_000_000, n_sd: int = 20) -> Genome:
    """2 Mbp i.i.d. uniform ACGT, 20 planted duplications of 1-20 kbp
    (log-uniform), half reverse-complemented, identity U[75, 99]%,
    uppercase, no N."""
    rng = np.random.default_rng(seed)
    seq = random_bases(rng, length, 0.5)
    planted = plant_duplications(rng, seq, n_sd, 1000, 20000, 0.75, 0.99,
                                 exact_half_rc=True)
    return genome_from_parts([seq], planted, "plain-2Mbp")


def chromosome_100mbp(seed: int = 0x5EDEF002, length: int = 100_000_000,
                      n_sd: int = 2000, sd_hi: int = 200_000,
                      mask_frac: float = 0.40) -> Genome:
    """Chromosome-scale self-search input: 41% GC, soft-masked repeat
    families of 300 bp and 6 kbp consensus (80-95% identity) covering about
    ``mask_frac`` of the bases, N-gaps of 10-50 kbp every ~10 Mbp and
    ``n_sd`` duplications of 1 kbp-``sd_hi`` (log-uniform) at 75-99.5%
    identity in both orientations."""
    rng = np.random.default_rng(seed)
    seq = random_bases(rng, length, 0.41)
    add_masked_repeats(rng, seq, mask_frac)
    planted = plant_duplications(rng, seq, n_sd, 1000, sd_hi, 0.75, 0.995)
    add_n_gaps(rng, seq, 10_000_000, 10_000, 50_000)
    return genome_from_parts([seq], planted, f"chromosome-{length // 1_000_000}Mbp")


def batch_genomes(seed: int = 0x5EDEF003, count: int = 200, len_lo: int = 1_000_000,
                  len_hi: int = 20_000_000, sd_lo: int = 50, sd_hi: int = 500,
                  max_genomes: int | None = None) -> list:
    """Independent genomes of log-uniform size, 41% GC, 30% soft-masked
    repeats, sd_lo..sd_hi planted duplications of 1-50 kbp at 75-99%.
    With max_genomes, only the first max_genomes of the same batch (the
    genomes are drawn one after another, so they are identical)."""
    rng = np.random.default_rng(seed)
    out = []
    sizes = log_uniform_int(rng, len_lo, len_hi + 1, size=count)
    if max_genomes is not None:
        sizes = sizes[:max_genomes]
    for g, L in enumerate(sizes):
        L = int(L)
        seq = random_bases(rng, L, 0.41)
        add_masked_repeats(rng, seq, 0.30)
        nsd = int(rng.integers(sd_lo, sd_hi + 1))
        planted = plant_duplications(rng, seq, nsd, 1000, 50_000, 0.75, 0.99)
        out.append(genome_from_parts([seq], planted, f"batch-{g}"))
    return out


def human_3gbp(seed: int = 0x5EDEF004, total: int = 3_100_000_000, nchrom: int = 24,
               len_lo: int = 50_000_000, len_hi: int = 250_000_000, n_sd: int = 20_000,
               sd_hi: int = 300_000, mask_frac: float = 0.50, inter_frac: float = 0.3) -> Genome:
    """Human-assembly-scale input: ``nchrom`` chromosomes of len_lo..len_hi
    bases summing to ``total``, 41% GC, soft-masked repeat families covering
    about ``mask_frac`` of each chromosome, N-gaps of 10-50 kbp every ~10 Mbp
    and ``n_sd`` duplications of 1 kbp-``sd_hi`` (log-uniform) at 75-99.5%
    identity, both orientations, a fraction ``inter_frac`` of them placed on
    another chromosome."""
    rng = np.random.default_rng(seed)
    share = rng.uniform(0.0, 1.0, size=nchrom)
    lengths = len_lo + np.floor((total - nchrom * len_lo) * share / share.sum()).astype(np.int64)
    lengths[-1] += total - lengths.sum()
    assert lengths.min() >= len_lo and lengths.max() <= len_hi
    offs = np.zeros(nchrom + 1, dtype=np.int64)
    offs[1:] = np.cumsum(lengths)
    seq = np.empty(total, dtype=np.uint8)
    for c in range(nchrom):
        sub = seq[offs[c]:offs[c + 1]]
        random_bases_chunked(rng, sub, 0.41)
        add_masked_repeats(rng, sub, mask_frac)
    planted = plant_duplications(rng, seq, n_sd, 1000, sd_hi, 0.75, 0.995, offsets=offs,
                                 inter_frac=inter_frac)
    for c in range(nchrom):
        add_n_gaps(rng, seq[offs[c]:offs[c + 1]], 10_000_000, 10_000, 50_000)
    return Genome(seq, offs, planted, f"human-{total / 1e9:.1f}Gbp")


def small_case(seed: int, lengths=(20_000,), n_sd: int = 3, sd_lo: int = 1000,
               sd_hi: int = 4000, id_lo: float = 0.85, id_hi: float = 0.99,
               mask_frac: float = 0.0, n_gaps: bool = False, gc: float = 0.5,
               inter_frac: float = 0.3, repeat_lengths=(60, 300)) -> Genome:
    """Small multi-sequence genome for parity and pin tests."""
    rng = np.random.default_rng(seed)
    parts = [random_bases(rng, int(L), gc) for L in lengths]
    offs = np.zeros(len(parts) + 1, dtype=np.int64)
    offs[1:] = np.cumsum([len(p) for p in parts])
    seq = np.concatenate(parts) if parts else np.zeros(0, dtype=np.uint8)
    if mask_frac > 0:
        for s in range(len(parts)):
            sub = seq[offs[s]:offs[s + 1]]
            add_masked_repeats(rng, sub, mask_frac, family_lengths=repeat_lengths)
    planted = plant_duplications(rng, seq, n_sd, sd_lo, sd_hi, id_lo, id_hi,
                                 offsets=offs, inter_frac=inter_frac, disjoint=True)
    if n_gaps:
        for s in range(len(parts)):
            sub = seq[offs[s]:offs[s + 1]]
            L = len(sub)
            if L > 400:
                add_n_gaps(rng, sub, max(L // 2, 200), 5, min(60, L // 8))
    return Genome(seq, offs, planted, f"small-{seed}")


def query_regions(genome: Genome, count: int, seed: int = 0x5EDEF005, len_lo: int = 10_000,
                  len_hi: int = 5_000_000, mut_lo: float = 0.0, mut_hi: float = 0.25) -> list:
    """Query regions for the serving workload: lengths log-uniform in
    [len_lo, len_hi] cut from the genome (within one sequence), mutated by a
    fraction U[mut_lo, mut_hi] of edit events, reverse-complemented half of
    the time.  Returns uint8 ASCII arrays."""
    rng = np.random.default_rng(seed)
    out = []
    seq_len = np.diff(genome.offsets)
    for _ in range(count):
        L = int(log_uniform_int(rng, len_lo, len_hi + 1))
        s = int(rng.choice(len(seq_len), p=seq_len / seq_len.sum()))
        L = min(L, int(seq_len[s]))
        a = int(genome.offsets[s] + rng.integers(0, seq_len[s] - L + 1))
        piece = mutate(rng, genome.seq[a:a + L], 1.0 - float(rng.uniform(mut_lo, mut_hi)))
        if rng.random() < 0.5:
            piece = reverse_complement(piece)
        out.append(np.ascontiguousarray(piece))
    return out
