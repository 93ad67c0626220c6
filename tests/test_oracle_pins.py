"""Pins for the CPU oracle: checks against what the paper and the mathematics
fix, independent of the oracle's own code paths.

- tau: the lower bound of Section 3.1 rebuilt from explicit sets that have
  the structure the derivation assumes (not by retyping the formula);
- hash: the 'random permutation' of Section 2.2 is a bijection on 4^k codes;
- pack and sketch: per-base definitions and winnowing (Section 2.2: minimal
  hash per window, rightmost on ties) by explicit string and window scans;
- winnowing invariant and density 2/(w+1) (Section 2.2);
- index: sorted unique (hash, position) pairs (Section 3.1) versus numpy;
- filter and refine: every window x every target start by explicit sets;
- chaining: longest chain by a different search on tiny anchor sets, and
  whole chain rows (anchor sets, axis flip, self-span rule, tie rule, m(s)
  drop) by exhaustive path enumeration;
- merge: connected components by networkx;
- planted duplications are recovered (the protocol of Section 4.1.1).
"""
import math

import numpy as np
import pytest

import oracle
from paper_1807_00205_gb300 import synth
from tests import bruteforce as bf

TINY = dict(k=5, w=4, n=40, step=3, max_occ=0, self_mode=1, gap_max=40,
            diag_max=4, min_unmasked=1, delta_m=0.15, delta_g=0.10)


def tiny_genome(seed, lengths=(260, 170), mask=0.15, gaps=True):
    return synth.small_case(seed, lengths=lengths, n_sd=3, sd_lo=50, sd_hi=110,
                            id_lo=0.9, id_hi=1.0, mask_frac=mask, n_gaps=gaps,
                            inter_frac=0.5, repeat_lengths=(15, 30))


# ---------------------------------------------------------------- tau ------

@pytest.mark.parametrize("k,dm,dg", [(12, 0.15, 0.10), (12, 0.15, 0.15), (11, 0.10, 0.05),
                                     (16, 0.05, 0.20)])
def test_tau_matches_set_construction(k, dm, dg):
    """Section 3.1 derivation rebuilt from explicit sets: t_M copied k-mers of
    which c = t_M e^{-k dM} survive in both copies, plus gap k-mers that the
    two sides do not share.  With t_G = t_M dG/(1-dG) gap k-mers per side (the
    premise) the exact Jaccard is at least tau; with t_G = dG/(1-dG) times
    |X^M_i u X^M_j| every step of the derivation is tight and the exact
    Jaccard equals tau up to the rounding of the set sizes."""
    t_m = 200_000
    c = round(t_m * math.exp(-k * dm))

    def jaccard_with_gaps(t_g):
        X = set(range(t_m)) | set(range(10**7, 10**7 + t_g))
        Y = set(range(c)) | set(range(2 * 10**7, 2 * 10**7 + t_m - c)) | \
            set(range(3 * 10**7, 3 * 10**7 + t_g))
        return len(X & Y) / len(X | Y)

    tau = oracle.tau(k, dm, dg)
    assert jaccard_with_gaps(round(t_m * dg / (1 - dg))) >= tau
    assert tau == pytest.approx(jaccard_with_gaps(round((2 * t_m - c) * dg / (1 - dg))), rel=2e-4)


def test_tau_default_value():
    # the defaults of Sections 2.1 and 3.3 (k = 12, dM = 0.15, dG = 0.10)
    assert oracle.tau() == pytest.approx(0.07371, abs=5e-6)


def test_mtable_is_least_integer():
    tau = oracle.tau()
    m = oracle.mtable(smax=739)
    s = np.arange(740)
    assert np.all(m >= tau * s - 1e-9)
    assert np.all((m - 1) < tau * s - 1e-9) or m[0] == 0
    assert m[0] == 0 and m[1] == 1 and np.all(np.diff(m) >= 0)


# ---------------------------------------------------------------- hash -----

@pytest.mark.parametrize("k", [2, 3, 5, 8, 11, 12])
def test_hash_is_permutation(k):
    h = oracle.hash_all(k)
    assert h.max() < (1 << (2 * k))
    assert len(np.unique(h)) == (1 << (2 * k))


# ---------------------------------------------------------------- pack -----

def test_pack_every_byte():
    rng = np.random.default_rng(7)
    seq = np.concatenate([np.arange(256, dtype=np.uint8),
                          rng.integers(0, 256, 1000).astype(np.uint8),
                          np.frombuffer(b"ACGTacgtNnRY-", dtype=np.uint8)])
    packed, mask, nbits = oracle.pack(seq)
    table = {ord(c): v for c, v in zip("ACGTacgt", [0, 1, 2, 3, 0, 1, 2, 3])}
    for p, b in enumerate(seq.tolist()):
        code = (int(packed[p // 16]) >> (2 * (p % 16))) & 3
        assert code == table.get(b, 0)
        assert ((int(mask[p // 32]) >> (p % 32)) & 1) == int(chr(b).islower() and chr(b).isalpha()
                                                           and b < 128)
        assert ((int(nbits[p // 32]) >> (p % 32)) & 1) == int(b not in table)


def test_pack_empty_and_ragged():
    for n in [0, 1, 15, 16, 17, 31, 32, 33]:
        seq = np.frombuffer(b"acgtN" * 10, dtype=np.uint8)[:n]
        packed, mask, nbits = oracle.pack(seq)
        assert len(packed) == (n + 15) // 16 and len(mask) == (n + 31) // 32


# --------------------------------------------------------------- sketch ----

def _sketch_cases():
    yield tiny_genome(1), dict(TINY)
    yield tiny_genome(2, lengths=(5, 9, 300)), dict(TINY, w=6)
    # tandem repeats (equal hashes inside one window -> rightmost tie) and a
    # palindromic 12-mer run
    rep = (b"ACGTTA" * 30) + (b"ACGTACGTACGT" * 6) + b"GATTACA" * 20 + (b"cagtc" * 12)
    offs = np.array([0, len(rep)], dtype=np.int64)
    yield synth.Genome(np.frombuffer(rep, dtype=np.uint8).copy(), offs, []), dict(TINY, k=12, w=16)
    yield tiny_genome(3, mask=0.5), dict(TINY, k=4, w=1)
    yield tiny_genome(4, mask=0.4), dict(TINY, k=6, w=5, min_unmasked=3)


@pytest.mark.parametrize("case", list(range(5)))
def test_sketch_matches_window_scan(case):
    g, p = list(_sketch_cases())[case]
    rows = oracle.sketch(g.seq, g.offsets, p)
    want = bf.sketch(g.seq.tobytes(), g.offsets, p["k"], p["w"],
                     lambda c: oracle.hash_code(c, p["k"]), p["min_unmasked"])
    assert set(map(tuple, rows.tolist())) == want
    assert np.all(np.diff(rows[:, 1]) > 0)  # sorted, unique positions


def test_winnow_invariant_and_density():
    rng = np.random.default_rng(11)
    L = 1_000_000
    seq = synth.random_bases(rng, L)
    offs = np.array([0, L], dtype=np.int64)
    p = oracle.params()
    rows = oracle.sketch(seq, offs, p)
    pos = rows[:, 1]
    # every full window of w k-mer starts holds a selected start (all k-mers
    # of an ACGT-only random sequence are eligible except palindromes)
    sel = np.zeros(L, dtype=np.int64)
    sel[pos] = 1
    cs = np.concatenate([[0], np.cumsum(sel)])
    nk = L - p["k"] + 1
    q = np.arange(nk - p["w"] + 1)
    assert np.all(cs[q + p["w"]] - cs[q] >= 1)
    # expected density 2/(w+1) for a random sequence (Section 2.2)
    dens = len(pos) / nk
    assert abs(dens - 2 / (p["w"] + 1)) < 0.003


# ---------------------------------------------------------------- index ----

def test_index_sorted_with_offsets():
    g = tiny_genome(5, lengths=(3000, 2000))
    p = dict(TINY, k=6, w=5)
    recs = oracle.sketch(g.seq, g.offsets, p)
    rows, off = oracle.index(recs, p["k"])
    order = np.lexsort((recs[:, 1], recs[:, 0]))
    assert np.array_equal(rows, recs[order])
    want = np.searchsorted(recs[order, 0], np.arange((1 << 12) + 1), side="left")
    assert np.array_equal(off.astype(np.int64), want)


# --------------------------------------------------------------- filter ----

FILTER_CASES = [
    (11, dict(TINY)),
    (12, dict(TINY, step=1, n=30)),
    (13, dict(TINY, self_mode=0)),
    (14, dict(TINY, max_occ=4)),
    (15, dict(TINY, k=4, w=3, n=25, step=5)),
    (16, dict(TINY, self_mode=2)),
]


@pytest.mark.parametrize("seed,p", FILTER_CASES)
def test_filter_and_refine_match_all_pairs(seed, p):
    g = tiny_genome(seed)
    recs = oracle.sketch(g.seq, g.offsets, p)
    tau = oracle.tau(p["k"], p["delta_m"], p["delta_g"])
    runs = oracle.filter_runs(recs, g.offsets, recs, g.offsets, p)
    rl = [tuple(map(int, r)) for r in bf.filter_runs([tuple(r) for r in recs.tolist()], g.offsets,
                                                    [tuple(r) for r in recs.tolist()], g.offsets,
                                                    p, tau)]
    assert len(rl) > 0
    assert [tuple(r[:8]) for r in runs.tolist()] == rl
    # refine: the estimate at every j of each run, by explicit sets
    trecs = [tuple(r) for r in recs.tolist()]
    for r in runs.tolist():
        i, o, ja, jb = r[0], r[1], r[2], r[3]
        wq = {}
        for h, pos, sg in trecs:
            if i <= pos <= i + p["n"] - p["k"]:
                wq.setdefault(h, set()).add(sg)
        if p["max_occ"] > 0:
            cnt = {}
            for h, _, _ in trecs:
                cnt[h] = cnt.get(h, 0) + 1
            wq = {h: v for h, v in wq.items() if cnt[h] <= p["max_occ"]}
        best, jstar, den = -1, None, None
        for j in range(ja, jb + 1):
            e, d = bf.estimate(wq, trecs, i, j, p, o)
            if e > best:
                best, jstar, den = e, j, d
        assert (r[8], r[9], r[10]) == (best, jstar, den)
        assert r[11] == int(best >= bf.m_of(tau, den))


def test_refine_breakpoints_equal_dense():
    g = tiny_genome(21, lengths=(600, 400))
    p = dict(TINY)
    recs = oracle.sketch(g.seq, g.offsets, p)
    a = oracle.filter_runs(recs, g.offsets, recs, g.offsets, p)
    b = oracle.filter_runs(recs, g.offsets, recs, g.offsets, p, dense=True)
    assert len(a) > 0 and np.array_equal(a, b)


def test_filter_window_subset_matches_full():
    g = tiny_genome(22, lengths=(600, 400))
    p = dict(TINY)
    recs = oracle.sketch(g.seq, g.offsets, p)
    full = oracle.filter_runs(recs, g.offsets, recs, g.offsets, p)
    wins = np.unique(full[:, 0])[::2]
    sub = oracle.filter_runs(recs, g.offsets, recs, g.offsets, p, windows=wins)
    assert np.array_equal(sub, full[np.isin(full[:, 0], wins)])


# ---------------------------------------------------------------- chain ----

@pytest.mark.parametrize("seed", range(30))
def test_chain_dp_is_longest(seed):
    """chain_anchors runs chain_dp, the same DP orc_chain runs per kept seed."""
    rng = np.random.default_rng(seed)
    A = int(rng.integers(1, 12))
    base = np.sort(rng.integers(0, 200, A))
    anc = np.stack([base, base + rng.integers(-6, 7, A) + (seed % 3) * 5], axis=1)
    if seed % 4 == 0:
        anc = rng.integers(0, 60, (A, 2))
    gap_max, diag_max = 60, 5
    rows = oracle.chain_anchors(anc, gap_max, diag_max)
    best, srt = bf.best_chain_length([tuple(a) for a in anc.tolist()], gap_max, diag_max)
    # duplicates of the same anchor cannot chain with each other
    assert rows[:, 2].max() == best
    # backtrack the oracle's chosen chain and check it is a valid chain
    end = int(np.argmax(rows[:, 2]))
    chain = []
    while end >= 0:
        chain.append((int(rows[end, 0]), int(rows[end, 1])))
        end = int(rows[end, 3])
    chain.reverse()
    assert len(chain) == best and bf.chain_is_valid(chain, gap_max, diag_max)


def tandem_genome(seed, period=33, copies=5, flank=120, mut=0.05):
    """A near-exact tandem repeat (period 33 < n), its partial reverse
    complement and random flanks: in self mode the target span of a tandem
    mate overlaps the query window's own span, and nearby copies give ties."""
    rng = np.random.default_rng(seed)
    unit = synth.random_bases(rng, period)
    rep = np.concatenate([unit] * copies)
    sub = rng.random(len(rep)) < mut
    rep[sub] = synth._ACGT[rng.integers(0, 4, int(sub.sum()))]
    seq = np.concatenate([synth.random_bases(rng, flank), rep, synth.random_bases(rng, flank),
                          synth.reverse_complement(rep)[:80], synth.random_bases(rng, 60)])
    return synth.Genome(np.ascontiguousarray(seq), np.array([0, len(seq)], dtype=np.int64), [])


def end_dup_genome(seed):
    """Two sequences, each ending with the second copy of a duplication
    (reverse-complemented on odd seeds), so that runs end where the target
    sequence ends and the last target k-mer can be an anchor."""
    rng = np.random.default_rng(seed)
    x = synth.random_bases(rng, 100)
    y = synth.reverse_complement(x) if seed % 2 else x.copy()
    s1 = np.concatenate([synth.random_bases(rng, int(rng.integers(20, 60))), x,
                         synth.random_bases(rng, int(rng.integers(40, 70))), y])
    z = synth.random_bases(rng, 150)
    s2 = np.concatenate([z, synth.random_bases(rng, int(rng.integers(30, 60))),
                         z[:int(rng.integers(90, 150))]])
    seq = np.concatenate([s1, s2])
    return synth.Genome(np.ascontiguousarray(seq), np.array([0, len(s1), len(seq)], dtype=np.int64),
                        [])


CHAIN_CASES = [
    ("tiny", 51, dict(TINY)),
    ("tiny", 52, dict(TINY, self_mode=0)),
    ("tiny", 54, dict(TINY, self_mode=2)),
    ("tiny", 55, dict(TINY, k=4, w=3, n=25, step=5, gap_max=25, diag_max=3)),
    ("tiny", 56, dict(TINY, max_occ=4)),
    ("tiny", 64, dict(TINY, diag_max=40, gap_max=40)),
    ("tandem", 60, dict(TINY, diag_max=12, gap_max=30)),
    ("tandem", 61, dict(TINY, diag_max=40, gap_max=40)),
    ("end_dup", 81, dict(TINY, step=1)),
    ("end_dup", 89, dict(TINY, step=1)),
]
CHAIN_SLIPS = ["pred_tie", "end_tie", "span_short", "no_self", "no_flip", "keep_all"]


def _chain_case(kind, seed, p):
    g = {"tiny": tiny_genome, "tandem": tandem_genome, "end_dup": end_dup_genome}[kind](seed)
    recs = oracle.sketch(g.seq, g.offsets, p)
    runs = oracle.filter_runs(recs, g.offsets, recs, g.offsets, p)
    got = [tuple(map(int, r)) for r in oracle.chain(runs, recs, g.offsets, recs, g.offsets, p).tolist()]
    R = [tuple(r) for r in recs.tolist()]
    tau = oracle.tau(p["k"], p["delta_m"], p["delta_g"])
    return got, lambda slip=None: bf.chain_rows(runs.tolist(), R, g.offsets, R, g.offsets, p,
                                                tau, slip)


@pytest.mark.parametrize("kind,seed,p", CHAIN_CASES)
def test_chain_rows_match_bruteforce(kind, seed, p):
    """orc_chain as the self-search calls it, against Section 3.3 restated by
    exhaustive path enumeration: anchor sets rebuilt from the raw records
    (target span [j_a, j_b+n-k], self-span exclusion, o = 1 axis flip), every
    maximal chain enumerated, the tie rule applied to the longest ones
    (chain end: the earliest anchor; then the later predecessor at every
    step), and chains below m(s) dropped.  Whole rows must match."""
    got, want = _chain_case(kind, seed, p)
    assert len(got) > 0
    assert got == want()


def test_chain_pin_detects_each_slip():
    """Every plausible slip (predecessor or end tie reversed, target span one
    short, self-span rule dropped, no o = 1 axis flip, no m(s) drop) changes
    at least one row of the cases above, so the pin would catch it."""
    cases = [_chain_case(*c) for c in CHAIN_CASES]
    for slip in CHAIN_SLIPS:
        assert any(got != want(slip) for got, want in cases), slip


def test_chain_rows_are_colinear_boxes():
    g = synth.small_case(31, lengths=(60_000,), n_sd=4, sd_lo=2000, sd_hi=5000, id_lo=0.9)
    p = oracle.params()
    r = oracle.selfsearch(g.seq, g.offsets, p)
    ch = r["chains"]
    assert len(ch) > 0
    assert np.all(ch[:, 4] > ch[:, 3]) and np.all(ch[:, 7] > ch[:, 6])
    m = oracle.mtable()
    assert np.all(ch[:, 8] >= m[ch[:, 9]])
    # in self mode the target box starts after the query window start
    assert np.all(ch[:, 6] > ch[:, 0])


# ---------------------------------------------------------------- merge ----

def test_merge_is_connected_components():
    nx = pytest.importorskip("networkx")
    rng = np.random.default_rng(3)
    p = oracle.params()
    rows = []
    for c in range(120):
        o = int(rng.integers(0, 2))
        q0 = int(rng.integers(0, 5000))
        ln = int(rng.integers(100, 700))
        t0 = q0 + int(rng.integers(3000, 3400))
        rows.append([q0, o, 0, q0, q0 + ln, 0, t0, t0 + ln + int(rng.integers(-50, 50)),
                     int(rng.integers(5, 40)), 80])
    ch = np.array(rows, dtype=np.int64)
    got = oracle.merge(ch, p)
    G = nx.Graph()
    G.add_nodes_from(range(len(ch)))

    def diag(c):
        return c[6] - c[3] if c[1] == 0 else c[7] + c[3]

    for a in range(len(ch)):
        for b in range(len(ch)):
            A, B = ch[a], ch[b]
            if a == b or A[1] != B[1]:
                continue
            if max(A[3], B[3]) <= min(A[4], B[4]) and max(A[6], B[6]) <= min(A[7], B[7]):
                ln = max(A[4] - A[3], B[4] - B[3])
                if abs(diag(A) - diag(B)) <= p["diag_max"] + math.ceil(p["delta_g"] * ln):
                    G.add_edge(a, b)
    want = []
    for comp in nx.connected_components(G):
        C = ch[list(comp)]
        want.append((0, C[:, 3].min(), C[:, 4].max(), 0, C[:, 6].min(), C[:, 7].max(),
                     C[0, 1], C[:, 8].sum(), len(C)))
    want.sort(key=lambda x: (x[1], x[4], x[6], x[2], x[5]))
    assert [tuple(r) for r in got.tolist()] == [tuple(map(int, w)) for w in want]


# -------------------------------------------------------------- recall -----

def test_planted_duplications_recovered():
    """Section 4.1.1 protocol on synthetic data: a duplication counts as found
    when candidates cover more than 95% of the bases of both mates.  Copies
    here diverge by at most 10% through substitutions and small indels.  The
    path ends at chaining (no extension step), so a mate's ends can be missed
    by up to one query step; the bar is: most pairs found, every pair at
    least 90% covered."""
    g = synth.small_case(41, lengths=(400_000,), n_sd=8, sd_lo=2000, sd_hi=8000,
                         id_lo=0.90, id_hi=0.995)
    p = oracle.params()
    r = oracle.selfsearch(g.seq, g.offsets, p)
    cands = r["cands"]
    assert len(g.planted) >= 6
    found = 0
    for sd in g.planted:
        a, b = (sd.src, sd.src + sd.length), (sd.dst, sd.dst + sd.copy_length)
        first, second = (a, b) if a[0] < b[0] else (b, a)
        o = 1 if sd.reverse else 0
        qcov = np.zeros(first[1] - first[0], dtype=bool)
        tcov = np.zeros(second[1] - second[0], dtype=bool)
        for c in cands.tolist():
            if c[6] != o:
                continue
            if c[2] <= first[0] or c[1] >= first[1] or c[5] <= second[0] or c[4] >= second[1]:
                continue
            qcov[max(c[1], first[0]) - first[0]:min(c[2], first[1]) - first[0]] = True
            tcov[max(c[4], second[0]) - second[0]:min(c[5], second[1]) - second[0]] = True
        assert qcov.mean() > 0.90 and tcov.mean() > 0.90, (sd, qcov.mean(), tcov.mean())
        found += int(qcov.mean() > 0.95 and tcov.mean() > 0.95)
    assert found >= 0.75 * len(g.planted)


def test_exact_jaccard_closed_form():
    """Section 3.1: with no repeated k-mer, J = c / (2t - c), t = n - k + 1."""
    rng = np.random.default_rng(5)
    n, k = 300, 12
    a = synth.random_bases(rng, n)
    b = a.copy()
    b[::37] = synth.random_bases(rng, len(b[::37]))
    seq = np.concatenate([a, b])
    J = oracle.jaccard(seq, 0, n, n, k)
    A = {a[x:x + k].tobytes() for x in range(n - k + 1)}
    B = {b[x:x + k].tobytes() for x in range(n - k + 1)}
    t = n - k + 1
    assert len(A) == t and len(B) == t
    c = len(A & B)
    assert J == pytest.approx(c / (2 * t - c), abs=1e-12)


# --------------------------------------------------------------- golden ----

def test_paper_constants_are_the_defaults():
    import json
    import os
    with open(os.path.join(os.path.dirname(__file__), "golden", "paper_constants.json")) as f:
        c = json.load(f)
    p = oracle.params()
    assert p["k"] == c["k_seeding"]["value"]
    assert p["delta_m"] == c["delta_m"]["value"]
    assert p["delta_m"] + p["delta_g"] == pytest.approx(c["delta"]["value"])
    assert p["n"] == c["seed_length_n"]["value"] == round(
        c["min_sd_length"]["value"] * (1 - c["delta"]["value"]))


def test_oracle_matches_stored_digests():
    import json
    import os
    from tests.golden import make_golden
    with open(os.path.join(os.path.dirname(__file__), "golden", "oracle_small.json")) as f:
        want = json.load(f)
    assert make_golden.compute() == want


def test_sketch_threads_do_not_change_rows():
    """Sequences are sketched independently, so sharing them out to threads
    gives the same rows in the same order."""
    g = synth.small_case(41, lengths=(30_000, 5, 2000, 60_000, 900), mask_frac=0.3, n_gaps=True)
    pd = oracle.params()
    one = oracle.sketch(g.seq, g.offsets, pd)
    for t in (2, 3, 8):
        assert np.array_equal(oracle.sketch(g.seq, g.offsets, pd, threads=t), one)


def test_filter_window_subset_equals_full_rows():
    """Filtering a subset of windows gives exactly those windows' rows of the
    full run (postings are built only for the hashes the subset holds)."""
    g = synth.small_case(42, lengths=(40_000, 25_000), n_sd=4, mask_frac=0.1)
    pd = oracle.params()
    recs = oracle.sketch(g.seq, g.offsets, pd)
    full = oracle.filter_runs(recs, g.offsets, recs, g.offsets, pd)
    win = np.unique(full[:, 0])[::3]
    sub = oracle.filter_runs(recs, g.offsets, recs, g.offsets, pd, windows=win)
    assert len(sub) > 0
    assert np.array_equal(sub, full[np.isin(full[:, 0], win)])


def test_filter_threads_do_not_change_rows():
    """Windows are filtered independently: any number of threads gives the
    same rows in the same order."""
    g = synth.small_case(43, lengths=(50_000, 20_000), n_sd=5, mask_frac=0.15)
    pd = oracle.params()
    recs = oracle.sketch(g.seq, g.offsets, pd)
    one = oracle.filter_runs(recs, g.offsets, recs, g.offsets, pd)
    assert len(one) > 0
    for t in (2, 5, 16):
        assert np.array_equal(oracle.filter_runs(recs, g.offsets, recs, g.offsets, pd, threads=t), one)


# ---------------------------------------------------------- f3 q-gram filter --

def test_qgram_bound_reduces_to_the_q_gram_lemma():
    """Section 3.2's bound with no gaps (delta_G = 0, p_G = 0) is the classic
    q-gram lemma: strings of length n at e substitutions share at least
    n - q + 1 - q e q-grams (Jokinen and Ukkonen); with the defaults it gives
    211 (q = 4) and 94 (q = 5) at n = 750 after rounding up."""
    for n, q, e in [(750, 4, 10), (1000, 3, 0), (100, 5, 7), (750, 1, 112)]:
        assert abs(oracle.qgram_bound(n, q, 0.0, e / n, 0.0) - (n - q + 1 - q * e)) < 1e-9
    assert math.ceil(oracle.qgram_bound(750, 4) - 1e-9) == 211
    assert math.ceil(oracle.qgram_bound(750, 5) - 1e-9) == 94
    # q = 1 has no overlap term: n (1 - delta_G - delta_M)
    assert abs(oracle.qgram_bound(750, 1) - 750 * 0.75) < 1e-9


def test_qgram_shared_special_cases():
    rng = np.random.default_rng(3)
    x = synth.random_bases(rng, 300)
    s = np.concatenate([x, x, synth.reverse_complement(x)])
    n = 300
    for q in (1, 2, 4, 5):
        assert oracle.qgram_shared(s, 0, 300, n, 0, q) == n - q + 1      # identical
        assert oracle.qgram_shared(s, 0, 600, n, 1, q) == n - q + 1      # reverse complement
    lower = np.frombuffer(bytes(x).lower(), dtype=np.uint8)
    s2 = np.concatenate([x, lower])
    assert oracle.qgram_shared(s2, 0, 300, n, 0, 4) == n - 4 + 1  # case is ignored
    # one N removes the q q-grams over it
    y = x.copy()
    y[150] = ord("N")
    s3 = np.concatenate([x, y])
    assert oracle.qgram_shared(s3, 0, 300, n, 0, 4) == n - 4 + 1 - 4
    # disjoint and multiplicity examples worked by hand
    s4 = np.frombuffer(b"AAAAAAAACCCCCCCC", dtype=np.uint8)
    assert oracle.qgram_shared(s4, 0, 8, 8, 0, 3) == 0
    s5 = np.frombuffer(b"ACGTACGTACACACGG", dtype=np.uint8)
    # q = 2: X has AC x2, CG x2, GT x2, TA x1; Y has AC x3, CA x2, CG x1, GG x1
    assert oracle.qgram_shared(s5, 0, 8, 8, 0, 2) == 2 + 1


def test_qgram_lemma_holds_under_the_error_model():
    """Pairs within the SD error model never fall below the bound: Y is X
    with e substitutions and g gaps (total gap length <= delta_G n), cut to
    n bases; Q(X, Y) >= n (1 - delta_G - q e/n) - (g + 1)(q - 1)."""
    rng = np.random.default_rng(11)
    n = 750
    for trial in range(60):
        x = synth.random_bases(rng, n + 200)
        y = x.copy()
        e = int(rng.integers(0, 113))
        pos = rng.choice(n, size=e, replace=False)
        y[pos] = synth._ACGT[(np.searchsorted(synth._ACGT, y[pos]) + rng.integers(1, 4, e)) % 4]
        g = int(rng.integers(0, 6))
        budget = int(0.10 * n)
        for _ in range(g):
            ln = int(rng.integers(1, max(2, budget // max(g, 1)) + 1))
            at = int(rng.integers(10, n - 10))
            if rng.random() < 0.5:
                y = np.delete(y, np.arange(at, at + ln))
            else:
                y = np.insert(y, at, synth._ACGT[rng.integers(0, 4, ln)])
        s = np.concatenate([x[:n], y[:n]])
        for q in (3, 4, 5):
            got = oracle.qgram_shared(s, 0, n, n, 0, q)
            assert got >= n * (1 - 0.10 - q * e / n) - (g + 1) * (q - 1) - 1e-9, (trial, q, got)


def test_qgram_rows_follow_the_threshold():
    g = synth.small_case(44, lengths=(60_000,), n_sd=4, sd_lo=2000, sd_hi=6000, id_lo=0.8)
    pd = oracle.params()
    recs = oracle.sketch(g.seq, g.offsets, pd)
    runs = oracle.filter_runs(recs, g.offsets, recs, g.offsets, pd)
    rows = oracle.qgram(g.seq, runs, pd, q=4)
    need = math.ceil(oracle.qgram_bound(750, 4) - 1e-9)
    keep = runs[:, oracle.RUN_COLS.index("keep")] == 1
    assert keep.sum() > 0 and len(rows) == len(runs)
    assert (rows[~keep] == 0).all()
    assert np.array_equal(rows[keep, 1], (rows[keep, 0] >= need).astype(np.int64))
    for r in np.nonzero(keep)[0][:10]:
        i, o, js = runs[r, 0], runs[r, 1], runs[r, oracle.RUN_COLS.index("j_star")]
        assert rows[r, 0] == oracle.qgram_shared(g.seq, i, js, 750, o, 4)


# ------------------------------------------------------- f1 SD extension ----

EXTEND_CASES = [
    ("tiny", 51, dict(TINY), 400),
    ("tiny", 52, dict(TINY, self_mode=0), 400),
    ("tiny", 54, dict(TINY, self_mode=2), 400),
    ("tiny", 57, dict(TINY), 120),                 # the length cap binds
    ("tiny", 58, dict(TINY, min_unmasked=2), 400),
    ("tandem", 60, dict(TINY), 400),               # overlapping mates
    ("end_dup", 81, dict(TINY, step=1), 400),      # regions reach sequence ends
    ("end_dup", 89, dict(TINY, step=1), 400),
]


def _extend_case(kind, seed, p, max_len):
    g = {"tiny": tiny_genome, "tandem": tandem_genome, "end_dup": end_dup_genome}[kind](seed)
    recs = oracle.sketch(g.seq, g.offsets, p)
    runs = oracle.filter_runs(recs, g.offsets, recs, g.offsets, p)
    allk = oracle.sketch(g.seq, g.offsets, dict(p, min_unmasked=0))  # Section 3.2: any k-mer
    got = [tuple(map(int, r)) for r in
           oracle.extend(runs, allk, g.offsets, allk, g.offsets, p, max_len=max_len).tolist()]
    R = [tuple(r) for r in allk.tolist()]
    tau = oracle.tau(p["k"], p["delta_m"], p["delta_g"])
    return g, got, lambda slip=None: bf.extend_rows(runs.tolist(), R, g.offsets, R, g.offsets,
                                                    p, tau, max_len, slip)


@pytest.mark.parametrize("kind,seed,p,max_len", EXTEND_CASES)
def test_extend_matches_bruteforce(kind, seed, p, max_len):
    """Section 3.2 restated step by step: the grown regions' estimate is
    recomputed from explicit sets after every one-base step on each side;
    the oracle's incremental growth must stop at the same regions."""
    g, got, want = _extend_case(kind, seed, p, max_len)
    assert len(got) > 0 and any(r[4] - r[3] > p["n"] for r in got)
    assert got == want()


def test_extend_mirror_is_pinned():
    """For o = 1 the target grows at the opposite end; growing it like o = 0
    changes rows of the cases above."""
    cases = [_extend_case(*c) for c in EXTEND_CASES]
    assert any(got != want("no_mirror") for _, got, want in cases)


def test_extend_limits_hold():
    """Regions grow in lockstep (equal lengths), stay inside their sequences,
    never exceed max_len, never overlap more than their seed did, and every
    grown region still passes the threshold."""
    tau = oracle.tau()
    for kind, seed, p, max_len in EXTEND_CASES:
        g, got, _ = _extend_case(kind, seed, p, max_len)
        m = oracle.mtable(p["k"], p["delta_m"], p["delta_g"], smax=4096)
        for i, o, js, qa, qb, ta, tb, est, den in got:
            assert qb - qa == tb - ta <= max(max_len, p["n"])
            qs = np.searchsorted(g.offsets, i, side="right") - 1
            ts = np.searchsorted(g.offsets, js, side="right") - 1
            assert g.offsets[qs] <= qa <= i and i + p["n"] <= qb <= g.offsets[qs + 1]
            assert g.offsets[ts] <= ta and tb <= g.offsets[ts + 1]
            if p["self_mode"] and qs == ts:
                ov = max(0, min(qb, tb) - max(qa, ta))
                assert ov <= max(0, min(i + p["n"], js + p["n"]) - max(i, js))
            if qb - qa > p["n"]:
                assert est >= m[den] and est >= tau * den - 1e-9


def test_extension_contains_planted_duplications():
    """The purpose of Section 3.2: seeds (750 bp) grown until the estimate
    drops find the boundaries of the duplications.  For every planted pair
    (2-8 kbp, 90-99.5% identity) one potential SD region holds both whole
    mates, which no single seed window can."""
    g = synth.small_case(41, lengths=(400_000,), n_sd=8, sd_lo=2000, sd_hi=8000,
                         id_lo=0.90, id_hi=0.995)
    p = oracle.params()
    r = oracle.selfsearch(g.seq, g.offsets, p, threads=8)
    allk = oracle.sketch(g.seq, g.offsets, oracle.params(min_unmasked=0))
    ext = oracle.extend(r["runs"], allk, g.offsets, allk, g.offsets, p, threads=8)
    assert len(g.planted) >= 6
    for sd in g.planted:
        a, b = (sd.src, sd.src + sd.length), (sd.dst, sd.dst + sd.copy_length)
        first, second = (a, b) if a[0] < b[0] else (b, a)
        o = 1 if sd.reverse else 0
        assert any(row[1] == o and row[3] <= first[0] and row[4] >= first[1]
                   and row[5] <= second[0] and row[6] >= second[1] for row in ext.tolist()), sd


# ------------------------------------------ f2 two-tier chaining (3.3) ----

@pytest.mark.parametrize("seed", range(6))
def test_seeds_are_maximal_exact_matches(seed):
    """The seeds of Section 3.3 (exact matches of at least k2 bases), found
    through a k-mer table, equal a scan of every diagonal."""
    rng = np.random.default_rng(seed)
    alpha = np.frombuffer(b"ACGTACGTACGTN", dtype=np.uint8)
    X = alpha[rng.integers(0, len(alpha), 150)]
    Y = alpha[rng.integers(0, len(alpha), 120)]
    core = synth.random_bases(rng, 40)
    X[20:60] = core
    Y[50:90] = core                  # a shared stretch (with a mismatch below)
    Y[70] = ord("A") if Y[70] != ord("A") else ord("C")
    X[100:130] = X[10:40]            # a repeat inside X
    k2 = 5 + seed % 3 * 3
    got = [tuple(r) for r in oracle.mems(X.tobytes(), Y.tobytes(), k2).tolist()]
    want = bf.mems(X.tobytes().decode(), Y.tobytes().decode(), k2)
    assert got == want and len(got) > 0


@pytest.mark.parametrize("seed", range(25))
def test_chain_tiers_match_chain_enumeration(seed):
    """Both chaining tiers (seeds into initial chains, initial chains into
    final chains with the affine penalty) against the same rules with every
    best score found by enumerating all chains."""
    rng = np.random.default_rng(100 + seed)
    n = int(rng.integers(2, 10))
    base = np.sort(rng.integers(0, 400, n))
    seeds = np.stack([base, base + rng.integers(-30, 31, n) + 50, rng.integers(11, 40, n)], axis=1)
    if seed % 5 == 0:  # seeds that overlap on one axis (indels)
        seeds[1:, 1] = seeds[:-1, 1] + seeds[:-1, 2] - rng.integers(0, 5, n - 1)
    g1, g2, go, gd = 25, 150, 6, 10
    got = [tuple(r) for r in oracle.chain_tiers(seeds, g1, g2, go, gd).tolist()]
    want = bf.chain_tiers([tuple(s) for s in seeds.tolist()], g1, g2, go, gd)
    assert got == want


def test_chain2_finds_the_planted_duplications():
    """Section 3.3's purpose: inside the potential SD regions the final
    chains recover each planted duplication (2-8 kbp, 90-99.5% identity,
    small indels) as one chain whose ends lie within 50 bp of the mates'."""
    g = synth.small_case(41, lengths=(400_000,), n_sd=8, sd_lo=2000, sd_hi=8000,
                         id_lo=0.90, id_hi=0.995)
    p = oracle.params()
    r = oracle.selfsearch(g.seq, g.offsets, p, threads=8)
    allk = oracle.sketch(g.seq, g.offsets, oracle.params(min_unmasked=0))
    ext = oracle.extend(r["runs"], allk, g.offsets, allk, g.offsets, p, threads=8)
    fin = oracle.chain2(g.seq, ext, threads=8)
    assert len(g.planted) >= 6
    for sd in g.planted:
        a, b = (sd.src, sd.src + sd.length), (sd.dst, sd.dst + sd.copy_length)
        first, second = (a, b) if a[0] < b[0] else (b, a)
        o = 1 if sd.reverse else 0
        assert any(row[1] == o and abs(row[2] - first[0]) <= 50 and abs(row[3] - first[1]) <= 50
                   and abs(row[4] - second[0]) <= 50 and abs(row[5] - second[1]) <= 50
                   for row in fin.tolist()), sd


def test_chain2_exact_copy_is_one_chain():
    """An exact copy inside its regions is one final chain covering the copy
    (one seed, score = its length, a few chance bases at most beyond)."""
    rng = np.random.default_rng(9)
    L = 3000
    core = synth.random_bases(rng, L)
    seq = np.concatenate([synth.random_bases(rng, 700), core, synth.random_bases(rng, 900),
                          synth.reverse_complement(core), synth.random_bases(rng, 500)])
    s0, s1 = 700 + L + 900, 700 + L + 900 + L
    for o, (ta, tb) in ((1, (s0 - 300, s1 + 200)),):
        regions = np.array([[700, o, s0, 500, 700 + L + 400, ta, tb, 0, 0]], dtype=np.int64)
        fin = oracle.chain2(seq, regions)
        assert len(fin) == 1
        _, oo, q0, q1, t0, t1, score, seeds, parts = fin[0].tolist()
        assert oo == 1 and parts == 1 and seeds == 1
        assert 690 <= q0 <= 700 and 700 + L <= q1 <= 700 + L + 10
        assert s0 - 10 <= t0 <= s0 and s1 <= t1 <= s1 + 10
        assert score == q1 - q0 == t1 - t0 >= L
