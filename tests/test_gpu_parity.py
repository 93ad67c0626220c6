"""GPU path versus the CPU oracle, element by element, through the C ABI.

All outputs are integers, so the bar is bit-exactness at every stage: packed
words, minimizer records, the sorted index and its offsets, runs with their
refined seeds, chains and SD candidates.  Cases cover several tiles with
ragged tails, multiple and tiny sequences, soft-masking, N runs, palindromic
and tandem k-mers, non-default (k, w, n, step), the occurrence cap, non-self
search, and windows that overflow the fast path's shared-memory budget (so the
global-memory path runs too).
"""
import numpy as np
import pytest

import oracle
from paper_1807_00205_gb300 import binding, synth
from tests.gpu_helpers import (assert_rows_equal, cand_rows_global, chain_rows, need_gpu,
                               rec_rows, run_rows)

pytestmark = pytest.mark.gpu

TINY = dict(k=5, w=4, n=40, step=3, max_occ=0, self_mode=1, gap_max=40,
            diag_max=4, min_unmasked=1, delta_m=0.15, delta_g=0.10)


@pytest.fixture(scope="module")
def ctx():
    need_gpu()
    c = binding.Context(0)
    yield c
    c.close()


def to_dev(a):
    torch = need_gpu()
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda:0")


def full_parity(ctx, g, pd, check_chain=True):
    """Every stage through the C ABI against the oracle.  check_chain=False
    stops after the filter (for degenerate inputs whose seeds have too many
    anchors for the quadratic chain DP)."""
    recs = oracle.sketch(g.seq, g.offsets, pd)
    idx_rows, idx_off = oracle.index(recs, pd["k"])
    runs = oracle.filter_runs(recs, g.offsets, recs, g.offsets, pd)
    ref = dict(recs=recs, index=idx_rows, offsets=idx_off, runs=runs)
    p = binding.params_from_dict(pd)
    d = to_dev(g.seq)
    packed, mask, nbits = ctx.sedef_pack(d)
    rec = ctx.sedef_sketch(packed, mask, nbits, g.offsets, p)
    srt, off = ctx.sedef_index(rec, p)
    druns, nr = ctx.sedef_filter(rec, g.offsets, rec, srt, off, g.offsets, p)
    out = dict(rec=rec, sorted=srt, off=off, runs=druns)
    want_pack = oracle.pack(g.seq)
    for got, w, name in zip((packed, mask, nbits), want_pack, ("packed", "mask", "nbits")):
        assert np.array_equal(got.cpu().numpy().view(np.uint32)[:len(w)], w), name
    assert_rows_equal(rec_rows(rec), recs, "sketch")
    assert_rows_equal(rec_rows(srt), idx_rows, "index")
    assert np.array_equal(off.cpu().numpy().view(np.uint32), idx_off)
    assert_rows_equal(run_rows(druns), runs, "runs")
    if check_chain:
        ref["chains"] = oracle.chain(runs, recs, g.offsets, recs, g.offsets, pd)
        ref["cands"] = oracle.merge(ref["chains"], pd)
        chains, nc = ctx.sedef_chain(druns, nr, rec, g.offsets, srt, off, g.offsets, p)
        cands, _ = ctx.sedef_merge(chains, nc, g.offsets, g.offsets, p)
        out.update(chains=chains, cands=cands)
        assert_rows_equal(chain_rows(chains), ref["chains"], "chains")
        assert_rows_equal(cand_rows_global(cands, g.offsets), ref["cands"], "candidates")
    return ref, out


# ----------------------------------------------------------------- pack ----

@pytest.mark.parametrize("n", [1, 15, 16, 17, 33, 1000, 100_003, 1 << 20])
@pytest.mark.parametrize("offset", [0, 3])
def test_pack(ctx, n, offset):
    rng = np.random.default_rng(n + offset)
    base = np.concatenate([np.frombuffer(b"ACGTacgtNnRY-\x00\xff", dtype=np.uint8),
                           rng.integers(0, 256, n + 32).astype(np.uint8)])
    seq = base[:n + offset]
    d = to_dev(seq)[offset:]  # an unaligned device pointer when offset != 0
    packed, mask, nbits = ctx.sedef_pack(d)
    want = oracle.pack(seq[offset:])
    for got, w, name in zip((packed, mask, nbits), want, ("packed", "mask", "nbits")):
        assert np.array_equal(got.cpu().numpy().view(np.uint32)[:len(w)], w), name


# ---------------------------------------------------------------- sketch ---

SKETCH_CASES = [
    (1, (30_000,), dict(oracle.DEFAULTS)),
    (2, (5, 11, 17, 40_000, 3, 9000), dict(oracle.DEFAULTS)),
    (3, (70_000,), dict(oracle.DEFAULTS, k=5, w=4)),
    (4, (50_000, 20_000), dict(oracle.DEFAULTS, k=15, w=1)),
    (5, (40_000,), dict(oracle.DEFAULTS, k=9, w=9)),
    (6, (40_000,), dict(oracle.DEFAULTS, k=11, w=64, min_unmasked=4)),
    (7, (30_000, 8000), dict(oracle.DEFAULTS, k=2, w=256)),
    (8, (33_333,), dict(oracle.DEFAULTS, k=13, w=8)),
]


@pytest.mark.parametrize("seed,lengths,pd", SKETCH_CASES)
def test_sketch_and_index(ctx, seed, lengths, pd):
    g = synth.small_case(seed, lengths=lengths, n_sd=2, sd_lo=200, sd_hi=800, mask_frac=0.3,
                         n_gaps=True)
    # tandem repeats and a palindromic run inside the first sequence
    motif = np.frombuffer((b"ACGTTA" * 20) + (b"ACGTACGTACGT" * 5) + (b"aaaaaaaaaaaaaaaaaaaaa"),
                          dtype=np.uint8)
    if len(g.seq) > len(motif) + 100:
        g.seq[50:50 + len(motif)] = motif
    p = binding.params_from_dict(pd)
    d = to_dev(g.seq)
    packed, mask, nbits = ctx.sedef_pack(d)
    rec = ctx.sedef_sketch(packed, mask, nbits, g.offsets, p)
    ref = oracle.sketch(g.seq, g.offsets, pd)
    assert_rows_equal(rec_rows(rec), ref, "sketch")
    srt, off = ctx.sedef_index(rec, p)
    want_rows, want_off = oracle.index(ref, pd["k"])
    assert_rows_equal(rec_rows(srt), want_rows, "index")
    assert np.array_equal(off.cpu().numpy().view(np.uint32), want_off)


def test_sketch_empty_and_short(ctx):
    p = binding.params()
    for lengths in [(0,), (5,), (26,), (27,), (0, 30, 0)]:
        offs = np.concatenate([[0], np.cumsum(lengths)]).astype(np.int64)
        seq = synth.random_bases(np.random.default_rng(1), int(offs[-1]))
        if len(seq) == 0:
            continue
        d = to_dev(seq)
        packed, mask, nbits = ctx.sedef_pack(d)
        rec = ctx.sedef_sketch(packed, mask, nbits, offs, p)
        ref = oracle.sketch(seq, offs, oracle.params())
        assert_rows_equal(rec_rows(rec), ref, f"sketch {lengths}")


# ------------------------------------------------------- filter to merge ---

@pytest.mark.parametrize("seed", [11, 12, 13])
def test_tiny_params_full(ctx, seed):
    g = synth.small_case(seed, lengths=(700, 450), n_sd=3, sd_lo=60, sd_hi=150, id_lo=0.9,
                         id_hi=1.0, mask_frac=0.15, n_gaps=True, inter_frac=0.5,
                         repeat_lengths=(15, 30))
    full_parity(ctx, g, dict(TINY))


@pytest.mark.parametrize("pd", [dict(TINY, self_mode=1, max_occ=4),
                                dict(TINY, step=1, n=30),
                                dict(TINY, k=4, w=3, n=25, step=5)])
def test_tiny_param_variants(ctx, pd):
    g = synth.small_case(21, lengths=(900, 300, 500), n_sd=4, sd_lo=60, sd_hi=200, id_lo=0.9,
                         id_hi=1.0, mask_frac=0.15, n_gaps=True, inter_frac=0.5,
                         repeat_lengths=(15, 30))
    full_parity(ctx, g, pd)


@pytest.mark.parametrize("seed", [31, 32])
def test_default_params_multi_sequence(ctx, seed):
    g = synth.small_case(seed, lengths=(120_000, 45_000, 2_000, 80_000), n_sd=8, sd_lo=1500,
                         sd_hi=9000, id_lo=0.85, id_hi=0.995, mask_frac=0.25, n_gaps=True,
                         inter_frac=0.4)
    ref, _ = full_parity(ctx, g, oracle.params())
    assert len(ref["cands"]) > 0


def test_dense_winnowing_large_domains(ctx):
    """w = 5 gives ~246 query minimizers per window and ~490 span records per
    run, so the refine's domain sort pads to 1024 entries."""
    g = synth.small_case(34, lengths=(60_000,), n_sd=4, sd_lo=2000, sd_hi=5000, id_lo=0.92,
                         mask_frac=0.1)
    full_parity(ctx, g, oracle.params(w=5))


def test_occurrence_cap(ctx):
    g = synth.small_case(33, lengths=(150_000,), n_sd=6, sd_lo=1500, sd_hi=6000, id_lo=0.9,
                         mask_frac=0.2)
    full_parity(ctx, g, oracle.params(max_occ=3))


def test_overflow_windows_use_global_path(ctx):
    """Windows with > 256 query minimizers (w = 1), > 65535 hits (a long
    unmasked poly-A run) or > 1024 collected hits go through the global-memory
    path; results must still equal the oracle's."""
    rng = np.random.default_rng(5)
    parts = [synth.random_bases(rng, 30_000)]
    parts[0][5_000:15_000] = ord("A")            # 10 kbp poly-A: many hits per window
    parts.append(np.full(3_000, ord("C"), dtype=np.uint8))
    parts.append(synth.random_bases(rng, 20_000))
    g = synth.genome_from_parts(parts)
    full_parity(ctx, g, oracle.params(), check_chain=False)
    full_parity(ctx, g, oracle.params(w=1, k=13), check_chain=False)


def repeat_family_genome(seed=91, length=300_000, elem=1000, copies=150, id_lo=0.97,
                         id_hi=0.995):
    """150 unmasked copies of one 1 kbp element (97-99.5% identity, either
    strand): posting lists ~150 long, like those of a large genome, so most
    windows have more than 4,096 hits."""
    rng = np.random.default_rng(seed)
    seq = synth.random_bases(rng, length, 0.41)
    unit = synth.random_bases(rng, elem, 0.41)
    starts = np.sort(rng.choice(np.arange(0, length - elem, elem + 200), size=copies,
                                replace=False))
    for a in starts:
        pc = synth.mutate(rng, unit, float(rng.uniform(id_lo, id_hi)))
        if rng.random() < 0.5:
            pc = synth.reverse_complement(pc)
        seq[a:a + len(pc)] = pc[:length - a]
    return synth.genome_from_parts([seq])


def test_wide_tier_long_postings(ctx):
    """Windows with more hits than a 2,048-slot prefilter can separate go to
    the wide tier (32,768 slots), and from there to the global path when
    they collect more than it holds; every stage must still equal the
    oracle, under every first-tier shape."""
    g = repeat_family_genome()
    ref, out = full_parity(ctx, g, oracle.params())
    assert len(ref["runs"]) > 10_000 and len(ref["cands"]) > 0
    st = ctx.sedef_filter_stats()
    assert st["windows"] > 1000
    p = binding.params()
    _, count = ctx.sedef_filter_variant()
    for v in range(0, count, 5):
        ctx.sedef_filter_variant(v)
        runs, _ = ctx.sedef_filter(out["rec"], g.offsets, out["rec"], out["sorted"], out["off"],
                                   g.offsets, p)
        assert_rows_equal(run_rows(runs), ref["runs"], f"runs (shape {v})")
    ctx.sedef_filter_variant(0)
    # under the shared-memory cap of a context that runs beside the serving
    # kernel the second wide tier's smaller form takes its place, and under
    # a lower cap its windows go to the global path
    with pytest.raises(binding.SedefError) as e:
        ctx.sedef_set_tier_smem_limit(64 * 1024)
    assert e.value.status == -5
    for cap, wide2, mid in [(-1, True, False), (160 * 1024, False, True),
                            (100 * 1024, False, False)]:
        ctx.sedef_set_tier_smem_limit(cap)
        ctx.sedef_trace_enable(True)
        ctx.sedef_trace_report(reset=True)
        runs, _ = ctx.sedef_filter(out["rec"], g.offsets, out["rec"], out["sorted"], out["off"],
                                   g.offsets, p)
        names = ctx.sedef_trace_report(reset=True)
        ctx.sedef_trace_enable(False)
        assert any(n.endswith("k_filter_wide2") for n in names) == wide2, sorted(names)
        assert any(n.endswith("k_filter_widemid") for n in names) == mid, sorted(names)
        assert_rows_equal(run_rows(runs), ref["runs"], f"runs (tier cap {cap})")
    ctx.sedef_set_tier_smem_limit(-1)


def test_chain_refuses_degenerate_seeds(ctx):
    """A seed inside a long unmasked poly-A run has millions of anchors; the
    chain call reports it instead of running the quadratic DP."""
    rng = np.random.default_rng(8)
    seq = synth.random_bases(rng, 40_000)
    seq[5_000:35_000] = ord("A")
    g = synth.genome_from_parts([seq])
    p = binding.params()
    d = to_dev(g.seq)
    rec = ctx.sedef_sketch(*ctx.sedef_pack(d), g.offsets, p)
    srt, off = ctx.sedef_index(rec, p)
    runs, nr = ctx.sedef_filter(rec, g.offsets, rec, srt, off, g.offsets, p)
    with pytest.raises(binding.SedefError) as e:
        ctx.sedef_chain(runs, nr, rec, g.offsets, srt, off, g.offsets, p)
    assert e.value.status == -5


def test_huge_posting_lists(ctx):
    rng = np.random.default_rng(6)
    seq = synth.random_bases(rng, 90_000)
    seq[2_000:75_000] = ord("T")                 # one hash with > 65535 postings
    g = synth.genome_from_parts([seq])
    full_parity(ctx, g, oracle.params(step=2000), check_chain=False)


def test_non_self_search(ctx):
    """Query windows against a separate target (non-self mode)."""
    g = synth.small_case(41, lengths=(200_000,), n_sd=0)
    rng = np.random.default_rng(41)
    pieces = []
    for a in [5_000, 60_000, 150_000]:
        pc = synth.mutate(rng, g.seq[a:a + 4000], 0.93)
        if a == 60_000:
            pc = synth.reverse_complement(pc)
        pieces.append(pc)
    q = synth.genome_from_parts(pieces + [synth.random_bases(rng, 3000)])
    pd = oracle.params(self_mode=0)
    p = binding.params_from_dict(pd)
    tq = oracle.sketch(q.seq, q.offsets, pd)
    tt = oracle.sketch(g.seq, g.offsets, pd)
    want_runs = oracle.filter_runs(tq, q.offsets, tt, g.offsets, pd)
    want_chains = oracle.chain(want_runs, tq, q.offsets, tt, g.offsets, pd)
    want_cands = oracle.merge(want_chains, pd)
    dq, dt = to_dev(q.seq), to_dev(g.seq)
    qrec = ctx.sedef_sketch(*ctx.sedef_pack(dq), q.offsets, p)
    trec = ctx.sedef_sketch(*ctx.sedef_pack(dt), g.offsets, p)
    srt, off = ctx.sedef_index(trec, p)
    runs, nr = ctx.sedef_filter(qrec, q.offsets, trec, srt, off, g.offsets, p)
    assert_rows_equal(run_rows(runs), want_runs, "runs")
    chains, nc = ctx.sedef_chain(runs, nr, qrec, q.offsets, srt, off, g.offsets, p)
    assert_rows_equal(chain_rows(chains), want_chains, "chains")
    cands, ncd = ctx.sedef_merge(chains, nc, q.offsets, g.offsets, p)
    got = binding.struct_view(cands, binding.CAND_DTYPE)
    # candidates: query coordinates are per query sequence, target per target
    if ncd:
        qo, to = q.offsets, g.offsets
        rows = np.stack([got["qseq"], got["q0"] + qo[got["qseq"]], got["q1"] + qo[got["qseq"]],
                         got["tseq"], got["t0"] + to[got["tseq"]], got["t1"] + to[got["tseq"]],
                         got["o"], got["score"], got["nchains"]], axis=1).astype(np.int64)
    else:
        rows = np.zeros((0, 9), dtype=np.int64)
    assert_rows_equal(rows, want_cands, "candidates")
    assert len(want_cands) >= 3


def test_plain_2mbp_full(ctx):
    """The 2 Mbp workload (20 planted duplications) end to end."""
    g = synth.plain_2mbp()
    ref, _ = full_parity(ctx, g, oracle.params())
    assert len(ref["cands"]) >= 10


def test_selfsearch_host_matches_stages(ctx):
    g = synth.small_case(51, lengths=(150_000, 60_000), n_sd=6, sd_lo=1500, sd_hi=6000,
                         id_lo=0.88, mask_frac=0.2, n_gaps=True)
    pd = oracle.params()
    ref = oracle.selfsearch(g.seq, g.offsets, pd)
    cands = ctx.sedef_selfsearch_host(g.seq, g.offsets, binding.params_from_dict(pd))
    assert_rows_equal(cand_rows_global(cands, g.offsets), ref["cands"], "candidates")


def test_every_filter_shape_gives_the_same_runs(ctx):
    """The first-tier shapes the autotuner picks from (and the tiers windows
    overflow into) must not change any result."""
    g = synth.small_case(61, lengths=(150_000, 40_000), n_sd=8, sd_lo=1500, sd_hi=9000,
                         id_lo=0.85, mask_frac=0.25, n_gaps=True, inter_frac=0.4)
    rng = np.random.default_rng(61)
    unit = synth.random_bases(rng, 600)
    g.seq[20_000:20_000 + 600 * 12] = np.tile(unit, 12)  # a 12-copy tandem array: large windows
    pd = oracle.params()
    recs = oracle.sketch(g.seq, g.offsets, pd)
    want = oracle.filter_runs(recs, g.offsets, recs, g.offsets, pd)
    p = binding.params_from_dict(pd)
    rec = ctx.sedef_sketch(*ctx.sedef_pack(to_dev(g.seq)), g.offsets, p)
    srt, off = ctx.sedef_index(rec, p)
    _, count = ctx.sedef_filter_variant()
    assert count >= 2
    for v in range(count):
        ctx.sedef_filter_variant(v)
        runs, _ = ctx.sedef_filter(rec, g.offsets, rec, srt, off, g.offsets, p)
        assert_rows_equal(run_rows(runs), want, f"runs (shape {v})")
    chosen = ctx.sedef_filter_autotune(rec, g.offsets, rec, srt, off, g.offsets, p)
    assert 0 <= chosen < count and ctx.sedef_filter_variant()[0] == chosen
    ctx.sedef_filter_variant(0)


# ------------------------------------------------------- f3 q-gram filter ----

@pytest.mark.parametrize("q", [1, 3, 4, 5])
def test_qgram_filter(ctx, q):
    """Shared q-grams and pass flags of every kept seed equal the oracle's
    (masked bases, N runs, both orientations, several sequences)."""
    g = synth.small_case(71 + q, lengths=(90_000, 40_000, 5_000), n_sd=6, sd_lo=1500, sd_hi=9000,
                         id_lo=0.78, mask_frac=0.2, n_gaps=True)
    pd = oracle.params()
    p = binding.params_from_dict(pd)
    recs = oracle.sketch(g.seq, g.offsets, pd)
    runs = oracle.filter_runs(recs, g.offsets, recs, g.offsets, pd)
    want = oracle.qgram(g.seq, runs, pd, q=q, p_gap=0.005)
    d = to_dev(g.seq)
    packed, mask, nbits = ctx.sedef_pack(d)
    rec = ctx.sedef_sketch(packed, mask, nbits, g.offsets, p)
    srt, off = ctx.sedef_index(rec, p)
    druns, nr = ctx.sedef_filter(rec, g.offsets, rec, srt, off, g.offsets, p)
    assert_rows_equal(run_rows(druns), runs, "runs")
    shared, ok, npass = ctx.sedef_qgram(packed, nbits, g.length, druns, nr, p, q=q, p_gap=0.005)
    got = np.stack([shared.cpu().numpy().view(np.uint32).astype(np.int64),
                    ok.cpu().numpy().astype(np.int64)], axis=1)
    assert_rows_equal(got, want, f"q-gram rows (q={q})")
    assert npass == int(want[:, 1].sum())
    assert (runs[:, oracle.RUN_COLS.index("keep")] == 1).sum() > 0
