"""Full-size parity on sampled outputs.

The chromosome-scale self-search (100 Mbp) runs exactly as the benchmark
runs it (autotuned filter shapes, one context, device-resident input); the
200-genome batch runs as one self_mode 2 pass.  The oracle checks what it can
compute one piece at a time: every sketch record and the whole index of the
100 Mbp genome, the runs and chains of sampled query windows (a random
sample plus windows inside planted duplications), whole genomes sampled from
the batch, and properties of the merged candidates that hold at any size.
"""
import numpy as np
import pytest

import oracle
from paper_1807_00205_gb300 import batch, binding, synth
from tests.gpu_helpers import (assert_rows_equal, cand_rows_global, chain_rows, need_gpu,
                               rec_rows, run_rows)
from tests.test_gpu_parity import full_parity, to_dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    need_gpu()
    c = binding.Context(0)
    yield c
    c.close()


def window_starts(g, pd):
    """Every query window start (each sequence start, then every query_step)."""
    out = []
    for s in range(g.nseq):
        a, b = int(g.offsets[s]), int(g.offsets[s + 1])
        out.append(np.arange(a, b - pd["n"] + 1, pd["step"], dtype=np.int64))
    return np.concatenate(out) if out else np.zeros(0, np.int64)


def sample_windows(g, pd, seed, n_random, n_planted):
    """A seeded random sample of window starts plus the first window inside
    the source and the copy of planted duplications."""
    rng = np.random.default_rng(seed)
    starts = window_starts(g, pd)
    pick = list(rng.choice(starts, size=min(n_random, len(starts)), replace=False))
    sds = [d for d in g.planted if d.length >= pd["n"] + pd["step"]]
    for d in [sds[k] for k in rng.permutation(len(sds))[:n_planted]]:
        for a, ln in ((d.src, d.length), (d.dst, d.copy_length)):
            k = np.searchsorted(starts, a)
            if k < len(starts) and starts[k] + pd["n"] <= a + ln:
                pick.append(starts[k])
    return np.unique(np.asarray(pick, dtype=np.int64))


def check_candidate_properties(chains: np.ndarray, cands: np.ndarray):
    """Merge invariants: candidates are sorted by (q0, t0, o, q1, t1); they
    account for every chain and all of its score; every chain's box lies in
    a candidate of the same (query sequence, target sequence, orientation)."""
    ci = {c: k for k, c in enumerate(oracle.CAND_COLS)}
    hi = {c: k for k, c in enumerate(oracle.CHAIN_COLS)}
    assert len(cands) > 0
    key = cands[:, [ci["q0"], ci["t0"], ci["o"], ci["q1"], ci["t1"]]]
    order = np.lexsort(key.T[::-1])
    assert np.array_equal(order, np.arange(len(cands))), "candidates not sorted"
    assert cands[:, ci["nchains"]].sum() == len(chains)
    assert cands[:, ci["score"]].sum() == chains[:, hi["score"]].sum()
    # containment: candidates of a (qseq, tseq, o) group sorted by q0; a
    # chain's container has q0 <= the chain's q0, so look back from there
    grp_c = (cands[:, ci["qseq"]] << 33) | (cands[:, ci["tseq"]] << 1) | cands[:, ci["o"]]
    grp_h = (chains[:, hi["qseq"]] << 33) | (chains[:, hi["tseq"]] << 1) | chains[:, hi["o"]]
    oc = np.lexsort((cands[:, ci["q0"]], grp_c))
    c_sorted = cands[oc]
    g_sorted = grp_c[oc]
    comp = (g_sorted.astype(np.float64) * 2.0**33) + c_sorted[:, ci["q0"]]
    want = (grp_h.astype(np.float64) * 2.0**33) + chains[:, hi["q0"]]
    top = np.searchsorted(comp, want, side="right") - 1
    # look back from each chain over its group's candidates (q0 <= the
    # chain's q0), only for the chains not yet placed
    todo = np.arange(len(chains))
    stuck = [np.zeros(0, dtype=np.int64)]
    for back in range(64):
        if len(todo) == 0:
            break
        k = top[todo] - back
        ok = (k >= 0) & (g_sorted[np.maximum(k, 0)] == grp_h[todo])
        kk = np.where(ok, k, 0)
        c = c_sorted[kk]
        h = chains[todo]
        inside = (ok & (c[:, ci["q0"]] <= h[:, hi["q0"]]) & (c[:, ci["q1"]] >= h[:, hi["q1"]])
                  & (c[:, ci["t0"]] <= h[:, hi["t0"]]) & (c[:, ci["t1"]] >= h[:, hi["t1"]]))
        stuck.append(todo[~ok])  # left its group without a container
        todo = todo[ok & ~inside]
    stuck = np.concatenate(stuck + [todo])
    # chains not placed within 64 candidates: a seeded sample of them, each
    # against every candidate of its group with q0 <= the chain's q0
    rng = np.random.default_rng(0)
    for x in rng.permutation(stuck)[:300]:
        lo = int(np.searchsorted(g_sorted, grp_h[x], side="left"))
        c = c_sorted[lo:top[x] + 1]
        inside = ((c[:, ci["q0"]] <= chains[x, hi["q0"]]) & (c[:, ci["q1"]] >= chains[x, hi["q1"]])
                  & (c[:, ci["t0"]] <= chains[x, hi["t0"]]) & (c[:, ci["t1"]] >= chains[x, hi["t1"]]))
        assert inside.any(), f"chain {chains[x].tolist()} lies in no candidate"


def test_chromosome_100mbp_sampled(ctx):
    g = synth.chromosome_100mbp()
    pd = oracle.params()
    p = binding.params_from_dict(pd)
    out = ctx.selfsearch(to_dev(g.seq), g.offsets, p, autotune=True)
    # sketch and index: every record
    recs = oracle.sketch(g.seq, g.offsets, pd)
    assert_rows_equal(rec_rows(out["rec"]), recs, "sketch")
    idx, off = oracle.index(recs, pd["k"])
    assert_rows_equal(rec_rows(out["sorted"]), idx, "index")
    assert np.array_equal(out["off"].cpu().numpy().view(np.uint32), off)
    del idx, off
    # filter, refine and chain: sampled windows
    win = sample_windows(g, pd, seed=11, n_random=150, n_planted=60)
    runs = oracle.filter_runs(recs, g.offsets, recs, g.offsets, pd, windows=win)
    got = run_rows(out["runs"])
    assert_rows_equal(got[np.isin(got[:, 0], win)], runs, "runs of sampled windows")
    assert (runs[:, oracle.RUN_COLS.index("keep")] == 1).sum() >= 40  # the sample has seeds
    chains = oracle.chain(runs, recs, g.offsets, recs, g.offsets, pd)
    gch = chain_rows(out["chains"])
    assert_rows_equal(gch[np.isin(gch[:, 0], win)], chains, "chains of sampled windows")
    # merge: invariants over the whole output
    check_candidate_properties(gch, cand_rows_global(out["cands"], g.offsets))


def test_batch_200_genomes_sampled(ctx):
    gs = synth.batch_genomes()
    seq, offs = batch.concatenate(gs)
    p = binding.params()
    out = batch.batched(ctx, to_dev(seq), offs, p)
    pd = oracle.params(self_mode=2)
    rec = binding.to_numpy_records(out["rec"])
    srt = binding.to_numpy_records(out["sorted"])
    # index: the records sorted by (hash, position), offsets over every hash
    assert np.array_equal(srt, np.sort(rec))
    h = (srt >> np.uint64(33)).astype(np.int64)
    want_off = np.searchsorted(h, np.arange((1 << (2 * pd["k"])) + 1)).astype(np.uint32)
    assert np.array_equal(out["off"].cpu().numpy().view(np.uint32), want_off)
    pos = ((rec >> np.uint64(1)) & np.uint64(0xFFFFFFFF)).astype(np.int64)
    runs = run_rows(out["runs"])
    chains = chain_rows(out["chains"])
    cands = binding.struct_view(out["cands"], binding.CAND_DTYPE)
    per = batch.split_candidates(cands, len(gs))
    check_candidate_properties(chains, cand_rows_global(cands, offs))
    # whole genomes against the oracle: three small ones and the last one
    rng = np.random.default_rng(5)
    small = [k for k, g in enumerate(gs) if g.length <= 2_500_000]
    sample = sorted(set(rng.choice(small, size=3, replace=False).tolist()) | {len(gs) - 1})
    for gi in sample:
        g = gs[gi]
        a, b = int(offs[gi]), int(offs[gi + 1])
        one = synth.Genome(g.seq, np.array([0, g.length], dtype=np.int64), g.planted)
        ref, _ = full_parity(ctx, one, pd)
        lo, hi = np.searchsorted(pos, [a, b])
        got = binding.records_to_rows(rec[lo:hi])
        got[:, 1] -= a
        assert_rows_equal(got, ref["recs"], f"sketch of genome {gi}")
        r = runs[(runs[:, 0] >= a) & (runs[:, 0] < b)].copy()
        for c in ("i", "j_a", "j_b", "j_at_max", "j_star"):
            r[:, oracle.RUN_COLS.index(c)] -= a
        assert_rows_equal(r, ref["runs"], f"runs of genome {gi}")
        c = chains[chains[:, oracle.CHAIN_COLS.index("qseq")] == gi].copy()
        for col in ("i", "q0", "q1", "t0", "t1"):
            c[:, oracle.CHAIN_COLS.index(col)] -= a
        for col in ("qseq", "tseq"):
            c[:, oracle.CHAIN_COLS.index(col)] = 0
        assert_rows_equal(c, ref["chains"], f"chains of genome {gi}")
        assert_rows_equal(cand_rows_global(per[gi], [0, g.length]), ref["cands"],
                          f"candidates of genome {gi}")


def test_human_3gbp_sampled(ctx):
    """The 3.1 Gbp human-scale self-search (24 chromosomes, index resident in
    HBM): every sketch record and the whole index against the oracle (which
    sketches the chromosomes on all host cores), the runs and chains of
    sampled windows, and the merge invariants."""
    import os
    g = synth.human_3gbp()
    pd = oracle.params()
    p = binding.params_from_dict(pd)
    d = to_dev(g.seq)
    out = ctx.selfsearch(d, g.offsets, p)  # default filter variant (parity holds for every one)
    del d
    recs = oracle.sketch(g.seq, g.offsets, pd, threads=os.cpu_count() or 1)
    assert_rows_equal(rec_rows(out["rec"]), recs, "sketch")
    # index: the whole sorted index and the offsets of every hash against
    # the oracle's
    idx_rows, idx_off = oracle.index(recs, pd["k"])
    assert_rows_equal(rec_rows(out["sorted"]), idx_rows, "index")
    assert np.array_equal(out["off"].cpu().numpy().view(np.uint32), idx_off)
    del idx_rows, idx_off
    win = sample_windows(g, pd, seed=13, n_random=100, n_planted=50)
    runs = oracle.filter_runs(recs, g.offsets, recs, g.offsets, pd, windows=win)
    got = run_rows(out["runs"])
    assert_rows_equal(got[np.isin(got[:, 0], win)], runs, "runs of sampled windows")
    assert (runs[:, oracle.RUN_COLS.index("keep")] == 1).sum() >= 30
    chains = oracle.chain(runs, recs, g.offsets, recs, g.offsets, pd)
    gch = chain_rows(out["chains"])
    assert_rows_equal(gch[np.isin(gch[:, 0], win)], chains, "chains of sampled windows")
    check_candidate_properties(gch, cand_rows_global(out["cands"], g.offsets))
    # serving against this resident index (the device work queue): 24
    # requests cut from the genome with mutation, each equal to the oracle's
    # non-self search of the region against the whole genome
    from paper_1807_00205_gb300 import serve
    from tests.test_gpu_serve import oracle_cands, served_rows
    index = serve.ResidentIndex.from_arrays(out["rec"], out["sorted"], out["off"], g.offsets, p)
    for key in ("runs", "chains", "cands", "packed", "mask", "nbits"):
        out.pop(key, None)
    pool = synth.query_regions(g, 24, seed=21, len_lo=10_000, len_hi=60_000)
    srv = serve.Server(index, p, batching=True, slots=6, slot_bases=100_000)
    srv.start()
    serve.run_load(srv, pool, rate=500.0, count=len(pool), seed=3)
    srv.close()
    got = {r.rid: r.cands for r in srv.completed}
    assert len(got) == len(pool)
    for k, q in enumerate(pool):
        assert_rows_equal(served_rows(got[k], g), oracle_cands(q, g, recs), f"served request {k}")
