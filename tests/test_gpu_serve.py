"""Serving: each request's candidates are the same alone, in one batch, and
through the continuously batched server with overlapping workers."""
import numpy as np
import pytest

import oracle
from paper_1807_00205_gb300 import binding, serve, synth
from tests.gpu_helpers import assert_rows_equal, need_gpu


def oracle_cands(q: np.ndarray, g, recs_t) -> np.ndarray:
    """The oracle's non-self search of one query region against the genome,
    as rows in global coordinates (the query is its own one-sequence input)."""
    pd = oracle.params(self_mode=0)
    qoff = np.array([0, len(q)], dtype=np.int64)
    tq = oracle.sketch(q, qoff, pd)
    runs = oracle.filter_runs(tq, qoff, recs_t, g.offsets, pd)
    chains = oracle.chain(runs, tq, qoff, recs_t, g.offsets, pd)
    return oracle.merge(chains, pd)


def served_rows(c: np.ndarray, g) -> np.ndarray:
    if len(c) == 0:
        return np.zeros((0, len(oracle.CAND_COLS)), dtype=np.int64)
    to = g.offsets
    return np.stack([c["qseq"], c["q0"], c["q1"], c["tseq"], c["t0"] + to[c["tseq"]],
                     c["t1"] + to[c["tseq"]], c["o"], c["score"], c["nchains"]],
                    axis=1).astype(np.int64)

pytestmark = pytest.mark.gpu


def test_results_same_alone_and_in_the_mix():
    need_gpu()
    g = synth.plain_2mbp()
    ctx = binding.Context(0)
    p = binding.params()
    index = serve.ResidentIndex(ctx, g.seq, g.offsets, p)
    pool = synth.query_regions(g, 14, seed=9, len_lo=5_000, len_hi=60_000)
    alone = []
    for k, q in enumerate(pool):
        r = serve.Request(rid=k, seq=q)
        serve.search(ctx, index, [r], p)
        alone.append(r.cands)
    mix = [serve.Request(rid=k, seq=q) for k, q in enumerate(pool)]
    serve.search(ctx, index, mix, p)
    for a, r in zip(alone, mix):
        assert np.array_equal(a, r.cands)
    assert sum(len(a) for a in alone) > 0
    # served results are the oracle's non-self search of each region
    recs_t = oracle.sketch(g.seq, g.offsets, oracle.params(self_mode=0))
    for k in range(0, len(pool), 3):
        assert_rows_equal(served_rows(alone[k], g), oracle_cands(pool[k], g, recs_t),
                          f"request {k}")
    srv = serve.Server(index, p, workers=2, batching=True)
    srv.start()
    res = serve.run_load(srv, pool, rate=2000.0, count=28, seed=1)
    srv.close()
    got = {r.rid: r.cands for r in srv.completed}
    for k in range(28):
        assert np.array_equal(got[k], alone[k % len(pool)]), k
    assert res["requests"] == 28
    ctx.close()


def test_index_blob_round_trip():
    """A resident index saved and restored gives the same arrays and the same
    candidates; a damaged blob is refused."""
    torch = need_gpu()
    g = synth.small_case(77, lengths=(200_000, 50_000), n_sd=5, sd_lo=2000, sd_hi=6000,
                         id_lo=0.9, mask_frac=0.2)
    ctx = binding.Context(0)
    p = binding.params()
    a = serve.ResidentIndex(ctx, g.seq, g.offsets, p)
    blob = a.save(ctx)
    b = serve.ResidentIndex(ctx, None, None, p, blob=blob)
    assert torch.equal(a.trec, b.trec) and torch.equal(a.tsorted, b.tsorted)
    assert torch.equal(a.toff, b.toff) and np.array_equal(a.offsets, b.offsets)
    pool = synth.query_regions(g, 4, seed=3, len_lo=3000, len_hi=20_000)
    ra = [serve.Request(rid=k, seq=q) for k, q in enumerate(pool)]
    rb = [serve.Request(rid=k, seq=q) for k, q in enumerate(pool)]
    serve.search(ctx, a, ra, p)
    serve.search(ctx, b, rb, p)
    for x, y in zip(ra, rb):
        assert np.array_equal(x.cands, y.cands)
    bad = bytearray(blob)
    bad[100] ^= 1
    with pytest.raises(binding.SedefError):
        serve.ResidentIndex(ctx, None, None, p, blob=bytes(bad))
    ctx.close()
