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


def _alone(ctx, index, pool, p):
    out = []
    for k, q in enumerate(pool):
        r = serve.Request(rid=k, seq=q)
        serve.search(ctx, index, [r], p)
        out.append(r.cands)
    return out


def test_device_queue_more_requests_than_slots():
    """Two slots, fourteen requests arriving at once: requests wait for a
    slot, join the running kernel as slots free up, and each result equals
    the request searched alone."""
    need_gpu()
    g = synth.small_case(88, lengths=(400_000, 150_000), n_sd=8, sd_lo=2000, sd_hi=12000,
                         id_lo=0.85, mask_frac=0.2, n_gaps=True)
    ctx = binding.Context(0)
    p = binding.params()
    index = serve.ResidentIndex(ctx, g.seq, g.offsets, p)
    pool = synth.query_regions(g, 14, seed=5, len_lo=3_000, len_hi=40_000)
    alone = _alone(ctx, index, pool, p)
    srv = serve.Server(index, p, batching=True, slots=2, slot_bases=50_000)
    assert srv.device_queue and srv.nslots == 2
    srv.start()
    serve.run_load(srv, pool, rate=1e6, count=len(pool), seed=2)
    srv.close()
    got = {r.rid: r.cands for r in srv.completed}
    for k in range(len(pool)):
        assert np.array_equal(got[k], alone[k]), k
    assert sum(len(a) for a in alone) > 0
    ctx.close()


def test_device_queue_idle_wait_times_out_and_restarts():
    """The persistent kernel's wait for work is bounded: with nothing
    submitted for longer than the idle limit it leaves and the server reports
    SEDEF_ERR_TIMEOUT; the next request launches it again and is served
    correctly."""
    import time
    need_gpu()
    g = synth.small_case(89, lengths=(200_000,), n_sd=4, sd_lo=2000, sd_hi=8000, id_lo=0.9)
    ctx = binding.Context(0)
    p = binding.params()
    index = serve.ResidentIndex(ctx, g.seq, g.offsets, p)
    pool = synth.query_regions(g, 2, seed=7, len_lo=5_000, len_hi=20_000)
    alone = _alone(ctx, index, pool, p)
    dev = binding.DeviceServer(ctx, index.trec, index.tsorted, index.toff, index.offsets, p,
                               slots=2, slot_bases=50_000, idle_timeout_s=0.2)

    def one(q):
        slot = dev.submit(q)
        assert slot is not None
        done = None
        t0 = time.time()
        while done is None and time.time() - t0 < 30:
            done = dev.poll(0.01)
        assert done == slot
        c = dev.finish(slot)
        c["qseq"] = 0
        return c

    assert np.array_equal(one(pool[0]), alone[0])
    time.sleep(1.0)  # nothing to do for five idle limits
    st = dev.status()
    assert st == {"status": -4, "running": False, "timed_out": True}
    assert np.array_equal(one(pool[1]), alone[1])  # relaunched
    assert dev.status()["status"] in (0, -4)
    dev.close()
    ctx.close()


def test_device_queue_finish_runs_beside_the_kernel():
    """Dense winnowing (w = 5) sends runs to the refine kernel with the
    largest shared-memory block (about 122 KB per CTA).  It must run on the
    SMs beside the persistent kernel rather than wait for that kernel to
    leave: with a 20 s idle limit the request still finishes in seconds, with
    the result of the request searched alone."""
    import time
    need_gpu()
    g = synth.small_case(90, lengths=(120_000,), n_sd=4, sd_lo=2000, sd_hi=6000, id_lo=0.92,
                         mask_frac=0.1)
    ctx = binding.Context(0)
    p = binding.params(w=5)
    index = serve.ResidentIndex(ctx, g.seq, g.offsets, p)
    pool = synth.query_regions(g, 2, seed=11, len_lo=20_000, len_hi=40_000, mut_hi=0.05)
    alone = _alone(ctx, index, pool, p)
    assert ctx.sedef_filter_stats()["big_refine"] > 0
    dev = binding.DeviceServer(ctx, index.trec, index.tsorted, index.toff, index.offsets, p,
                               slots=2, slot_bases=50_000, idle_timeout_s=20.0)
    assert dev.smem_left() >= 100 * 1024
    for q, want in zip(pool, alone):
        slot = dev.submit(q)
        assert slot is not None
        done = None
        t0 = time.time()
        while done is None and time.time() - t0 < 30:
            done = dev.poll(0.01)
        assert done == slot
        c = dev.finish(slot)
        took = time.time() - t0
        assert dev.status()["running"]  # the kernel is still resident
        c["qseq"] = 0
        assert np.array_equal(c, want)
        assert took < 5.0, took
    dev.close()
    ctx.close()
