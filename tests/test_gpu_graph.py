"""The captured pass (sedef_graph_*): one CUDA graph per input layout, no
host synchronization inside, capacities instead of exact sizes.  Its
outputs must equal the step-by-step calls bit for bit (and so the oracle's),
on replays, after the input is refilled, in batch mode, through the global
path; overflow of any capacity must be reported with the exact totals."""
import numpy as np
import pytest

import oracle
from paper_1807_00205_gb300 import batch, binding, synth
from tests.gpu_helpers import assert_rows_equal, cand_rows_global, chain_rows, need_gpu, rec_rows, run_rows
from tests.test_gpu_parity import full_parity, to_dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    need_gpu()
    c = binding.Context(0)
    yield c
    c.close()


def assert_same(got: dict, want: dict, what: str):
    assert np.array_equal(rec_rows(got["rec"]), rec_rows(want["rec"])), what + " records"
    assert np.array_equal(rec_rows(got["sorted"]), rec_rows(want["sorted"])), what + " index"
    assert np.array_equal(got["off"].cpu().numpy(), want["off"].cpu().numpy()), what + " offsets"
    assert_rows_equal(run_rows(got["runs"]), run_rows(want["runs"]), what + " runs")
    assert_rows_equal(chain_rows(got["chains"]), chain_rows(want["chains"]), what + " chains")
    a = binding.struct_view(got["cands"], binding.CAND_DTYPE)
    b = binding.struct_view(want["cands"], binding.CAND_DTYPE)
    assert np.array_equal(a, b), what + " candidates"


def test_graph_equals_stages_and_oracle(ctx):
    g = synth.small_case(91, lengths=(120_000, 3_000, 60_000, 900), n_sd=6, sd_lo=1500,
                         sd_hi=8000, id_lo=0.85, mask_frac=0.25, n_gaps=True)
    pd = oracle.params()
    p = binding.params_from_dict(pd)
    d = to_dev(g.seq)
    eager = ctx.selfsearch(d, g.offsets, p)
    gr = ctx.selfsearch_graph(d, g.offsets, p)
    assert gr.nodes > 20
    assert_same(gr.outputs(), eager, "first run")
    ref, _ = full_parity(ctx, g, pd)
    assert_rows_equal(cand_rows_global(gr.outputs()["cands"], g.offsets), ref["cands"], "oracle")
    # replays give the same outputs, and each counts its kernel nodes
    n0 = binding.Context.sedef_launch_count()
    for _ in range(3):
        gr.launch()
        gr.wait()
    assert binding.Context.sedef_launch_count() - n0 == 3 * gr.nodes
    assert_same(gr.outputs(), eager, "replay")
    gr.close()


def test_graph_reads_refilled_input(ctx):
    """The graph reads the input buffer at every launch: new bases in the same
    layout give that input's results."""
    a = synth.small_case(92, lengths=(80_000, 40_000), n_sd=4, mask_frac=0.1)
    b = synth.small_case(93, lengths=(80_000, 40_000), n_sd=5, mask_frac=0.3)
    p = binding.params()
    d = to_dev(a.seq)
    caps = {k: 200_000 for k in binding.CAP_NAMES}
    gr = binding.Graph(ctx, d, a.offsets, p, caps)
    gr.launch()
    gr.wait()
    assert_same(gr.outputs(), ctx.selfsearch(to_dev(a.seq), a.offsets, p), "input a")
    d.copy_(to_dev(b.seq))
    gr.launch()
    gr.wait()
    assert_same(gr.outputs(), ctx.selfsearch(to_dev(b.seq), b.offsets, p), "input b")
    gr.close()


def test_graph_capacity_overflow_reports_totals(ctx):
    g = synth.small_case(94, lengths=(150_000,), n_sd=8, sd_lo=2000, sd_hi=10_000, mask_frac=0.2)
    p = binding.params()
    d = to_dev(g.seq)
    eager = ctx.selfsearch(d, g.offsets, p)
    for name in ["records", "runs", "chains", "cands"]:
        caps = {k: 1 << 20 for k in binding.CAP_NAMES}
        caps[name] = 3
        gr = binding.Graph(ctx, d, g.offsets, p, caps)
        gr.launch()
        with pytest.raises(binding.SedefError) as e:
            gr.wait()
        assert e.value.status == binding.SEDEF_ERR_CAPACITY
        assert name in str(e.value)
        gr.close()
    # exact totals from a graph that fits
    gr = ctx.selfsearch_graph(d, g.offsets, p)
    need = gr.need
    assert need["records"] == eager["rec"].numel()
    assert need["runs"] == eager["nruns"] and need["chains"] == eager["nchains"]
    assert need["cands"] == eager["ncands"]
    # the rebuild loop: start from capacities of 1
    gr2 = ctx.selfsearch_graph(d, g.offsets, p, caps={k: 1 for k in binding.CAP_NAMES})
    assert_same(gr2.outputs(), eager, "rebuilt")
    gr.close()
    gr2.close()


def test_graph_global_path(ctx):
    """w = 1 puts every window on the global (overflow) path; the graph runs
    it in one planned batch."""
    g = synth.small_case(95, lengths=(60_000, 30_000), n_sd=4, sd_lo=1500, sd_hi=6000,
                         id_lo=0.9)
    pd = oracle.params(w=1, k=13)
    p = binding.params_from_dict(pd)
    d = to_dev(g.seq)
    eager = ctx.selfsearch(d, g.offsets, p)
    assert ctx.sedef_filter_stats()["overflow_windows"] > 0
    gr = ctx.selfsearch_graph(d, g.offsets, p)
    assert gr.need["slow_hits"] > 0
    assert_same(gr.outputs(), eager, "global path")
    caps = dict(gr.caps)
    caps["slow_hits"] = gr.need["slow_hits"] - 1
    small = binding.Graph(ctx, d, g.offsets, p, caps)
    small.launch()
    with pytest.raises(binding.SedefError, match="slow_hits"):
        small.wait()
    small.close()
    gr.close()


def test_graph_anchor_limit(ctx):
    """A seed with more than 65,536 anchors is refused, as by sedef_chain."""
    rng = np.random.default_rng(6)
    seq = synth.random_bases(rng, 60_000)
    seq[10_000:40_000] = ord("A")
    g = synth.genome_from_parts([seq])
    p = binding.params()
    caps = binding.default_caps(g.length)
    caps["slow_hits"] = 1 << 23
    gr = binding.Graph(ctx, to_dev(g.seq), g.offsets, p, caps)
    gr.launch()
    with pytest.raises(binding.SedefError) as e:
        gr.wait()
    assert e.value.status == -5  # SEDEF_ERR_UNSUPPORTED
    gr.close()


def test_graph_batch_self_mode_2(ctx):
    from tests.test_gpu_batch import small_batch
    gs = small_batch(17, count=10)
    seq, offs = batch.concatenate(gs)
    p = binding.params(self_mode=2)
    d = to_dev(seq)
    eager = batch.batched(ctx, d, offs, p)
    gr = ctx.selfsearch_graph(d, offs, p)
    assert_same(gr.outputs(), eager, "batch")
    gr.close()


def test_graph_plain_2mbp(ctx):
    g = synth.plain_2mbp()
    p = binding.params()
    d = to_dev(g.seq)
    ctx.selfsearch(d, g.offsets, p, autotune=True)
    eager = ctx.selfsearch(d, g.offsets, p)
    gr = ctx.selfsearch_graph(d, g.offsets, p)
    assert_same(gr.outputs(), eager, "2 Mbp")
    gr.close()
