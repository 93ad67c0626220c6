"""f1 (Section 3.2, SD extension) through the C ABI against the CPU oracle.

Every kept seed grows into a potential SD region; the regions (both
intervals, the final estimate and its denominator) must equal the oracle's
bit for bit.  The seeds come from the oracle's own filter for the oracle
and from the GPU filter for the GPU (equal, as the filter parity tests
show); the extension sketches (all k-mers) likewise.
"""
import numpy as np
import pytest

import oracle
from paper_1807_00205_gb300 import binding, synth
from tests.gpu_helpers import assert_rows_equal, need_gpu
from tests.test_oracle_pins import EXTEND_CASES, _extend_case

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    need_gpu()
    c = binding.Context(0)
    yield c
    c.close()


def to_dev(a):
    torch = need_gpu()
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda:0")


def region_rows(t) -> np.ndarray:
    r = binding.struct_view(t, binding.REGION_DTYPE)
    if len(r) == 0:
        return np.zeros((0, len(oracle.EXTEND_COLS)), dtype=np.int64)
    return np.stack([r[c].astype(np.int64) for c in oracle.EXTEND_COLS], axis=1)


def gpu_extend(ctx, g, pd, max_len, keep_runs=None):
    """Seeds by the GPU filter, extension sketch and regions by the GPU."""
    p = binding.params_from_dict(pd)
    pa = binding.params_from_dict(dict(pd, min_unmasked=0))
    d = to_dev(g.seq)
    packed, mask, nbits = ctx.sedef_pack(d)
    rec = ctx.sedef_sketch(packed, mask, nbits, g.offsets, p)
    srt, off = ctx.sedef_index(rec, p)
    runs, nr = ctx.sedef_filter(rec, g.offsets, rec, srt, off, g.offsets, p)
    ext = ctx.sedef_sketch(packed, mask, nbits, g.offsets, pa)
    if keep_runs is not None:  # only these runs (indices) stay kept seeds
        v = binding.struct_view(runs, binding.RUN_DTYPE).copy()
        sel = np.zeros(len(v), dtype=bool)
        sel[keep_runs] = True
        v["keep"] = np.where(sel, v["keep"], 0)
        runs = to_dev(v.view(np.uint8))
    regions, n = ctx.sedef_extend(runs, nr, ext, g.offsets, ext, g.offsets, p, max_len=max_len)
    return region_rows(regions), binding.struct_view(runs, binding.RUN_DTYPE)


@pytest.mark.parametrize("kind,seed,p,max_len", EXTEND_CASES)
def test_extend_tiny_cases(ctx, kind, seed, p, max_len):
    g, want, _ = _extend_case(kind, seed, p, max_len)
    got, _ = gpu_extend(ctx, g, p, max_len)
    assert_rows_equal(got, np.array(want, dtype=np.int64).reshape(-1, 9), "regions")


@pytest.mark.parametrize("self_mode", [1, 2])
def test_extend_small_genome(ctx, self_mode):
    """Default parameters (k = 12, n = 750) on 60 kbp + 25 kbp with planted
    duplications, soft-masking (the extension uses masked k-mers) and N runs."""
    g = synth.small_case(7, lengths=(60_000, 25_000), n_sd=4, sd_lo=1500, sd_hi=5000,
                         id_lo=0.88, id_hi=0.99, mask_frac=0.2, n_gaps=True)
    pd = oracle.params(self_mode=self_mode)
    recs = oracle.sketch(g.seq, g.offsets, pd)
    runs = oracle.filter_runs(recs, g.offsets, recs, g.offsets, pd)
    allk = oracle.sketch(g.seq, g.offsets, dict(pd, min_unmasked=0))
    want = oracle.extend(runs, allk, g.offsets, allk, g.offsets, pd, threads=8)
    got, _ = gpu_extend(ctx, g, pd, oracle.MAX_SD_LENGTH)
    assert len(want) > 10
    assert_rows_equal(got, want, "regions")


def test_extend_plain_2mbp(ctx):
    """The 2 Mbp workload (20 planted duplications of 1-20 kbp): the regions
    of every kept seed."""
    g = synth.plain_2mbp()
    pd = oracle.params()
    recs = oracle.sketch(g.seq, g.offsets, pd)
    runs = oracle.filter_runs(recs, g.offsets, recs, g.offsets, pd, threads=8)
    allk = oracle.sketch(g.seq, g.offsets, dict(pd, min_unmasked=0))
    want = oracle.extend(runs, allk, g.offsets, allk, g.offsets, pd, threads=16)
    got, _ = gpu_extend(ctx, g, pd, oracle.MAX_SD_LENGTH)
    assert len(want) > 100
    assert_rows_equal(got, want, "regions")
    assert (want[:, 4] - want[:, 3] > pd["n"]).sum() > len(want) // 2


def test_extend_chromosome_sampled(ctx):
    """The 100 Mbp chromosome: the regions of 12 kept seeds of evenly spaced
    query windows, with potential SDs capped at 100 kbp (the oracle's
    per-step rescan makes 1 Mbp regions too slow for a test)."""
    g = synth.chromosome_100mbp()
    pd = oracle.params()
    recs = oracle.sketch(g.seq, g.offsets, pd)
    wins = np.arange(0, g.length - pd["n"] + 1, pd["step"], dtype=np.int64)
    runs = oracle.filter_runs(recs, g.offsets, recs, g.offsets, pd, windows=wins[::200],
                              threads=16)
    kept = np.nonzero(runs[:, oracle.RUN_COLS.index("keep")] == 1)[0]
    pick_rows = runs[kept[np.linspace(0, len(kept) - 1, 12).astype(np.int64)]]
    allk = oracle.sketch(g.seq, g.offsets, dict(pd, min_unmasked=0))
    want = oracle.extend(pick_rows, allk, g.offsets, allk, g.offsets, pd, max_len=100_000,
                         threads=12)
    # the GPU extends exactly these seeds (the filter's parity at this size is
    # covered by the full-size tests)
    p = binding.params_from_dict(pd)
    pa = binding.params_from_dict(dict(pd, min_unmasked=0))
    d = to_dev(g.seq)
    packed, mask, nbits = ctx.sedef_pack(d)
    ext = ctx.sedef_sketch(packed, mask, nbits, g.offsets, pa)
    cols = oracle.RUN_COLS
    v = np.zeros(len(pick_rows), dtype=binding.RUN_DTYPE)
    for c in cols:
        v[c] = pick_rows[:, cols.index(c)]
    runs_t = to_dev(v.view(np.uint8))
    regions, n = ctx.sedef_extend(runs_t, len(v), ext, g.offsets, ext, g.offsets, p,
                                  max_len=100_000)
    assert n == len(pick_rows)
    assert_rows_equal(region_rows(regions), want, "regions")


def test_extend_refuses_large_k_and_bad_cap(ctx):
    g = synth.small_case(8, lengths=(20_000,), n_sd=2)
    p = binding.params(k=13)
    d = to_dev(g.seq)
    packed, mask, nbits = ctx.sedef_pack(d)
    ext = ctx.sedef_sketch(packed, mask, nbits, g.offsets, binding.params(k=13, min_unmasked=0))
    runs = to_dev(np.zeros(1, dtype=binding.RUN_DTYPE).view(np.uint8))
    with pytest.raises(binding.SedefError) as e:
        ctx.sedef_extend(runs, 1, ext, g.offsets, ext, g.offsets, p)
    assert e.value.status == -5
    with pytest.raises(binding.SedefError) as e:
        ctx.sedef_extend(runs, 1, ext, g.offsets, ext, g.offsets, binding.params(), max_len=10)
    assert e.value.status == -1
