"""f2 (Section 3.3, final SDs inside the potential SD regions) through the C
ABI against the CPU oracle: seeds, both chaining tiers and the greedy
extractions must give the oracle's SD rows bit for bit.  Each side grows the
regions with its own extension (equal, as the extension tests show)."""
import numpy as np
import pytest

import oracle
from paper_1807_00205_gb300 import binding, synth
from tests.gpu_helpers import assert_rows_equal, need_gpu
from tests.test_gpu_extend import gpu_extend, region_rows, to_dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    need_gpu()
    c = binding.Context(0)
    yield c
    c.close()


def sd_rows(t) -> np.ndarray:
    r = binding.struct_view(t, binding.SD_DTYPE)
    if len(r) == 0:
        return np.zeros((0, len(oracle.CHAIN2_COLS)), dtype=np.int64)
    return np.stack([r[c].astype(np.int64) for c in oracle.CHAIN2_COLS], axis=1)


def both(ctx, g, pd, threads=16):
    recs = oracle.sketch(g.seq, g.offsets, pd)
    runs = oracle.filter_runs(recs, g.offsets, recs, g.offsets, pd, threads=threads)
    allk = oracle.sketch(g.seq, g.offsets, dict(pd, min_unmasked=0))
    ext = oracle.extend(runs, allk, g.offsets, allk, g.offsets, pd, threads=threads)
    want = oracle.chain2(g.seq, ext, threads=threads)
    # the GPU: its own regions (checked equal to the oracle's), then chain2
    p = binding.params_from_dict(pd)
    got_regions, _ = gpu_extend(ctx, g, pd, oracle.MAX_SD_LENGTH)
    assert_rows_equal(got_regions, ext, "regions")
    v = np.zeros(len(got_regions), dtype=binding.REGION_DTYPE)
    for c in oracle.EXTEND_COLS:
        v[c] = got_regions[:, oracle.EXTEND_COLS.index(c)]
    packed, _, nbits = ctx.sedef_pack(to_dev(g.seq))
    out, n = ctx.sedef_chain2(packed, nbits, g.length, to_dev(v.view(np.uint8)), len(v), p)
    return sd_rows(out), want


def test_chain2_planted_duplications(ctx):
    """A 400 kbp genome with eight planted duplications (2-8 kbp, 90-99.5%
    identity, both strands)."""
    g = synth.small_case(41, lengths=(400_000,), n_sd=8, sd_lo=2000, sd_hi=8000,
                         id_lo=0.90, id_hi=0.995)
    got, want = both(ctx, g, oracle.params())
    assert len(want) >= 8
    assert_rows_equal(got, want, "SDs")


def test_chain2_masked_multi_sequence(ctx):
    """Soft-masked repeats (read as bases here), N runs, several sequences
    and inter-sequence duplications."""
    g = synth.small_case(52, lengths=(150_000, 90_000), n_sd=6, sd_lo=1500, sd_hi=9000,
                         id_lo=0.85, mask_frac=0.25, n_gaps=True, inter_frac=0.5)
    got, want = both(ctx, g, oracle.params())
    assert len(want) > 0
    assert_rows_equal(got, want, "SDs")


def test_chain2_plain_2mbp(ctx):
    """Every potential SD region of the 2 Mbp workload."""
    got, want = both(ctx, synth.plain_2mbp(), oracle.params())
    assert len(want) >= 20
    assert_rows_equal(got, want, "SDs")
