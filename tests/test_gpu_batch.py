"""Batched self-search of independent genomes (self_mode 2) against the
oracle and against the one-genome-per-pass form."""
import numpy as np
import pytest

import oracle
from paper_1807_00205_gb300 import batch, binding, synth
from tests.gpu_helpers import assert_rows_equal, cand_rows_global, need_gpu
from tests.test_gpu_parity import full_parity, to_dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    need_gpu()
    c = binding.Context(0)
    yield c
    c.close()


def small_batch(seed, count=9):
    rng = np.random.default_rng(seed)
    out = []
    for g in range(count):
        L = int(rng.integers(3_000, 60_000))
        out.append(synth.small_case(seed * 100 + g, lengths=(L,), n_sd=2, sd_lo=1000,
                                    sd_hi=max(1001, L // 8), id_lo=0.88, mask_frac=0.2))
    return out


def test_batch_matches_oracle_self_mode_2(ctx):
    gs = small_batch(7)
    seq, offs = batch.concatenate(gs)
    g = synth.Genome(seq, offs, [])
    full_parity(ctx, g, oracle.params(self_mode=2))


def test_batched_equals_plain(ctx):
    gs = small_batch(8, count=12)
    seq, offs = batch.concatenate(gs)
    p = binding.params()
    out = batch.batched(ctx, to_dev(seq), offs, p)
    per = batch.split_candidates(binding.struct_view(out["cands"], binding.CAND_DTYPE), len(gs))
    plain = batch.plain(ctx, [to_dev(g.seq) for g in gs], [g.offsets for g in gs], p)
    assert sum(len(x) for x in per) > 0
    for gi, (a, b) in enumerate(zip(per, plain)):
        want = binding.struct_view(b["cands"], binding.CAND_DTYPE)
        assert np.array_equal(a, want), gi
