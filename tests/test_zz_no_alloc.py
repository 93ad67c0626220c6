"""The allocation-free sketch entry point (sedef_sketch_noalloc) against
sedef_sketch, through the C ABI, on two calls in a row.

Callers that cannot allocate device memory (a framework that owns the whole
device heap through its own pool, or a path that must not pay cudaMalloc's
implicit synchronization) use this entry point; its scratch is a fixed static
device array shared by all calls.  This file is collected last on purpose.
"""
import numpy as np
import pytest

from paper_1807_00205_gb300 import binding, synth
from tests.gpu_helpers import need_gpu

pytestmark = pytest.mark.gpu


def test_noalloc_sketch_matches_sketch_twice():
    torch = need_gpu()
    ctx = binding.Context(0)
    stream = torch.cuda.Stream()
    cases = [
        (synth.small_case(101, lengths=(70_000, 9, 33_333, 4_000), n_sd=3, mask_frac=0.3,
                          n_gaps=True), binding.params()),
        (synth.small_case(102, lengths=(150_001,), n_sd=4, mask_frac=0.2, n_gaps=True),
         binding.params(k=11, w=9)),
    ]
    for g, p in cases:  # two calls in a row share (and reuse) the static scratch
        d = torch.from_numpy(g.seq).cuda()
        packed, mask, nbits = ctx.sedef_pack(d)
        want = binding.to_numpy_records(ctx.sedef_sketch(packed, mask, nbits, g.offsets, p))
        torch.cuda.synchronize()
        rec = torch.full((len(want) + 17,), -1, dtype=torch.int64, device="cuda")
        with torch.cuda.stream(stream):
            n = binding.sedef_sketch_noalloc(packed, mask, nbits, g.offsets, p, rec, stream)
        stream.synchronize()
        assert n == len(want)
        assert np.array_equal(binding.to_numpy_records(rec[:n]), want)
    ctx.close()


def test_noalloc_sketch_rejects_oversize_input():
    torch = need_gpu()
    offs = np.arange(4098, dtype=np.int64) * 30  # 4097 sequences: more than the 4096 allowed
    seq = synth.random_bases(np.random.default_rng(3), int(offs[-1]))
    ctx = binding.Context(0)
    packed, mask, nbits = ctx.sedef_pack(torch.from_numpy(seq).cuda())
    rec = torch.empty(1024, dtype=torch.int64, device="cuda")
    with pytest.raises(binding.SedefError) as e:
        binding.sedef_sketch_noalloc(packed, mask, nbits, offs, binding.params(), rec,
                                     torch.cuda.current_stream())
    assert e.value.status == -5
    ctx.close()
