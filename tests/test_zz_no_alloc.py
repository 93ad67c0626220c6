"""The allocation-free sketch entry point (sedef_sketch_noalloc) through the
C ABI, on two calls in a row: against sedef_sketch and against the CPU
oracle's sketch.

Callers that cannot allocate device memory (a framework that owns the whole
device heap through its own pool, or a path that must not pay cudaMalloc's
implicit synchronization) use this entry point; its scratch is a fixed static
device array shared by all calls.  The file name sorts last, so a run that
stops at its first failure has run every other test before this one; the
checks do not depend on that order, and one of them repeats the two calls in
a fresh process.
"""
import os
import subprocess
import sys

import numpy as np
import pytest

import oracle
from paper_1807_00205_gb300 import binding, synth
from tests.gpu_helpers import need_gpu

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _cases():
    return [
        (synth.small_case(101, lengths=(70_000, 9, 33_333, 4_000), n_sd=3, mask_frac=0.3,
                          n_gaps=True), {}),
        (synth.small_case(102, lengths=(150_001,), n_sd=4, mask_frac=0.2, n_gaps=True),
         dict(k=11, w=9)),
    ]


def two_calls_in_a_row(check_oracle: bool) -> int:
    """Each case through sedef_sketch (context scratch) and then through
    sedef_sketch_noalloc (the static array, reused by the second call):
    records must be identical, and the first case's must equal the oracle's
    rows.  Returns the number of cases checked."""
    import torch
    ctx = binding.Context(0)
    stream = torch.cuda.Stream()
    done = 0
    for c, (g, kw) in enumerate(_cases()):
        p = binding.params(**kw)
        d = torch.from_numpy(g.seq).cuda()
        packed, mask, nbits = ctx.sedef_pack(d)
        want = binding.to_numpy_records(ctx.sedef_sketch(packed, mask, nbits, g.offsets, p))
        torch.cuda.synchronize()
        rec = torch.full((len(want) + 17,), -1, dtype=torch.int64, device="cuda")
        with torch.cuda.stream(stream):
            n = binding.sedef_sketch_noalloc(packed, mask, nbits, g.offsets, p, rec, stream)
        stream.synchronize()
        assert n == len(want)
        got = binding.to_numpy_records(rec[:n])
        assert np.array_equal(got, want)
        if check_oracle and c == 0:
            rows = oracle.sketch(g.seq, g.offsets, oracle.params(**kw))
            assert np.array_equal(binding.records_to_rows(got), rows)
        done += 1
    ctx.close()
    return done


def test_noalloc_sketch_matches_sketch_and_oracle_twice():
    need_gpu()
    assert two_calls_in_a_row(check_oracle=True) == 2


def test_noalloc_sketch_in_a_fresh_process():
    """The same two calls as the first thing a new process does on the GPU."""
    need_gpu()
    code = ("import sys; sys.path.insert(0, %r); "
            "from tests.test_zz_no_alloc import two_calls_in_a_row; "
            "print('cases', two_calls_in_a_row(False))" % ROOT)
    r = subprocess.run([sys.executable, "-c", code], cwd=ROOT, capture_output=True, text=True,
                       timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    assert "cases 2" in r.stdout


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
