"""Failure handling through the C ABI, with no GPU fault: bad arguments are
refused before any kernel runs, allocation failures come back as
SEDEF_ERR_OOM from every call that allocates, and the context stays usable
after both."""
import ctypes

import numpy as np
import pytest

import oracle
from paper_1807_00205_gb300 import binding, synth
from tests.gpu_helpers import assert_rows_equal, cand_rows_global, need_gpu

pytestmark = pytest.mark.gpu

INVALID, OOM, UNSUPPORTED = -1, -2, -5


@pytest.fixture(scope="module")
def small():
    torch = need_gpu()
    g = synth.small_case(17, lengths=(60_000, 25_000), n_sd=4, sd_lo=1500, sd_hi=5000,
                         id_lo=0.88, mask_frac=0.2, n_gaps=True)
    ctx = binding.Context(0)
    p = binding.params()
    d = torch.from_numpy(g.seq).cuda()
    out = ctx.selfsearch(d, g.offsets, p)
    torch.cuda.synchronize()
    yield g, ctx, p, d, out
    ctx.close()


def test_bad_arguments_launch_nothing(small):
    """Decreasing or shifted offsets, NULL buffers, parameters out of range
    and mismatched self-search arrays are refused (INVALID or UNSUPPORTED)
    without a single kernel launch."""
    g, ctx, p, d, out = small
    lib, h = ctx.lib, ctx.handle
    n64 = ctypes.c_int64()
    ptr = binding._ptr
    good = np.ascontiguousarray(g.offsets, dtype=np.int64)
    shifted = good.copy()
    shifted[0] = 5
    decreasing = good.copy()
    decreasing[1] = good[2] + 1
    rec, srt, off, runs = out["rec"], out["sorted"], out["off"], out["runs"]
    nr, nrec = out["nruns"], rec.numel()

    def par(**kw):
        q = binding.params_from_struct(p)
        for k, v in kw.items():
            setattr(q, k, v)
        return ctypes.byref(q)

    bad_params = [par(k=16), par(k=1), par(w=0), par(w=300), par(n=10), par(n=2000),
                  par(query_step=0), par(self_mode=3), par(delta_g=1.5), par(max_occ=-1)]
    calls = []
    for P in bad_params:
        calls.append(lambda P=P: lib.sedef_sketch(h, ptr(out["packed"]), ptr(out["mask"]),
                                                  ptr(out["nbits"]), good.ctypes.data,
                                                  len(good) - 1, P, ptr(rec), nrec,
                                                  ctypes.byref(n64)))
        calls.append(lambda P=P: lib.sedef_filter(h, ptr(rec), nrec, good.ctypes.data,
                                                  len(good) - 1, ptr(rec), ptr(srt), ptr(off),
                                                  nrec, good.ctypes.data, len(good) - 1, P,
                                                  ptr(runs), nr, ctypes.byref(n64)))
    P = ctypes.byref(p)
    for o in (shifted, decreasing):
        calls.append(lambda o=o: lib.sedef_sketch(h, ptr(out["packed"]), ptr(out["mask"]),
                                                  ptr(out["nbits"]), o.ctypes.data, len(o) - 1, P,
                                                  ptr(rec), nrec, ctypes.byref(n64)))
        calls.append(lambda o=o: lib.sedef_chain(h, ptr(runs), nr, ptr(rec), nrec, o.ctypes.data,
                                                 len(o) - 1, ptr(srt), ptr(off), nrec,
                                                 good.ctypes.data, len(good) - 1, P, ptr(runs), 1,
                                                 ctypes.byref(n64)))
        calls.append(lambda o=o: lib.sedef_selfsearch(h, ptr(d), o.ctypes.data, len(o) - 1, P,
                                                      None, 0, ctypes.byref(n64)))
    calls += [
        lambda: lib.sedef_pack(h, None, 100, ptr(out["packed"]), ptr(out["mask"]),
                               ptr(out["nbits"])),
        lambda: lib.sedef_pack(h, ptr(d), -1, ptr(out["packed"]), ptr(out["mask"]),
                               ptr(out["nbits"])),
        lambda: lib.sedef_index(h, ptr(rec), nrec, P, ptr(rec), ptr(off)),  # in place
        lambda: lib.sedef_index(h, ptr(rec), nrec, P, None, ptr(off)),
        # self mode with a query that is not the target
        lambda: lib.sedef_filter(h, ptr(rec), nrec - 1, good.ctypes.data, len(good) - 1, ptr(rec),
                                 ptr(srt), ptr(off), nrec, good.ctypes.data, len(good) - 1, P,
                                 ptr(runs), nr, ctypes.byref(n64)),
        lambda: lib.sedef_filter(h, ptr(rec), nrec, good.ctypes.data, len(good) - 1, ptr(rec),
                                 ptr(srt), ptr(off), nrec, good.ctypes.data, len(good) - 1, P,
                                 None, 5, ctypes.byref(n64)),
        lambda: lib.sedef_merge(h, None, 3, good.ctypes.data, len(good) - 1, good.ctypes.data,
                                len(good) - 1, P, None, 0, ctypes.byref(n64)),
        lambda: lib.sedef_extend(h, ptr(runs), nr, ptr(rec), nrec, good.ctypes.data, len(good) - 1,
                                 ptr(rec), nrec, good.ctypes.data, len(good) - 1, P, 10, None, 0,
                                 ctypes.byref(n64)),
        lambda: lib.sedef_qgram(h, ptr(out["packed"]), ptr(out["nbits"]), g.length, ptr(runs), nr,
                                P, 9, 0.005, None, None, ctypes.byref(n64)),
        lambda: lib.sedef_set_scratch_limit(None, 0),
        lambda: lib.sedef_filter_variant(h, 10_000, None, None),
    ]
    before = binding.Context.sedef_launch_count()
    for k, call in enumerate(calls):
        st = call()
        assert st in (INVALID, UNSUPPORTED), (k, st, lib.sedef_last_error())
    assert binding.Context.sedef_launch_count() == before
    # the context still works
    again = ctx.selfsearch(d, g.offsets, p)
    assert again["ncands"] == out["ncands"]


def test_allocation_failures_return_oom_and_leave_the_context_usable(small):
    """With the context's scratch capped at zero, every call that needs
    scratch returns SEDEF_ERR_OOM; with the cap lifted the same context gives
    the oracle's candidates."""
    g, _, p, d, out = small
    torch = need_gpu()
    ctx = binding.Context(0)
    ctx.sedef_set_scratch_limit(0)
    rec, srt, off, runs, nr = out["rec"], out["sorted"], out["off"], out["runs"], out["nruns"]
    ext = out["rec"]  # any records sorted by position will do: the call stops first
    attempts = {
        "sketch": lambda: ctx.sedef_sketch(out["packed"], out["mask"], out["nbits"], g.offsets, p),
        "index": lambda: ctx.sedef_index(rec, p),
        "filter": lambda: ctx.sedef_filter(rec, g.offsets, rec, srt, off, g.offsets, p),
        "chain": lambda: ctx.sedef_chain(runs, nr, rec, g.offsets, srt, off, g.offsets, p),
        "merge": lambda: ctx.sedef_merge(out["chains"], out["nchains"], g.offsets, g.offsets, p),
        "extend": lambda: ctx.sedef_extend(runs, nr, ext, g.offsets, ext, g.offsets, p),
        "selfsearch": lambda: ctx.sedef_selfsearch(d, g.offsets, p),
        "selfsearch_host": lambda: ctx.sedef_selfsearch_host(g.seq, g.offsets, p),
        "graph": lambda: binding.Graph(ctx, d, g.offsets, p, binding.default_caps(g.length)),
    }
    for name, call in attempts.items():
        try:
            call()
        except binding.SedefError as e:
            assert e.status == OOM, (name, e)
        else:
            raise AssertionError(f"{name} ran with no scratch memory")
    ctx.sedef_set_scratch_limit(-1)
    torch.cuda.synchronize()
    want = oracle.selfsearch(g.seq, g.offsets, oracle.params())["cands"]
    cands, nc = ctx.sedef_selfsearch(d, g.offsets, p)
    assert_rows_equal(cand_rows_global(cands, g.offsets), want, "candidates after OOM")
    ctx.close()
