"""Host-side logic of the serving loop (no GPU): admission by free device
memory and the per-batch base budget."""
import collections

import numpy as np

from paper_1807_00205_gb300.serve import BYTES_PER_QUERY_BASE, Admission, Request


def reqs(lengths):
    return collections.deque(Request(rid=k, seq=np.zeros(L, dtype=np.uint8))
                             for k, L in enumerate(lengths))


def test_admission_respects_base_budget():
    adm = Admission(max_batch_bases=100, reserve_bytes=0, free_bytes_fn=lambda: 1 << 40)
    q = reqs([40, 40, 40, 10])
    a = adm.take(q)
    assert [r.rid for r in a] == [0, 1]
    b = adm.take(q)
    assert [r.rid for r in b] == [2, 3]
    assert not q


def test_admission_respects_free_memory_and_releases():
    free = [300 * BYTES_PER_QUERY_BASE]
    adm = Admission(max_batch_bases=10_000, reserve_bytes=100 * BYTES_PER_QUERY_BASE,
                    free_bytes_fn=lambda: free[0])
    q = reqs([150, 100, 10])
    a = adm.take(q)                    # 200 bases of room: only the first fits
    assert [r.rid for r in a] == [0]
    assert adm.take(q) == []           # 50 left after the in-flight 150: wait
    adm.release(a)
    b = adm.take(q)
    assert [r.rid for r in b] == [1, 2]


def test_plain_mode_takes_one_request():
    adm = Admission(max_batch_bases=1, reserve_bytes=0, free_bytes_fn=lambda: 1 << 40)
    q = reqs([5000, 10, 10])
    assert len(adm.take(q)) == 1 and len(adm.take(q)) == 1 and len(adm.take(q)) == 1


def test_failed_batch_does_not_stall_the_server(monkeypatch):
    """A batch whose search raises (an allocation failure, say) marks its
    requests failed; the worker keeps serving and run_load reports the
    failure instead of waiting forever."""
    import pytest

    from paper_1807_00205_gb300 import serve

    class FakeCtx:
        def close(self):
            pass

    def fake_search(ctx, index, reqs, p):
        if any(r.rid == 3 for r in reqs):
            raise MemoryError("device allocation failed")
        for r in reqs:
            r.cands = np.zeros(0)

    monkeypatch.setattr(serve, "search", fake_search)
    srv = serve.Server(None, None, workers=2, batching=False, free_bytes_fn=lambda: 1 << 40,
                       reserve_bytes=0, ctx_factory=FakeCtx)
    srv.start()
    pool = [np.zeros(100, dtype=np.uint8)]
    with pytest.raises(RuntimeError, match="1 requests failed"):
        serve.run_load(srv, pool, rate=5000.0, count=8, seed=1, deadline_s=30)
    assert len(srv.completed) == 8
    assert all(r.cands is not None for r in srv.completed if r.rid != 3)
    srv.close()


def test_run_load_deadline(monkeypatch):
    """A request that never completes ends run_load with a TimeoutError."""
    import pytest

    from paper_1807_00205_gb300 import serve

    class FakeCtx:
        def close(self):
            pass

    srv = serve.Server(None, None, workers=1, batching=False, free_bytes_fn=lambda: 0,
                       reserve_bytes=1, ctx_factory=FakeCtx)  # nothing is ever admitted
    srv.start()
    with pytest.raises(TimeoutError):
        serve.run_load(srv, [np.zeros(10, dtype=np.uint8)], rate=1000.0, count=2, seed=0,
                       deadline_s=0.5)
    with srv.cv:
        srv.queue.clear()
    srv.close()
