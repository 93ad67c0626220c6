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
