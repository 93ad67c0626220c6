"""Serving: a resident target index and a continuously batched request loop.

The target genome is packed, sketched and indexed once and stays in device
memory.  Requests (query regions) arrive on a host queue.  Each worker -- a
host thread with its own library context and CUDA stream -- repeatedly takes
every request that is waiting (up to a base budget, and only while the
admission controller finds room in device memory), runs pack, sketch,
filter, refine, chain and merge for them in one pass against the resident
index (non-self mode, one query sequence per request), and splits the
candidates back by request.  Requests that arrive while a batch is on the
GPU are admitted to the next free worker, so batches of different workers
overlap on the device.  The plain form runs one request per pass on one
worker.

Results of a request are the same alone and in a batch: every query window
is compared with the whole target independently of the other sequences.
"""
from __future__ import annotations

import collections
import dataclasses
import threading
import time

import numpy as np

from . import binding

BYTES_PER_QUERY_BASE = 64  # device bytes a request needs per query base (estimate)


@dataclasses.dataclass
class Request:
    rid: int
    seq: np.ndarray          # uint8 ASCII query region
    arrival: float = 0.0     # perf_counter() time it entered the queue
    done: float = 0.0
    cands: np.ndarray = None  # sedef_cand_t rows (qseq = 0)
    error: str = ""          # set when the request's batch failed


class Admission:
    """Admits a batch while its estimated device bytes fit in the free device
    memory minus a reserve (and under a cap on query bases per batch)."""

    def __init__(self, max_batch_bases: int, reserve_bytes: int, free_bytes_fn):
        self.max_batch_bases = max_batch_bases
        self.reserve_bytes = reserve_bytes
        self.free_bytes_fn = free_bytes_fn
        self.lock = threading.Lock()
        self.in_flight = 0  # bytes admitted and not yet released

    def take(self, queue: collections.deque) -> list:
        """Pops the longest admissible prefix of the queue (at least one
        request when the queue is non-empty and it fits alone)."""
        with self.lock:
            budget = self.free_bytes_fn() - self.reserve_bytes - self.in_flight
            out, bases = [], 0
            while queue:
                r = queue[0]
                need = len(r.seq) * BYTES_PER_QUERY_BASE
                if out and (bases + len(r.seq) > self.max_batch_bases or need > budget):
                    break
                if not out and need > budget:
                    break  # wait for memory to free up
                queue.popleft()
                out.append(r)
                bases += len(r.seq)
                budget -= need
            self.in_flight += bases * BYTES_PER_QUERY_BASE
            return out

    def release(self, reqs: list):
        with self.lock:
            self.in_flight -= sum(len(r.seq) for r in reqs) * BYTES_PER_QUERY_BASE


class ResidentIndex:
    """The target genome's records and index, kept on the device.  Built
    from the sequence, or restored from a blob written by `save` (a serving
    process restarts without re-indexing)."""

    def __init__(self, ctx: "binding.Context", seq: np.ndarray, offsets, p: "binding.Params",
                 blob: bytes = None):
        import torch
        self.p_index = binding.params_from_struct(p, self_mode=1)
        if blob is not None:
            self.trec, self.tsorted, self.toff, self.offsets, k = ctx.sedef_index_load(blob)
            if k != p.k:
                raise ValueError(f"index blob has k={k}, parameters have k={p.k}")
        else:
            self.offsets = np.ascontiguousarray(offsets, dtype=np.int64)
            d = torch.from_numpy(np.ascontiguousarray(seq)).to(ctx.device)
            packed, mask, nbits = ctx.sedef_pack(d)
            self.trec = ctx.sedef_sketch(packed, mask, nbits, self.offsets, self.p_index)
            self.tsorted, self.toff = ctx.sedef_index(self.trec, self.p_index)
        torch.cuda.synchronize(ctx.device)

    def save(self, ctx: "binding.Context") -> bytes:
        return ctx.sedef_index_save(self.trec, self.tsorted, self.toff, self.p_index.k,
                                    self.offsets)


def search(ctx: "binding.Context", index: ResidentIndex, reqs: list, p: "binding.Params"):
    """One pass for a batch of requests; fills each request's candidates."""
    import torch
    q = binding.params_from_struct(p, self_mode=0)
    parts = [r.seq for r in reqs]
    offs = np.zeros(len(parts) + 1, dtype=np.int64)
    offs[1:] = np.cumsum([len(x) for x in parts])
    seq = np.concatenate(parts)
    with torch.cuda.stream(ctx.stream):
        d = torch.from_numpy(seq).to(ctx.device, non_blocking=False)
        packed, mask, nbits = ctx.sedef_pack(d)
        qrec = ctx.sedef_sketch(packed, mask, nbits, offs, q)
        runs, nr = ctx.sedef_filter(qrec, offs, index.trec, index.tsorted, index.toff,
                                    index.offsets, q)
        chains, nc = ctx.sedef_chain(runs, nr, qrec, offs, index.tsorted, index.toff,
                                     index.offsets, q)
        cands, _ = ctx.sedef_merge(chains, nc, offs, index.offsets, q)
        rows = binding.struct_view(cands, binding.CAND_DTYPE)
    for k, r in enumerate(reqs):
        c = rows[rows["qseq"] == k].copy()
        c["qseq"] = 0
        r.cands = c


class Server:
    """Continuous batching over `workers` host threads (each its own stream)."""

    def __init__(self, index: ResidentIndex, p: "binding.Params", workers: int = 2,
                 batching: bool = True, max_batch_bases: int = 64 << 20,
                 reserve_bytes: int = 8 << 30, device: int = 0, free_bytes_fn=None,
                 ctx_factory=None):
        import torch
        self.index = index
        self.p = p
        self.batching = batching
        self.queue = collections.deque()
        self.cv = threading.Condition()
        self.stop = False
        self.completed = []
        if free_bytes_fn is None:
            free_bytes_fn = lambda: torch.cuda.mem_get_info(device)[0]  # noqa: E731
        self.admission = Admission(max_batch_bases if batching else 1, reserve_bytes,
                                   free_bytes_fn)
        if ctx_factory is None:
            ctx_factory = lambda: binding.Context(device, stream=torch.cuda.Stream(device))  # noqa: E731
        self.ctxs = [ctx_factory() for _ in range(workers)]
        self.threads = [threading.Thread(target=self._work, args=(c,), daemon=True)
                        for c in self.ctxs]
        self.batches = 0

    def warm(self, seqs: list, autotune: bool = True):
        """Picks the filter shape on these query sequences against the
        resident index (autotuner, first worker's context; every worker takes
        the result), then one untimed pass per worker over them."""
        if autotune and seqs:
            import torch
            c0 = self.ctxs[0]
            q = binding.params_from_struct(self.p, self_mode=0)
            offs = np.zeros(len(seqs) + 1, dtype=np.int64)
            offs[1:] = np.cumsum([len(x) for x in seqs])
            with torch.cuda.stream(c0.stream):
                d = torch.from_numpy(np.concatenate(seqs)).to(c0.device)
                packed, mask, nbits = c0.sedef_pack(d)
                qrec = c0.sedef_sketch(packed, mask, nbits, offs, q)
                v = c0.sedef_filter_autotune(qrec, offs, self.index.trec, self.index.tsorted,
                                             self.index.toff, self.index.offsets, q)
            for c in self.ctxs:
                c.sedef_filter_variant(v)
        for c in self.ctxs:
            search(c, self.index, [Request(rid=-1, seq=q) for q in seqs], self.p)

    def start(self):
        for t in self.threads:
            t.start()

    def submit(self, r: Request):
        r.arrival = time.perf_counter()
        with self.cv:
            self.queue.append(r)
            self.cv.notify()

    def _work(self, ctx):
        while True:
            with self.cv:
                while not self.queue and not self.stop:
                    self.cv.wait(0.05)
                if self.stop and not self.queue:
                    return
                reqs = self.admission.take(self.queue)
            if not reqs:
                time.sleep(0.001)
                continue
            try:
                search(ctx, self.index, reqs, self.p)
            except Exception as e:  # the batch fails, the worker goes on
                for r in reqs:
                    r.error = f"{type(e).__name__}: {e}"
                    r.cands = None
            finally:
                self.admission.release(reqs)
            now = time.perf_counter()
            with self.cv:
                for r in reqs:
                    r.done = now
                self.completed.extend(reqs)
                self.batches += 1

    def close(self):
        with self.cv:
            self.stop = True
            self.cv.notify_all()
        for t in self.threads:
            if t.is_alive():
                t.join()
        for c in self.ctxs:
            c.close()


def run_load(server: Server, pool: list, rate: float, count: int, seed: int = 0,
             deadline_s: float = 600.0) -> dict:
    """Submits `count` requests (cycling through `pool`) at Poisson arrivals
    of `rate` per second; returns latency percentiles and throughput.
    Raises TimeoutError when the requests have not all completed
    `deadline_s` seconds after the last submission, and RuntimeError when a
    request failed."""
    rng = np.random.default_rng(seed)
    gaps = rng.exponential(1.0 / rate, size=count)
    with server.cv:
        server.completed = []
        server.batches = 0
    t0 = time.perf_counter()
    due = t0
    reqs = []
    for k in range(count):
        due += gaps[k]
        wait = due - time.perf_counter()
        if wait > 0:
            time.sleep(wait)
        r = Request(rid=k, seq=pool[k % len(pool)])
        reqs.append(r)
        server.submit(r)
    give_up = time.perf_counter() + deadline_s
    while True:
        with server.cv:
            if len(server.completed) >= count:
                break
        if time.perf_counter() > give_up:
            raise TimeoutError(f"{count - len(server.completed)} of {count} requests "
                               f"still pending after {deadline_s} s")
        time.sleep(0.001)
    failed = [r for r in reqs if r.error]
    if failed:
        raise RuntimeError(f"{len(failed)} requests failed; first: {failed[0].error}")
    t1 = max(r.done for r in reqs)
    lat = np.array([r.done - r.arrival for r in reqs]) * 1000.0
    bases = sum(len(r.seq) for r in reqs)
    return {"rate": rate, "requests": count, "p50_ms": float(np.percentile(lat, 50)),
            "p99_ms": float(np.percentile(lat, 99)), "mean_ms": float(lat.mean()),
            "mbp_s": bases / (t1 - t0) / 1e6, "offered_mbp_s": bases / (due - t0) / 1e6,
            "batches": server.batches}
