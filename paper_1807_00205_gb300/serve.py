"""Serving: a resident target index and continuous batching of requests.

The target genome is packed, sketched and indexed once and stays in device
memory.  Requests (query regions) arrive on a host queue.

Served form (batching=True): continuous batching on the device through the
library's server (sedef_server_*).  A persistent filter kernel drains a work
queue of query windows; an admission thread moves waiting requests into free
request slots as slots free up (the slots are sized once, from free device
memory), so a request that arrives while others are on the GPU joins the
running kernel at once.  The kernel keeps the windows with at most 4,096
hits and hands the heavier ones on; a completion thread polls for requests
whose windows are done and passes each to one of five finishing threads,
which run the rest on their own streams (the wide tier over the handed-on
windows, the global path, refine, chaining, merging) while the kernel keeps
filtering the others.

Plain form (batching=False): one request per pass (pack ... merge) on one
worker.  With several workers and batching=False each worker takes every
waiting request (admitted by free memory) into one pass.

Results of a request are the same alone, in a batch and served: every query
window is compared with the whole target independently of the others.
"""
from __future__ import annotations

import collections
import concurrent.futures
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

    @classmethod
    def from_arrays(cls, trec, tsorted, toff, offsets, p: "binding.Params") -> "ResidentIndex":
        """An index already on the device (records by position, records by
        hash, offsets) over sequences at `offsets`."""
        self = cls.__new__(cls)
        self.p_index = binding.params_from_struct(p, self_mode=1)
        self.trec, self.tsorted, self.toff = trec, tsorted, toff
        self.offsets = np.ascontiguousarray(offsets, dtype=np.int64)
        return self

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
    """Serves requests against a resident index: the device work queue
    (batching=True) or host workers (batching=False; see the module notes)."""

    SLOT_BYTES_PER_BASE = 32  # device bytes a request slot holds per query base
    FINISHERS = 5             # sedef_server_finish calls that run at once

    def __init__(self, index: ResidentIndex, p: "binding.Params", workers: int = 2,
                 batching: bool = True, max_batch_bases: int = 64 << 20,
                 reserve_bytes: int = 8 << 30, device: int = 0, free_bytes_fn=None,
                 ctx_factory=None, slots: int = 8, slot_bases: int = 5_000_000,
                 idle_timeout_s: float = 1.0):
        import torch
        self.index = index
        self.p = p
        self.batching = batching
        self.queue = collections.deque()
        self.cv = threading.Condition()
        self.stop = False
        self.completed = []
        self.batches = 0
        if free_bytes_fn is None:
            free_bytes_fn = lambda: torch.cuda.mem_get_info(device)[0]  # noqa: E731
        self.device_queue = batching and ctx_factory is None
        if self.device_queue:
            # admission by free HBM: as many slots as the free memory (less a
            # reserve for the finishing passes) holds, at most `slots`
            per_slot = slot_bases * self.SLOT_BYTES_PER_BASE
            fit = max(1, (free_bytes_fn() - reserve_bytes) // per_slot)
            self.nslots = int(min(slots, fit))
            self.ctx = binding.Context(device)
            self.dev = binding.DeviceServer(self.ctx, index.trec, index.tsorted, index.toff,
                                            index.offsets, p, slots=self.nslots,
                                            slot_bases=slot_bases, idle_timeout_s=idle_timeout_s)
            self.inflight = {}
            self.finishing = concurrent.futures.ThreadPoolExecutor(self.FINISHERS)
            self.threads = [threading.Thread(target=self._admit, daemon=True),
                            threading.Thread(target=self._complete, daemon=True)]
            self.ctxs = [self.ctx]
            # a request longer than a slot goes through one plain pass, with
            # filter tiers that fit beside the persistent kernel
            self.fallback = binding.Context(device, stream=torch.cuda.Stream(device))
            self.fallback.sedef_set_tier_smem_limit(self.dev.smem_left())
            return
        self.admission = Admission(max_batch_bases if batching else 1, reserve_bytes,
                                   free_bytes_fn)
        if ctx_factory is None:
            ctx_factory = lambda: binding.Context(device, stream=torch.cuda.Stream(device))  # noqa: E731
        self.ctxs = [ctx_factory() for _ in range(workers)]
        self.threads = [threading.Thread(target=self._work, args=(c,), daemon=True)
                        for c in self.ctxs]

    def warm(self, seqs: list, autotune: bool = True):
        """Untimed passes over these query sequences.  Host workers first
        pick the filter shape on them against the resident index (autotuner;
        every worker takes the result)."""
        if self.device_queue:
            for q in seqs:
                if len(q) > self.dev.slot_bases:
                    continue
                slot = self.dev.submit(q)
                while slot is None:
                    time.sleep(0.001)
                    slot = self.dev.submit(q)
                done = None
                while done is None:
                    done = self.dev.poll(0.01)
                self.dev.finish(done)
            return
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

    def _done(self, reqs: list):
        now = time.perf_counter()
        with self.cv:
            for r in reqs:
                r.done = now
            self.completed.extend(reqs)
            self.batches += 1

    # -- device work queue ---------------------------------------------------

    def _admit(self):
        """Moves waiting requests into free slots, oldest first."""
        while True:
            with self.cv:
                while not self.queue and not self.stop:
                    self.cv.wait(0.05)
                if self.stop and not self.queue:
                    return
                r = self.queue[0]
            try:
                if len(r.seq) > self.dev.slot_bases:
                    search(self.fallback, self.index, [r], self.p)
                    with self.cv:
                        self.queue.popleft()
                    self._done([r])
                    continue
                slot = self.dev.submit(r.seq)
            except Exception as e:  # the request fails, admission goes on
                r.error = f"{type(e).__name__}: {e}"
                with self.cv:
                    self.queue.popleft()
                self._done([r])
                continue
            if slot is None:  # every slot is busy: wait for one to free up
                time.sleep(0.0002)
                continue
            with self.cv:
                self.queue.popleft()
                self.inflight[slot] = r
                self.cv.notify_all()

    def _complete(self):
        """Finishes every request whose windows the kernel has filtered."""
        while True:
            with self.cv:
                if self.stop and not self.queue and not self.inflight:
                    return
            try:
                slot = self.dev.poll(0.002)
            except Exception as e:
                with self.cv:
                    failed = list(self.inflight.values())
                    self.inflight.clear()
                for r in failed:
                    r.error = f"{type(e).__name__}: {e}"
                self._done(failed)
                continue
            if slot is None:
                continue
            with self.cv:
                # the admission thread records the slot right after submit
                # returns; a short request can be filtered before that
                give_up = time.perf_counter() + 5.0
                while slot not in self.inflight and time.perf_counter() < give_up:
                    self.cv.wait(0.001)
                r = self.inflight.pop(slot, None)
            if r is None:
                self.dev.finish(slot)  # an orphan (cannot happen): free its slot
                continue
            # finishing runs on its own threads (the library runs up to
            # FINISHERS of them at once, each on its own stream), so polling
            # goes on meanwhile
            self.finishing.submit(self._finish_one, slot, r)

    def _finish_one(self, slot: int, r: Request):
        try:
            c = self.dev.finish(slot)
            c["qseq"] = 0
            r.cands = c
        except Exception as e:
            r.error = f"{type(e).__name__}: {e}"
            r.cands = None
        self._done([r])

    # -- host workers ------------------------------------------------------

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
            self._done(reqs)

    def close(self):
        with self.cv:
            self.stop = True
            self.cv.notify_all()
        for t in self.threads:
            if t.is_alive():
                t.join()
        if self.device_queue:
            self.finishing.shutdown(wait=True)
            self.dev.close()
            self.fallback.close()
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
