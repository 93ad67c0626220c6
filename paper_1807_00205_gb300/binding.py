"""Thin ctypes binding of libsedef (include/sedef.h).

Argument marshalling only: torch allocates device buffers and provides the
stream; every step of the seeding filter runs in the library's CUDA kernels.
There is no fallback: if the library cannot be loaded, the calls raise.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

SEDEF_OK = 0
SEDEF_ERR_CAPACITY = -6

RUN_DTYPE = np.dtype([("i", "<u4"), ("j_a", "<u4"), ("j_b", "<u4"), ("j_at_max", "<u4"),
                      ("j_star", "<u4"), ("s", "<u2"), ("m", "<u2"), ("max_shared", "<u2"),
                      ("est", "<u2"), ("den", "<u2"), ("o", "u1"), ("keep", "u1")])
CHAIN_DTYPE = np.dtype([("i", "<u4"), ("qseq", "<u4"), ("q0", "<u4"), ("q1", "<u4"),
                        ("tseq", "<u4"), ("t0", "<u4"), ("t1", "<u4"), ("score", "<u2"),
                        ("s", "<u2"), ("o", "<u4"), ("reserved", "<u4")])
REGION_DTYPE = np.dtype([("i", "<u4"), ("j_star", "<u4"), ("qa", "<u4"), ("qb", "<u4"),
                         ("ta", "<u4"), ("tb", "<u4"), ("est", "<u4"), ("den", "<u4"),
                         ("o", "<u4"), ("reserved", "<u4")])
SD_DTYPE = np.dtype([("region", "<u4"), ("o", "<u4"), ("q0", "<u4"), ("q1", "<u4"),
                     ("t0", "<u4"), ("t1", "<u4"), ("score", "<u4"), ("seeds", "<u4"),
                     ("parts", "<u4"), ("reserved", "<u4")])
CAND_DTYPE = np.dtype([("qseq", "<u4"), ("q0", "<u4"), ("q1", "<u4"), ("tseq", "<u4"),
                       ("t0", "<u4"), ("t1", "<u4"), ("o", "<u4"), ("score", "<u4"),
                       ("nchains", "<u4"), ("reserved", "<u4")])
assert RUN_DTYPE.itemsize == 32 and CHAIN_DTYPE.itemsize == 40 and CAND_DTYPE.itemsize == 40
assert REGION_DTYPE.itemsize == 40


class Params(ctypes.Structure):
    _fields_ = [("k", ctypes.c_int32), ("w", ctypes.c_int32), ("n", ctypes.c_int32),
                ("query_step", ctypes.c_int32), ("max_occ", ctypes.c_int32),
                ("self_mode", ctypes.c_int32), ("gap_max", ctypes.c_int32),
                ("diag_max", ctypes.c_int32), ("min_unmasked", ctypes.c_int32),
                ("reserved", ctypes.c_int32), ("delta_m", ctypes.c_double),
                ("delta_g", ctypes.c_double)]


EXPORTS = ["sedef_default_params", "sedef_last_error", "sedef_create", "sedef_destroy",
           "sedef_set_stream", "sedef_set_scratch_limit", "sedef_set_tier_smem_limit",
           "sedef_trace_enable", "sedef_trace_report", "sedef_launch_count", "sedef_filter_stats",
           "sedef_threshold_table", "sedef_pack", "sedef_sketch", "sedef_sketch_noalloc",
           "sedef_index", "sedef_filter", "sedef_filter_autotune", "sedef_filter_variant",
           "sedef_chain", "sedef_extend", "sedef_chain2", "sedef_merge", "sedef_selfsearch",
           "sedef_selfsearch_host",
           "sedef_index_blob_size",
           "sedef_index_save", "sedef_index_blob_info", "sedef_index_load", "sedef_graph_create",
           "sedef_graph_launch", "sedef_graph_wait", "sedef_graph_nodes", "sedef_graph_destroy",
           "sedef_qgram", "sedef_server_create", "sedef_server_submit", "sedef_server_poll",
           "sedef_server_finish", "sedef_server_status", "sedef_server_smem_left",
           "sedef_server_destroy"]

CAP_NAMES = ["records", "slow_hits", "runs", "anchors", "chains", "cands"]


class GraphCaps(ctypes.Structure):
    _fields_ = [(n, ctypes.c_int64) for n in CAP_NAMES]

_lib = None


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Loads libsedef.so (building it first when allowed)."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.LIB
    if build_if_missing:
        path = _build.build()
    if not os.path.exists(path):
        raise RuntimeError(f"libsedef not built: {path} is missing")
    lib = ctypes.CDLL(path)
    vp, i32, i64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64
    P = ctypes.POINTER(Params)
    lib.sedef_default_params.argtypes = [P]
    lib.sedef_last_error.restype = ctypes.c_char_p
    lib.sedef_create.argtypes = [ctypes.c_int, vp, ctypes.POINTER(vp)]
    lib.sedef_destroy.argtypes = [vp]
    lib.sedef_set_stream.argtypes = [vp, vp]
    lib.sedef_set_scratch_limit.argtypes = [vp, i64]
    lib.sedef_set_tier_smem_limit.argtypes = [vp, i64]
    lib.sedef_threshold_table.argtypes = [P, vp, i32, ctypes.POINTER(ctypes.c_double)]
    lib.sedef_pack.argtypes = [vp, vp, i64, vp, vp, vp]
    lib.sedef_sketch.argtypes = [vp, vp, vp, vp, vp, i32, P, vp, i64, ctypes.POINTER(i64)]
    lib.sedef_sketch_noalloc.argtypes = [vp, vp, vp, vp, i32, P, vp, i64, ctypes.POINTER(i64), vp]
    lib.sedef_index.argtypes = [vp, vp, i64, P, vp, vp]
    lib.sedef_filter.argtypes = [vp, vp, i64, vp, i32, vp, vp, vp, i64, vp, i32, P, vp, i64,
                                 ctypes.POINTER(i64)]
    lib.sedef_filter_autotune.argtypes = [vp, vp, i64, vp, i32, vp, vp, vp, i64, vp, i32, P,
                                          ctypes.POINTER(i32)]
    lib.sedef_filter_variant.argtypes = [vp, i32, ctypes.POINTER(i32), ctypes.POINTER(i32)]
    lib.sedef_index_blob_size.restype = i64
    lib.sedef_index_blob_size.argtypes = [i32, i64, i32]
    lib.sedef_index_save.argtypes = [vp, vp, vp, vp, i64, i32, vp, i32, vp, i64]
    lib.sedef_index_blob_info.argtypes = [vp, i64, ctypes.POINTER(i32), ctypes.POINTER(i64),
                                          ctypes.POINTER(i32)]
    lib.sedef_index_load.argtypes = [vp, vp, i64, vp, i32, vp, vp, vp, i64]
    lib.sedef_graph_create.argtypes = [vp, vp, vp, i32, P, ctypes.POINTER(GraphCaps), vp, vp, vp,
                                       vp, vp, vp, ctypes.POINTER(vp)]
    lib.sedef_qgram.argtypes = [vp, vp, vp, i64, vp, i64, P, i32, ctypes.c_double, vp, vp,
                                ctypes.POINTER(i64)]
    lib.sedef_graph_launch.argtypes = [vp, vp]
    lib.sedef_graph_wait.argtypes = [vp, vp]
    lib.sedef_graph_nodes.restype = i64
    lib.sedef_graph_nodes.argtypes = [vp]
    lib.sedef_graph_destroy.argtypes = [vp]
    lib.sedef_chain.argtypes = [vp, vp, i64, vp, i64, vp, i32, vp, vp, i64, vp, i32, P, vp, i64,
                                ctypes.POINTER(i64)]
    lib.sedef_merge.argtypes = [vp, vp, i64, vp, i32, vp, i32, P, vp, i64, ctypes.POINTER(i64)]
    lib.sedef_extend.argtypes = [vp, vp, i64, vp, i64, vp, i32, vp, i64, vp, i32, P, i64, vp, i64,
                                 ctypes.POINTER(i64)]
    lib.sedef_chain2.argtypes = [vp, vp, vp, i64, vp, i64, P, vp, i64, ctypes.POINTER(i64)]
    lib.sedef_selfsearch.argtypes = [vp, vp, vp, i32, P, vp, i64, ctypes.POINTER(i64)]
    lib.sedef_selfsearch_host.argtypes = [vp, vp, vp, i32, P, vp, i64, ctypes.POINTER(i64)]
    lib.sedef_server_create.argtypes = [vp, vp, vp, vp, i64, vp, i32, P, i32, i64,
                                        ctypes.c_double, ctypes.POINTER(vp)]
    lib.sedef_server_submit.argtypes = [vp, vp, i64, ctypes.POINTER(i32)]
    lib.sedef_server_poll.argtypes = [vp, ctypes.c_double, ctypes.POINTER(i32)]
    lib.sedef_server_finish.argtypes = [vp, i32, vp, i64, ctypes.POINTER(i64)]
    lib.sedef_server_status.argtypes = [vp, ctypes.POINTER(i32), ctypes.POINTER(i32)]
    lib.sedef_server_smem_left.argtypes = [vp, ctypes.POINTER(i64)]
    lib.sedef_server_destroy.argtypes = [vp]
    lib.sedef_trace_enable.argtypes = [vp, ctypes.c_int]
    lib.sedef_trace_report.argtypes = [vp, ctypes.c_char_p, i64, ctypes.c_int]
    lib.sedef_launch_count.restype = ctypes.c_uint64
    lib.sedef_launch_count.argtypes = []
    lib.sedef_filter_stats.argtypes = [vp, vp, i32]
    for name in EXPORTS:
        if name not in ("sedef_default_params", "sedef_last_error", "sedef_launch_count",
                        "sedef_index_blob_size", "sedef_graph_nodes"):
            getattr(lib, name).restype = ctypes.c_int
    _lib = lib
    return lib


class SedefError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"libsedef status {status}: {msg}")
        self.status = status


def _check(status: int):
    if status != SEDEF_OK:
        raise SedefError(status, load().sedef_last_error().decode())


def params(**kw) -> Params:
    p = Params()
    load().sedef_default_params(ctypes.byref(p))
    for key, v in kw.items():
        if key == "step":
            key = "query_step"
        setattr(p, key, v)
    return p


def params_from_dict(d: dict) -> Params:
    keys = {"k", "w", "n", "step", "max_occ", "self_mode", "gap_max", "diag_max",
            "min_unmasked", "delta_m", "delta_g"}
    return params(**{k: v for k, v in d.items() if k in keys})


def params_from_struct(p: Params, **kw) -> Params:
    """A copy of p with some fields replaced."""
    q = Params()
    ctypes.pointer(q)[0] = p
    for key, v in kw.items():
        setattr(q, "query_step" if key == "step" else key, v)
    return q


def _ptr(t) -> int:
    if t is None:
        return None
    if isinstance(t, np.ndarray):
        return t.ctypes.data
    return t.data_ptr()


def _offsets(off) -> np.ndarray:
    return np.ascontiguousarray(off, dtype=np.int64)


class Context:
    """A libsedef context bound to one device and one CUDA stream."""

    def __init__(self, device: int = 0, stream=None):
        import torch
        self.torch = torch
        self.lib = load()
        self.device = torch.device("cuda", device)
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        h = ctypes.c_void_p()
        _check(self.lib.sedef_create(device, ctypes.c_void_p(self.stream.cuda_stream),
                                     ctypes.byref(h)))
        self.handle = h
        self._run_cap = 0   # largest run count seen (first run-buffer size next time)
        self._cand_cap = 0

    def close(self):
        if self.handle:
            self.lib.sedef_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _empty(self, n, dtype):
        return self.torch.empty(max(int(n), 1), dtype=dtype, device=self.device)

    def sedef_set_scratch_limit(self, nbytes: int):
        """Caps the context's device scratch (< 0: no cap)."""
        _check(self.lib.sedef_set_scratch_limit(self.handle, int(nbytes)))

    def sedef_set_tier_smem_limit(self, nbytes: int):
        """Caps the shared memory per CTA of the filter tiers (< 0: no cap)."""
        _check(self.lib.sedef_set_tier_smem_limit(self.handle, int(nbytes)))

    # -- tracing ----------------------------------------------------------------

    def sedef_trace_enable(self, on: bool = True):
        _check(self.lib.sedef_trace_enable(self.handle, 1 if on else 0))

    def sedef_trace_report(self, reset: bool = True) -> dict:
        """{kernel name: (launches, total ms)} since the last reset."""
        n = self.lib.sedef_trace_report(self.handle, None, 0, 0)
        if n < 0:
            _check(n)
        buf = ctypes.create_string_buffer(n + 1)
        self.lib.sedef_trace_report(self.handle, buf, n + 1, 1 if reset else 0)
        out = {}
        for line in buf.value.decode().splitlines():
            name, cnt, ms = line.split()
            out[name] = (int(cnt), float(ms))
        return out

    def sedef_filter_stats(self) -> dict:
        v = np.zeros(8, dtype=np.int64)
        _check(self.lib.sedef_filter_stats(self.handle, v.ctypes.data, 8))
        keys = ["windows", "overflow_windows", "hits", "collected", "runs", "big_refine",
                "slow_hits", "anchors"]
        return {k: int(x) for k, x in zip(keys, v)}

    @staticmethod
    def sedef_launch_count() -> int:
        return int(load().sedef_launch_count())

    # -- stages ---------------------------------------------------------------

    def sedef_pack(self, d_seq):
        n = d_seq.numel()
        t = self.torch
        packed = self._empty((n + 15) // 16, t.int32)
        mask = self._empty((n + 31) // 32, t.int32)
        nbits = self._empty((n + 31) // 32, t.int32)
        _check(self.lib.sedef_pack(self.handle, _ptr(d_seq), n, _ptr(packed), _ptr(mask),
                                   _ptr(nbits)))
        return packed, mask, nbits

    def sedef_sketch(self, packed, mask, nbits, offsets, p: Params, cap=None):
        off = _offsets(offsets)
        n = int(off[-1])
        cap = cap if cap is not None else n // 4 + 1024
        count = ctypes.c_int64()
        for _ in range(2):
            rec = self._empty(cap, self.torch.int64)
            st = self.lib.sedef_sketch(self.handle, _ptr(packed), _ptr(mask), _ptr(nbits),
                                       off.ctypes.data, len(off) - 1, ctypes.byref(p), _ptr(rec),
                                       cap, ctypes.byref(count))
            if st == SEDEF_ERR_CAPACITY:
                cap = count.value
                continue
            _check(st)
            return rec[:count.value]
        raise SedefError(SEDEF_ERR_CAPACITY, "sketch capacity")

    def sedef_index(self, rec, p: Params):
        t = self.torch
        nrec = rec.numel()
        srt = self._empty(nrec, t.int64)
        off = self._empty((1 << (2 * p.k)) + 1, t.int32)
        _check(self.lib.sedef_index(self.handle, _ptr(rec), nrec, ctypes.byref(p), _ptr(srt),
                                    _ptr(off)))
        return srt[:nrec], off

    def sedef_filter(self, qrec, qoff, trec, tsorted, toff_tab, toff, p: Params, cap=None):
        qo, to = _offsets(qoff), _offsets(toff)
        if cap is None:
            cap = max(4096, int(qo[-1]) // 16, self._run_cap + self._run_cap // 8)
        count = ctypes.c_int64()
        for _ in range(2):
            runs = self._empty(cap * RUN_DTYPE.itemsize, self.torch.uint8)
            st = self.lib.sedef_filter(self.handle, _ptr(qrec), qrec.numel(), qo.ctypes.data,
                                       len(qo) - 1, _ptr(trec), _ptr(tsorted), _ptr(toff_tab),
                                       trec.numel(), to.ctypes.data, len(to) - 1, ctypes.byref(p),
                                       _ptr(runs), cap, ctypes.byref(count))
            if st == SEDEF_ERR_CAPACITY:
                cap = count.value
                continue
            _check(st)
            self._run_cap = max(self._run_cap, count.value)
            return runs[:count.value * RUN_DTYPE.itemsize], count.value
        raise SedefError(SEDEF_ERR_CAPACITY, "filter capacity")

    def sedef_filter_autotune(self, qrec, qoff, trec, tsorted, toff_tab, toff, p: Params) -> int:
        qo, to = _offsets(qoff), _offsets(toff)
        v = ctypes.c_int32()
        _check(self.lib.sedef_filter_autotune(self.handle, _ptr(qrec), qrec.numel(), qo.ctypes.data,
                                              len(qo) - 1, _ptr(trec), _ptr(tsorted), _ptr(toff_tab),
                                              trec.numel(), to.ctypes.data, len(to) - 1,
                                              ctypes.byref(p), ctypes.byref(v)))
        return v.value

    def sedef_filter_variant(self, set_to: int = -1) -> tuple:
        cur, cnt = ctypes.c_int32(), ctypes.c_int32()
        _check(self.lib.sedef_filter_variant(self.handle, set_to, ctypes.byref(cur), ctypes.byref(cnt)))
        return cur.value, cnt.value

    def sedef_index_save(self, rec, srt, off, k: int, offsets) -> bytes:
        o = _offsets(offsets)
        n = self.lib.sedef_index_blob_size(k, rec.numel(), len(o) - 1)
        blob = np.zeros(n, dtype=np.uint8)
        _check(self.lib.sedef_index_save(self.handle, _ptr(rec), _ptr(srt), _ptr(off), rec.numel(),
                                         k, o.ctypes.data, len(o) - 1, blob.ctypes.data, n))
        return blob.tobytes()

    def sedef_index_load(self, blob: bytes):
        """(records by position, records by hash, offsets, sequence offsets, k)."""
        b = np.frombuffer(blob, dtype=np.uint8)
        k, nrec, nseq = ctypes.c_int32(), ctypes.c_int64(), ctypes.c_int32()
        _check(self.lib.sedef_index_blob_info(b.ctypes.data, len(b), ctypes.byref(k),
                                              ctypes.byref(nrec), ctypes.byref(nseq)))
        t = self.torch
        rec = self._empty(nrec.value, t.int64)
        srt = self._empty(nrec.value, t.int64)
        off = self._empty((1 << (2 * k.value)) + 1, t.int32)
        so = np.zeros(nseq.value + 1, dtype=np.int64)
        _check(self.lib.sedef_index_load(self.handle, b.ctypes.data, len(b), so.ctypes.data,
                                         nseq.value, _ptr(rec), _ptr(srt), _ptr(off), nrec.value))
        return rec[:nrec.value], srt[:nrec.value], off, so, k.value

    def sedef_chain(self, runs, nruns, qrec, qoff, tsorted, toff_tab, toff, p: Params):
        qo, to = _offsets(qoff), _offsets(toff)
        cap = max(int(nruns), 1)
        count = ctypes.c_int64()
        chains = self._empty(cap * CHAIN_DTYPE.itemsize, self.torch.uint8)
        _check(self.lib.sedef_chain(self.handle, _ptr(runs), nruns, _ptr(qrec), qrec.numel(),
                                    qo.ctypes.data, len(qo) - 1, _ptr(tsorted), _ptr(toff_tab),
                                    tsorted.numel(), to.ctypes.data, len(to) - 1, ctypes.byref(p),
                                    _ptr(chains), cap, ctypes.byref(count)))
        return chains[:count.value * CHAIN_DTYPE.itemsize], count.value

    def sedef_extend(self, runs, nruns, qext, qoff, text, toff, p: Params,
                     max_len: int = 1_000_000):
        """f1: potential SD regions of the kept seeds (device uint8 tensor of
        sedef_region_t, count).  qext / text: extension sketches
        (sedef_sketch with min_unmasked = 0)."""
        qo, to = _offsets(qoff), _offsets(toff)
        cap = max(int(nruns), 1)
        count = ctypes.c_int64()
        out = self._empty(cap * REGION_DTYPE.itemsize, self.torch.uint8)
        _check(self.lib.sedef_extend(self.handle, _ptr(runs), int(nruns), _ptr(qext), qext.numel(),
                                     qo.ctypes.data, len(qo) - 1, _ptr(text), text.numel(),
                                     to.ctypes.data, len(to) - 1, ctypes.byref(p), int(max_len),
                                     _ptr(out), cap, ctypes.byref(count)))
        return out[:count.value * REGION_DTYPE.itemsize], count.value

    def sedef_chain2(self, packed, nbits, nbases: int, regions, nregions: int, p: Params,
                     cap: int = None):
        """f2: the SDs inside the potential SD regions (device uint8 tensor of
        sedef_sd_t, count)."""
        cap = cap if cap is not None else max(1024, 4 * int(nregions))
        count = ctypes.c_int64()
        for _ in range(2):
            out = self._empty(cap * SD_DTYPE.itemsize, self.torch.uint8)
            st = self.lib.sedef_chain2(self.handle, _ptr(packed), _ptr(nbits), int(nbases),
                                       _ptr(regions), int(nregions), ctypes.byref(p), _ptr(out), cap,
                                       ctypes.byref(count))
            if st == SEDEF_ERR_CAPACITY:
                cap = count.value
                continue
            _check(st)
            return out[:count.value * SD_DTYPE.itemsize], count.value
        raise SedefError(SEDEF_ERR_CAPACITY, "chain2 capacity")

    def sedef_merge(self, chains, nchains, qoff, toff, p: Params):
        qo, to = _offsets(qoff), _offsets(toff)
        cap = max(int(nchains), 1)
        count = ctypes.c_int64()
        cands = self._empty(cap * CAND_DTYPE.itemsize, self.torch.uint8)
        _check(self.lib.sedef_merge(self.handle, _ptr(chains), nchains, qo.ctypes.data,
                                    len(qo) - 1, to.ctypes.data, len(to) - 1, ctypes.byref(p),
                                    _ptr(cands), cap, ctypes.byref(count)))
        return cands[:count.value * CAND_DTYPE.itemsize], count.value

    def sedef_qgram(self, packed, nbits, nbases: int, runs, nruns: int, p: Params, q: int = 4,
                    p_gap: float = 0.005):
        """f3: (shared q-grams per run (int32 view of u32), pass flags (uint8), passing count)."""
        t = self.torch
        shared = self._empty(nruns, t.int32)
        ok = self._empty(nruns, t.uint8)
        npass = ctypes.c_int64()
        _check(self.lib.sedef_qgram(self.handle, _ptr(packed), _ptr(nbits), int(nbases), _ptr(runs),
                                    int(nruns), ctypes.byref(p), int(q), float(p_gap), _ptr(shared),
                                    _ptr(ok), ctypes.byref(npass)))
        return shared[:nruns], ok[:nruns], npass.value

    def sedef_selfsearch(self, d_seq, offsets, p: Params, cap=None):
        """The whole self-search of a device-resident sequence in one call;
        returns (candidates as a device uint8 tensor of sedef_cand_t, count)."""
        off = _offsets(offsets)
        if cap is None:
            cap = max(4096, self._cand_cap + self._cand_cap // 8)
        count = ctypes.c_int64()
        for _ in range(2):
            out = self._empty(cap * CAND_DTYPE.itemsize, self.torch.uint8)
            st = self.lib.sedef_selfsearch(self.handle, _ptr(d_seq), off.ctypes.data, len(off) - 1,
                                           ctypes.byref(p), _ptr(out), cap, ctypes.byref(count))
            if st == SEDEF_ERR_CAPACITY:
                cap = count.value
                continue
            _check(st)
            self._cand_cap = max(self._cand_cap, count.value)
            return out[:count.value * CAND_DTYPE.itemsize], count.value
        raise SedefError(SEDEF_ERR_CAPACITY, "selfsearch capacity")

    def sedef_selfsearch_host(self, seq: np.ndarray, offsets, p: Params, cap=None):
        seq = np.ascontiguousarray(seq, dtype=np.uint8)
        off = _offsets(offsets)
        if cap is None:
            cap = max(4096, len(seq) // 256, self._cand_cap + self._cand_cap // 8)
        count = ctypes.c_int64()
        for _ in range(2):
            out = np.zeros(cap, dtype=CAND_DTYPE)
            st = self.lib.sedef_selfsearch_host(self.handle, seq.ctypes.data, off.ctypes.data,
                                                len(off) - 1, ctypes.byref(p), out.ctypes.data,
                                                cap, ctypes.byref(count))
            if st == SEDEF_ERR_CAPACITY:
                cap = count.value
                continue
            _check(st)
            self._cand_cap = max(self._cand_cap, count.value)
            return out[:count.value]
        raise SedefError(SEDEF_ERR_CAPACITY, "selfsearch capacity")

    # -- whole path -------------------------------------------------------------

    def selfsearch_graph(self, d_seq, offsets, p: Params, caps: dict = None, slack: float = 1.25):
        """A Graph for this device sequence, run once; rebuilt with larger
        capacities (reported totals x slack) until nothing overflows."""
        caps = dict(caps or default_caps(int(_offsets(offsets)[-1])))
        # a stage's total is exact only once the stages before it fit, so a
        # pass that starts far too small takes a few rebuilds
        for _ in range(8):
            g = Graph(self, d_seq, offsets, p, caps)
            g.launch()
            try:
                g.wait()
                return g
            except SedefError as e:
                if e.status != SEDEF_ERR_CAPACITY:
                    g.close()
                    raise
                for k, v in e.need.items():
                    if v > caps[k]:
                        caps[k] = int(v * slack) + 1024
                g.close()
        raise SedefError(SEDEF_ERR_CAPACITY, "graph capacities did not converge")

    def selfsearch(self, d_seq, offsets, p: Params, autotune: bool = False):
        """All stages on a device-resident sequence; returns every output.
        With autotune, the filter's first-tier shape is chosen first."""
        packed, mask, nbits = self.sedef_pack(d_seq)
        rec = self.sedef_sketch(packed, mask, nbits, offsets, p)
        srt, off = self.sedef_index(rec, p)
        if autotune:
            self.sedef_filter_autotune(rec, offsets, rec, srt, off, offsets, p)
        runs, nruns = self.sedef_filter(rec, offsets, rec, srt, off, offsets, p)
        chains, nch = self.sedef_chain(runs, nruns, rec, offsets, srt, off, offsets, p)
        cands, nc = self.sedef_merge(chains, nch, offsets, offsets, p)
        return dict(packed=packed, mask=mask, nbits=nbits, rec=rec, sorted=srt, off=off,
                    runs=runs, nruns=nruns, chains=chains, nchains=nch, cands=cands, ncands=nc)


class Graph:
    """One captured self-search pass (sedef_graph_*): recorded once for a
    device sequence and its offsets, replayed by `run`.  Output buffers are
    torch tensors held here; `need` after a run holds the exact totals."""

    def __init__(self, ctx: "Context", d_seq, offsets, p: Params, caps: dict):
        t = ctx.torch
        self.ctx, self.lib, self.d_seq = ctx, ctx.lib, d_seq
        self.offsets = _offsets(offsets)
        self.p = params_from_struct(p)
        self.caps = {k: max(1, int(caps[k])) for k in CAP_NAMES}
        c = self.caps
        self.rec = ctx._empty(c["records"], t.int64)
        self.sorted = ctx._empty(c["records"], t.int64)
        self.off = ctx._empty((1 << (2 * p.k)) + 1, t.int32)
        self.runs = ctx._empty(c["runs"] * RUN_DTYPE.itemsize, t.uint8)
        self.chains = ctx._empty(c["chains"] * CHAIN_DTYPE.itemsize, t.uint8)
        self.cands = ctx._empty(c["cands"] * CAND_DTYPE.itemsize, t.uint8)
        gc = GraphCaps(**c)
        h = ctypes.c_void_p()
        _check(self.lib.sedef_graph_create(
            ctx.handle, _ptr(d_seq), self.offsets.ctypes.data, len(self.offsets) - 1,
            ctypes.byref(self.p), ctypes.byref(gc), _ptr(self.rec), _ptr(self.sorted),
            _ptr(self.off), _ptr(self.runs), _ptr(self.chains), _ptr(self.cands), ctypes.byref(h)))
        self.handle = h
        self.nodes = int(self.lib.sedef_graph_nodes(h))
        self.need = None

    def launch(self, stream=None):
        """Enqueues one replay on `stream` (default: the context's stream, so
        that it follows the work that filled the input)."""
        stream = stream if stream is not None else self.ctx.stream
        _check(self.lib.sedef_graph_launch(self.handle, ctypes.c_void_p(stream.cuda_stream)))

    def wait(self) -> dict:
        """Synchronizes; the exact totals.  Raises SedefError (with .need)
        when a capacity was exceeded."""
        need = np.zeros(6, dtype=np.int64)
        st = self.lib.sedef_graph_wait(self.handle, need.ctypes.data)
        self.need = {k: int(v) for k, v in zip(CAP_NAMES, need)}
        if st != SEDEF_OK:
            err = SedefError(st, self.lib.sedef_last_error().decode())
            err.need = self.need
            raise err
        return self.need

    def outputs(self) -> dict:
        """The last run's outputs (views of the graph's buffers)."""
        n = {k: min(self.need[k], self.caps[k]) for k in CAP_NAMES}
        return dict(rec=self.rec[:n["records"]], sorted=self.sorted[:n["records"]], off=self.off,
                    runs=self.runs[:n["runs"] * RUN_DTYPE.itemsize], nruns=n["runs"],
                    chains=self.chains[:n["chains"] * CHAIN_DTYPE.itemsize], nchains=n["chains"],
                    cands=self.cands[:n["cands"] * CAND_DTYPE.itemsize], ncands=n["cands"])

    def close(self):
        if self.handle:
            self.lib.sedef_graph_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def caps_from_run(out: dict, stats: dict, slack: float = 1.25) -> dict:
    """Capacities for a captured pass from an eager pass over the same kind
    of input (its counts and the context's statistics) times `slack`."""
    need = {"records": out["rec"].numel(), "slow_hits": stats["slow_hits"], "runs": out["nruns"],
            "anchors": stats["anchors"], "chains": out["nchains"], "cands": out["ncands"]}
    return {k: int(v * slack) + 1024 for k, v in need.items()}


def default_caps(n_bases: int) -> dict:
    """First-guess capacities for a pass over n_bases bases (a graph that
    overflows is rebuilt from the reported totals)."""
    return {"records": n_bases // 4 + 1024, "slow_hits": n_bases // 16 + (1 << 20),
            "runs": n_bases // 32 + 4096, "anchors": n_bases // 8 + (1 << 16),
            "chains": n_bases // 32 + 4096, "cands": n_bases // 32 + 4096}


def sedef_sketch_noalloc(packed, mask, nbits, offsets, p: Params, rec, stream) -> int:
    """The allocation-free sketch: `rec` is a caller-allocated device tensor
    (int64) whose capacity is its length; returns the number of records
    written (raises SedefError, with status -6 and the needed count in the
    message, when rec is too small)."""
    off = _offsets(offsets)
    count = ctypes.c_int64()
    st = load().sedef_sketch_noalloc(_ptr(packed), _ptr(mask), _ptr(nbits), off.ctypes.data,
                                     len(off) - 1, ctypes.byref(p), _ptr(rec), rec.numel(),
                                     ctypes.byref(count), ctypes.c_void_p(stream.cuda_stream))
    _check(st)
    return count.value


def to_numpy_records(t) -> np.ndarray:
    """Device int64 record tensor -> numpy uint64."""
    return t.cpu().numpy().view(np.uint64)


def records_to_rows(rec: np.ndarray) -> np.ndarray:
    """uint64 records -> int64 rows (hash, pos, strand) as the oracle prints them."""
    rec = rec.view(np.uint64)
    out = np.zeros((len(rec), 3), dtype=np.int64)
    out[:, 0] = (rec >> np.uint64(33)).astype(np.int64)
    out[:, 1] = ((rec >> np.uint64(1)) & np.uint64(0xFFFFFFFF)).astype(np.int64)
    out[:, 2] = (rec & np.uint64(1)).astype(np.int64)
    return out


def struct_view(t, dtype) -> np.ndarray:
    return t.cpu().numpy().view(dtype)


class DeviceServer:
    """sedef_server_*: continuous batching over a resident target index.  A
    persistent filter kernel drains a device work queue of query windows;
    `submit` admits a request into a free slot (None when none is free),
    `poll` returns a slot whose windows are filtered, `finish` completes it
    and returns its candidates."""

    def __init__(self, ctx: "Context", trec, tsorted, toff_tab, toffsets, p: Params,
                 slots: int = 8, slot_bases: int = 5_000_000, idle_timeout_s: float = 1.0):
        self.lib = ctx.lib
        self.ctx = ctx  # the index tensors and the context outlive the server
        self.keep = (trec, tsorted, toff_tab)
        off = _offsets(toffsets)
        self.p = params_from_struct(p, self_mode=0)
        self.slots = slots
        self.slot_bases = slot_bases
        h = ctypes.c_void_p()
        _check(self.lib.sedef_server_create(ctx.handle, _ptr(trec), _ptr(tsorted), _ptr(toff_tab),
                                            trec.numel(), off.ctypes.data, len(off) - 1,
                                            ctypes.byref(self.p), slots, slot_bases,
                                            float(idle_timeout_s), ctypes.byref(h)))
        self.handle = h
        self._cap = 1 << 16

    def submit(self, seq: np.ndarray):
        """The slot the request went to, or None when every slot is busy."""
        seq = np.ascontiguousarray(seq, dtype=np.uint8)
        slot = ctypes.c_int32(-1)
        st = self.lib.sedef_server_submit(self.handle, seq.ctypes.data, len(seq), ctypes.byref(slot))
        if st == SEDEF_ERR_CAPACITY:
            return None
        _check(st)
        return slot.value

    def poll(self, wait_s: float = 0.0):
        slot = ctypes.c_int32(-1)
        _check(self.lib.sedef_server_poll(self.handle, float(wait_s), ctypes.byref(slot)))
        return slot.value if slot.value >= 0 else None

    def finish(self, slot: int) -> np.ndarray:
        count = ctypes.c_int64()
        for _ in range(2):
            out = np.zeros(self._cap, dtype=CAND_DTYPE)
            st = self.lib.sedef_server_finish(self.handle, slot, out.ctypes.data, self._cap,
                                              ctypes.byref(count))
            if st == SEDEF_ERR_CAPACITY:
                self._cap = int(count.value) + 1024
                continue
            _check(st)
            return out[:count.value]
        raise SedefError(SEDEF_ERR_CAPACITY, "server candidates")

    def status(self) -> dict:
        run, tmo = ctypes.c_int32(), ctypes.c_int32()
        st = self.lib.sedef_server_status(self.handle, ctypes.byref(run), ctypes.byref(tmo))
        return {"status": st, "running": bool(run.value), "timed_out": bool(tmo.value)}

    def smem_left(self) -> int:
        """Shared memory per CTA that kernels of other streams find beside
        the persistent kernel."""
        n = ctypes.c_int64()
        _check(self.lib.sedef_server_smem_left(self.handle, ctypes.byref(n)))
        return n.value

    def close(self):
        if self.handle:
            self.lib.sedef_server_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
