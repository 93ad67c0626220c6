"""CPU oracle for the SEDEF seeding filter -- TEST INFRASTRUCTURE ONLY.

A plain, slow restatement (``sedef_oracle.cpp``, compiled with g++) of what
the seeding filter computes, written from the paper's text.  Only the tests,
``__graft_entry__.smoke()`` and the benchmark's CPU-baseline leg may import
it.  The CUDA library never loads it, and it shares no code with that library.

Every function returns numpy arrays of int64 rows; column meanings are given
in each docstring and in ``sedef_oracle.cpp``.
"""
from __future__ import annotations

import ctypes
import os
import struct
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "sedef_oracle.cpp")
_LIB_PATH = os.path.join(_HERE, "_build", "liboracle.so")
_lock = threading.Lock()
_lib = None

# Parameter defaults.  k = 12 (Section 3.3), n = 750 (Section 3, n >=
# 1000*(1-delta)), delta_M = 0.15 and delta_G = 0.10 (Section 2.1, delta =
# 0.25).  w, step, gap_max and diag_max are readings (the paper is silent):
# w = 16, step = 250 (= 1000 - n, so every 1 kbp duplication holds a whole
# query window), gap_max = n, diag_max = ceil(n * delta_G).
DEFAULTS = dict(k=12, w=16, n=750, step=250, max_occ=0, self_mode=1,
                gap_max=750, diag_max=75, min_unmasked=1,
                delta_m=0.15, delta_g=0.10)

RUN_COLS = ["i", "o", "j_a", "j_b", "max_shared", "j_at_max", "s", "m",
            "est", "j_star", "den", "keep"]
CHAIN_COLS = ["i", "o", "qseq", "q0", "q1", "tseq", "t0", "t1", "score", "s"]
CAND_COLS = ["qseq", "q0", "q1", "tseq", "t0", "t1", "o", "score", "nchains"]


def build(force: bool = False) -> str:
    """Compile the oracle (plain C++17, -O2) and return the library path."""
    os.makedirs(os.path.dirname(_LIB_PATH), exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    subprocess.check_call(["g++", "-O2", "-std=c++17", "-shared", "-fPIC", "-pthread",
                           "-o", tmp, _SRC])
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            vp, i64, i32 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int
            lib.orc_table_rows.restype = i64
            lib.orc_table_rows.argtypes = [vp]
            lib.orc_table_cols.restype = i64
            lib.orc_table_cols.argtypes = [vp]
            lib.orc_table_copy.argtypes = [vp, vp]
            lib.orc_table_free.argtypes = [vp]
            lib.orc_pack.argtypes = [vp, i64, vp, vp, vp]
            lib.orc_hash.restype = ctypes.c_uint64
            lib.orc_hash.argtypes = [ctypes.c_uint64, i32]
            lib.orc_hash_all.argtypes = [i32, vp]
            lib.orc_tau.restype = ctypes.c_double
            lib.orc_tau.argtypes = [i64, ctypes.c_double, ctypes.c_double]
            lib.orc_mtable.argtypes = [i64, ctypes.c_double, ctypes.c_double, i64, vp]
            lib.orc_sketch.restype = vp
            lib.orc_sketch.argtypes = [vp, vp, i32, vp, i32]
            lib.orc_index.restype = vp
            lib.orc_index.argtypes = [vp, i64, i32, vp]
            lib.orc_filter.restype = vp
            lib.orc_filter.argtypes = [vp, i64, vp, i32, vp, i64, vp, i32, vp, vp, i64, i32, i32]
            lib.orc_chain.restype = vp
            lib.orc_chain.argtypes = [vp, i64, i64, vp, i64, vp, i32, vp, i64, vp, i32, vp]
            lib.orc_chain_anchors.restype = vp
            lib.orc_chain_anchors.argtypes = [vp, i64, i64, i64]
            lib.orc_merge.restype = vp
            lib.orc_merge.argtypes = [vp, i64, i64, vp]
            lib.orc_jaccard.restype = ctypes.c_double
            lib.orc_jaccard.argtypes = [vp, i64, i64, i64, i32]
            lib.orc_qgram_bound.restype = ctypes.c_double
            lib.orc_qgram_bound.argtypes = [i64, i32, ctypes.c_double, ctypes.c_double,
                                            ctypes.c_double]
            lib.orc_qgram_shared.restype = i64
            lib.orc_qgram_shared.argtypes = [vp, i64, i64, i64, i32, i32]
            lib.orc_qgram.restype = vp
            lib.orc_qgram.argtypes = [vp, vp, i64, i64, vp, i32, ctypes.c_double]
            lib.orc_mems.restype = vp
            lib.orc_mems.argtypes = [vp, i64, vp, i64, i64]
            lib.orc_chain_tiers.restype = vp
            lib.orc_chain_tiers.argtypes = [vp, i64, i64, i64, i64, i64]
            lib.orc_chain2.restype = vp
            lib.orc_chain2.argtypes = [vp, vp, i64, i64, i64, i64, i64, i64, i64, i64, i32]
            lib.orc_extend.restype = vp
            lib.orc_extend.argtypes = [vp, i64, i64, vp, i64, vp, i32, vp, i64, vp, i32, vp, i64,
                                       i32]
            _lib = lib
    return _lib


def params(**kw) -> dict:
    p = dict(DEFAULTS)
    p.update(kw)
    return p


def _par_array(p: dict) -> np.ndarray:
    a = np.zeros(11, dtype=np.int64)
    for idx, key in enumerate(["k", "w", "n", "step", "max_occ", "self_mode",
                               "gap_max", "diag_max", "min_unmasked"]):
        a[idx] = int(p[key])
    a[9] = struct.unpack("<q", struct.pack("<d", float(p["delta_m"])))[0]
    a[10] = struct.unpack("<q", struct.pack("<d", float(p["delta_g"])))[0]
    return a


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _table(lib, h) -> np.ndarray:
    try:
        rows, cols = lib.orc_table_rows(h), lib.orc_table_cols(h)
        out = np.zeros((rows, cols), dtype=np.int64)
        if rows:
            lib.orc_table_copy(h, _ptr(out))
        return out
    finally:
        lib.orc_table_free(h)


def _c(a, dtype):
    return np.ascontiguousarray(a, dtype=dtype)


def pack(seq: np.ndarray):
    """a1: returns (packed u32[ceil(N/16)], mask u32[ceil(N/32)], nbits u32[ceil(N/32)])."""
    lib = _load()
    seq = _c(seq, np.uint8)
    n = len(seq)
    packed = np.zeros((n + 15) // 16, dtype=np.uint32)
    mask = np.zeros((n + 31) // 32, dtype=np.uint32)
    nbits = np.zeros((n + 31) // 32, dtype=np.uint32)
    lib.orc_pack(_ptr(seq), n, _ptr(packed), _ptr(mask), _ptr(nbits))
    return packed, mask, nbits


def hash_code(code: int, k: int) -> int:
    return int(_load().orc_hash(code, k))


def hash_all(k: int) -> np.ndarray:
    out = np.zeros(1 << (2 * k), dtype=np.uint64)
    _load().orc_hash_all(k, _ptr(out))
    return out


def tau(k=12, delta_m=0.15, delta_g=0.10) -> float:
    return float(_load().orc_tau(k, delta_m, delta_g))


def mtable(k=12, delta_m=0.15, delta_g=0.10, smax=739) -> np.ndarray:
    out = np.zeros(smax + 1, dtype=np.int64)
    _load().orc_mtable(k, delta_m, delta_g, smax, _ptr(out))
    return out


def sketch(seq: np.ndarray, offsets: np.ndarray, p: dict, threads: int = 1) -> np.ndarray:
    """a2: rows (hash, pos, strand), sorted by pos.  `threads` > 1 shares the
    (independent) sequences out to threads; the rows are the same."""
    lib = _load()
    seq = _c(seq, np.uint8)
    offsets = _c(offsets, np.int64)
    return _table(lib, lib.orc_sketch(_ptr(seq), _ptr(offsets), len(offsets) - 1,
                                      _ptr(_par_array(p)), int(threads)))


def index(recs: np.ndarray, k: int):
    """a3: (rows sorted by (hash, pos), offsets u32[4^k + 1])."""
    lib = _load()
    recs = _c(recs, np.int64)
    off = np.zeros((1 << (2 * k)) + 1, dtype=np.uint32)
    rows = _table(lib, lib.orc_index(_ptr(recs), len(recs), k, _ptr(off)))
    return rows, off


def filter_runs(qrecs, qoff, trecs, toff, p: dict, windows=None, dense=False,
                threads: int = 1) -> np.ndarray:
    """a4-a6: run rows (see RUN_COLS), in (i, o, j_a) order.  `threads` > 1
    shares the (independent) windows out to threads; the rows are the same."""
    lib = _load()
    qrecs, trecs = _c(qrecs, np.int64), _c(trecs, np.int64)
    qoff, toff = _c(qoff, np.int64), _c(toff, np.int64)
    if windows is None:
        win, nwin = np.zeros(1, dtype=np.int64), -1
    else:
        win = _c(windows, np.int64)
        nwin = len(win)
    h = lib.orc_filter(_ptr(qrecs), len(qrecs), _ptr(qoff), len(qoff) - 1,
                       _ptr(trecs), len(trecs), _ptr(toff), len(toff) - 1,
                       _ptr(_par_array(p)), _ptr(win), nwin, 1 if dense else 0, int(threads))
    return _table(lib, h)


def chain(runs, qrecs, qoff, trecs, toff, p: dict) -> np.ndarray:
    """a7 (chaining): chain rows (see CHAIN_COLS), one per kept seed whose
    best chain reaches m[s], in run order."""
    lib = _load()
    runs = _c(runs, np.int64).reshape(-1, len(RUN_COLS))
    qrecs, trecs = _c(qrecs, np.int64), _c(trecs, np.int64)
    qoff, toff = _c(qoff, np.int64), _c(toff, np.int64)
    h = lib.orc_chain(_ptr(runs), len(runs), runs.shape[1],
                      _ptr(qrecs), len(qrecs), _ptr(qoff), len(qoff) - 1,
                      _ptr(trecs), len(trecs), _ptr(toff), len(toff) - 1,
                      _ptr(_par_array(p)))
    return _table(lib, h)


def chain_anchors(anchors: np.ndarray, gap_max: int, diag_max: int) -> np.ndarray:
    """Chain DP on one explicit anchor list: rows (p, t', f, pred), sorted."""
    lib = _load()
    anchors = _c(anchors, np.int64).reshape(-1, 2)
    return _table(lib, lib.orc_chain_anchors(_ptr(anchors), len(anchors), gap_max, diag_max))


def merge(chains: np.ndarray, p: dict) -> np.ndarray:
    """a7 (merge): candidate rows (see CAND_COLS), global coordinates."""
    lib = _load()
    chains = _c(chains, np.int64).reshape(-1, len(CHAIN_COLS))
    return _table(lib, lib.orc_merge(_ptr(chains), len(chains), chains.shape[1],
                                     _ptr(_par_array(p))))


def jaccard(seq: np.ndarray, i: int, j: int, n: int, k: int) -> float:
    seq = _c(seq, np.uint8)
    return float(_load().orc_jaccard(_ptr(seq), i, j, n, k))


QGRAM_COLS = ["shared", "pass"]


def qgram_bound(n: int, q: int, delta_g=0.10, delta_m=0.15, p_gap=0.005) -> float:
    """Section 3.2's lower bound on the q-grams a pair within the SD error
    model shares."""
    return float(_load().orc_qgram_bound(n, q, delta_g, delta_m, p_gap))


def qgram_shared(seq: np.ndarray, i: int, j: int, n: int, o: int, q: int) -> int:
    """Q of G[i, i+n) and G[j, j+n) (reverse-complemented for o = 1)."""
    seq = _c(seq, np.uint8)
    return int(_load().orc_qgram_shared(_ptr(seq), i, j, n, o, q))


def qgram(seq: np.ndarray, runs: np.ndarray, p: dict, q: int = 4, p_gap: float = 0.005) -> np.ndarray:
    """f3: per run rows (shared q-grams, pass) of each kept seed (Section 3.2)."""
    lib = _load()
    seq = _c(seq, np.uint8)
    runs = _c(runs, np.int64).reshape(-1, len(RUN_COLS))
    h = lib.orc_qgram(_ptr(seq), _ptr(runs), len(runs), len(RUN_COLS), _ptr(_par_array(p)),
                      int(q), float(p_gap))
    return _table(lib, h)


EXTEND_COLS = ["i", "o", "j_star", "qa", "qb", "ta", "tb", "est", "den"]
MAX_SD_LENGTH = 1_000_000  # Section 3.2: potential SDs of at most 1 Mbp


def extend(runs, qrecs_all, qoff, trecs_all, toff, p: dict, max_len: int = MAX_SD_LENGTH,
           threads: int = 1) -> np.ndarray:
    """f1 (Section 3.2): one potential SD region per kept seed, in run order
    (see EXTEND_COLS; global coordinates).  qrecs_all / trecs_all are the
    extension sketches: all k-mers, masked ones included (sketch with
    min_unmasked = 0).  `threads` > 1 shares the seeds out to threads."""
    lib = _load()
    runs = _c(runs, np.int64).reshape(-1, len(RUN_COLS))
    qrecs_all, trecs_all = _c(qrecs_all, np.int64), _c(trecs_all, np.int64)
    qoff, toff = _c(qoff, np.int64), _c(toff, np.int64)
    h = lib.orc_extend(_ptr(runs), len(runs), runs.shape[1], _ptr(qrecs_all), len(qrecs_all),
                       _ptr(qoff), len(qoff) - 1, _ptr(trecs_all), len(trecs_all), _ptr(toff),
                       len(toff) - 1, _ptr(_par_array(p)), int(max_len), int(threads))
    return _table(lib, h)


# Section 3.3: exact seeds of at least 11 bases; initial chains with gaps of
# at most l * delta_G = 100 (l = 1,000); final chains with gaps of at most
# 10,000 and an affine penalty (readings: open 25, one per 50 gap bases);
# an SD spans at least 1,000 bases.
CHAIN2 = dict(k2=11, g1=100, g2=10_000, gap_open=25, gap_div=50, min_len=1000)
CHAIN2_COLS = ["region", "o", "q0", "q1", "t0", "t1", "score", "seeds", "parts"]


def mems(x: bytes, y: bytes, k2: int = 11) -> np.ndarray:
    """Maximal exact ACGT matches of at least k2 bases: rows (x, y, L)."""
    lib = _load()
    bx, by = np.frombuffer(x, dtype=np.uint8), np.frombuffer(y, dtype=np.uint8)
    return _table(lib, lib.orc_mems(_ptr(bx), len(bx), _ptr(by), len(by), k2))


def chain_tiers(seeds, g1=100, g2=10_000, gap_open=25, gap_div=50) -> np.ndarray:
    """Both chaining tiers on explicit seeds (x, y, L): final chains
    (x0, x1, y0, y1, score, seeds, parts) in extraction order."""
    lib = _load()
    seeds = _c(seeds, np.int64).reshape(-1, 3)
    return _table(lib, lib.orc_chain_tiers(_ptr(seeds), len(seeds), g1, g2, gap_open, gap_div))


def chain2(seq, regions, c: dict = None, threads: int = 1) -> np.ndarray:
    """f2 (Section 3.3): the final chains (SDs) inside each potential SD
    region (rows of `extend`); see CHAIN2_COLS."""
    lib = _load()
    c = dict(CHAIN2, **(c or {}))
    seq = _c(seq, np.uint8)
    regions = _c(regions, np.int64).reshape(-1, len(EXTEND_COLS))
    h = lib.orc_chain2(_ptr(seq), _ptr(regions), len(regions), regions.shape[1], c["k2"], c["g1"],
                       c["g2"], c["gap_open"], c["gap_div"], c["min_len"], int(threads))
    return _table(lib, h)


def selfsearch(seq, offsets, p: dict, threads: int = 1):
    """All steps for a self-search: returns dict of every intermediate.
    `threads` > 1 runs the sketch (per sequence) and the filter (per window)
    on threads; the results are the same."""
    recs = sketch(seq, offsets, p, threads=threads)
    idx_rows, off = index(recs, p["k"])
    runs = filter_runs(recs, offsets, recs, offsets, p, threads=threads)
    chains = chain(runs, recs, offsets, recs, offsets, p)
    cands = merge(chains, p)
    return dict(recs=recs, index=idx_rows, offsets=off, runs=runs, chains=chains, cands=cands)
