"""The C ABI library builds, loads without a GPU and exports every function
that include/sedef.h declares (no compute calls here)."""
import ctypes
import os
import re

from paper_1807_00205_gb300 import binding
from paper_1807_00205_gb300 import build as libbuild

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    text = open(os.path.join(ROOT, "include", "sedef.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(sedef_[a-z_0-9]+)\s*\(", text)) -
                  {"sedef_params"})


def test_header_declares_the_path():
    names = declared_functions()
    for n in ["sedef_pack", "sedef_sketch", "sedef_index", "sedef_filter", "sedef_chain",
              "sedef_merge"]:
        assert n in names


def test_library_exports_every_declared_symbol():
    path = libbuild.build()
    lib = ctypes.CDLL(path)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing
    assert set(binding.EXPORTS) == set(declared_functions())


def test_host_only_calls():
    lib = binding.load()
    p = binding.params()
    assert (p.k, p.w, p.n, p.query_step) == (12, 16, 750, 250)
    tau = ctypes.c_double()
    m = (ctypes.c_int32 * 740)()
    assert lib.sedef_threshold_table(ctypes.byref(p), m, 739, ctypes.byref(tau)) == 0
    import oracle
    assert abs(tau.value - oracle.tau()) < 1e-15
    assert list(m) == [int(x) for x in oracle.mtable(smax=739)]
    bad = binding.params(k=16)
    assert lib.sedef_threshold_table(ctypes.byref(bad), m, 739, ctypes.byref(tau)) == -5
    assert b"k must be" in lib.sedef_last_error()


def test_index_blob_checks_on_host():
    """The blob size follows its stated layout, and a buffer that is not a
    well-formed blob is refused without touching a device."""
    import numpy as np
    lib = binding.load()
    assert lib.sedef_index_blob_size(12, 1000, 3) == 32 + 8 * 4 + 16 * 1000 + 4 * (4**12 + 1) + 8
    assert lib.sedef_index_blob_size(16, 10, 1) == -1
    k, n, s = ctypes.c_int32(), ctypes.c_int64(), ctypes.c_int32()
    junk = np.zeros(4096, dtype=np.uint8)
    assert lib.sedef_index_blob_info(junk.ctypes.data, len(junk), ctypes.byref(k),
                                     ctypes.byref(n), ctypes.byref(s)) == -1
    assert b"not an index blob" in lib.sedef_last_error()
    head = np.frombuffer(b"SEDEFIDX" + bytes([1, 0, 0, 0, 12, 0, 0, 0]) + bytes(16), np.uint8)
    junk[:32] = head
    assert lib.sedef_index_blob_info(junk.ctypes.data, len(junk), ctypes.byref(k),
                                     ctypes.byref(n), ctypes.byref(s)) == -1
    assert b"size does not match" in lib.sedef_last_error()


def test_null_handles_are_refused_without_a_gpu():
    """Every entry point that takes a context, graph or server refuses a NULL
    one with SEDEF_ERR_INVALID (-1) before any CUDA call, and NULL output
    pointers are refused the same way; nothing here needs a GPU."""
    lib = binding.load()
    p = binding.params()
    P = ctypes.byref(p)
    n64 = ctypes.c_int64()
    n32 = ctypes.c_int32()
    off = (ctypes.c_int64 * 2)(0, 1000)
    N = None
    calls = {
        "sedef_pack": lambda: lib.sedef_pack(N, N, 10, N, N, N),
        "sedef_sketch": lambda: lib.sedef_sketch(N, N, N, N, off, 1, P, N, 0, ctypes.byref(n64)),
        "sedef_sketch_noalloc": lambda: lib.sedef_sketch_noalloc(N, N, N, off, 1, P, N, 0, N, N),
        "sedef_index": lambda: lib.sedef_index(N, N, 10, P, N, N),
        "sedef_filter": lambda: lib.sedef_filter(N, N, 0, off, 1, N, N, N, 0, off, 1, P, N, 0,
                                                 ctypes.byref(n64)),
        "sedef_filter_autotune": lambda: lib.sedef_filter_autotune(N, N, 0, off, 1, N, N, N, 0, off,
                                                                   1, P, ctypes.byref(n32)),
        "sedef_filter_variant": lambda: lib.sedef_filter_variant(N, 0, N, N),
        "sedef_filter_stats": lambda: lib.sedef_filter_stats(N, N, 8),
        "sedef_chain": lambda: lib.sedef_chain(N, N, 0, N, 0, off, 1, N, N, 0, off, 1, P, N, 0,
                                               ctypes.byref(n64)),
        "sedef_extend": lambda: lib.sedef_extend(N, N, 0, N, 0, off, 1, N, 0, off, 1, P, 10**6, N,
                                                 0, ctypes.byref(n64)),
        "sedef_merge": lambda: lib.sedef_merge(N, N, 0, off, 1, off, 1, P, N, 0, ctypes.byref(n64)),
        "sedef_chain2": lambda: lib.sedef_chain2(N, N, N, 0, N, 0, P, N, 0, ctypes.byref(n64)),
        "sedef_qgram": lambda: lib.sedef_qgram(N, N, N, 0, N, 0, P, 4, 0.005, N, N,
                                               ctypes.byref(n64)),
        "sedef_selfsearch": lambda: lib.sedef_selfsearch(N, N, off, 1, P, N, 0, ctypes.byref(n64)),
        "sedef_selfsearch_host": lambda: lib.sedef_selfsearch_host(N, N, off, 1, P, N, 0,
                                                                   ctypes.byref(n64)),
        "sedef_set_stream": lambda: lib.sedef_set_stream(N, N),
        "sedef_set_scratch_limit": lambda: lib.sedef_set_scratch_limit(N, 0),
        "sedef_set_tier_smem_limit": lambda: lib.sedef_set_tier_smem_limit(N, 0),
        "sedef_trace_enable": lambda: lib.sedef_trace_enable(N, 1),
        "sedef_trace_report": lambda: lib.sedef_trace_report(N, N, 0, 0),
        "sedef_index_save": lambda: lib.sedef_index_save(N, N, N, N, 0, 12, off, 1, N, 0),
        "sedef_index_load": lambda: lib.sedef_index_load(N, N, 0, N, 0, N, N, N, 0),
        "sedef_graph_create": lambda: lib.sedef_graph_create(N, N, off, 1, P, N, N, N, N, N, N, N,
                                                             N),
        "sedef_graph_launch": lambda: lib.sedef_graph_launch(N, N),
        "sedef_graph_wait": lambda: lib.sedef_graph_wait(N, N),
        "sedef_server_create": lambda: lib.sedef_server_create(N, N, N, N, 0, off, 1, P, 1, 1000,
                                                               1.0, N),
        "sedef_server_submit": lambda: lib.sedef_server_submit(N, N, 0, ctypes.byref(n32)),
        "sedef_server_poll": lambda: lib.sedef_server_poll(N, 0.0, ctypes.byref(n32)),
        "sedef_server_finish": lambda: lib.sedef_server_finish(N, 0, N, 0, ctypes.byref(n64)),
        "sedef_server_status": lambda: lib.sedef_server_status(N, N, N),
        "sedef_server_smem_left": lambda: lib.sedef_server_smem_left(N, N),
        "sedef_threshold_table": lambda: lib.sedef_threshold_table(N, N, 0, N),
        "sedef_index_blob_info": lambda: lib.sedef_index_blob_info(N, 0, N, N, N),
    }
    for name, call in calls.items():
        assert call() == -1, name
        assert lib.sedef_last_error() != b"", name
    # destroying nothing is a no-op; a graph's node count of nothing is -1
    assert lib.sedef_destroy(N) == 0 and lib.sedef_graph_destroy(N) == 0
    assert lib.sedef_server_destroy(N) == 0 and lib.sedef_graph_nodes(N) == -1
    declared = set(declared_functions())
    covered = set(calls) | {"sedef_destroy", "sedef_graph_destroy", "sedef_server_destroy",
                            "sedef_graph_nodes", "sedef_create", "sedef_default_params",
                            "sedef_last_error", "sedef_launch_count", "sedef_index_blob_size"}
    assert declared <= covered, declared - covered
