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
