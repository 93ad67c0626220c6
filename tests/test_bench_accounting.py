"""The benchmark's algorithmic-byte accounting (host logic, no GPU): the
filter's count of query records, distinct query hashes and postings per
window, against a direct count over explicit windows."""
import numpy as np
import pytest

import oracle
from paper_1807_00205_gb300 import synth


def _records(rows: np.ndarray) -> np.ndarray:
    """Oracle rows (hash, pos, strand) in the library's uint64 layout."""
    return ((rows[:, 0].astype(np.uint64) << np.uint64(33)) |
            (rows[:, 1].astype(np.uint64) << np.uint64(1)) | rows[:, 2].astype(np.uint64))


@pytest.mark.parametrize("self_mode", [1, 2])
def test_filter_bytes_match_direct_count(self_mode):
    torch = pytest.importorskip("torch")
    import bench
    g = synth.small_case(5, lengths=(30_000, 12_000, 700, 20_000), n_sd=4, mask_frac=0.2)
    pd = oracle.params(self_mode=self_mode)
    rows = oracle.sketch(g.seq, g.offsets, pd)
    rec = torch.from_numpy(_records(rows).view(np.int64))
    got = bench.filter_algorithmic_bytes(rec, g.offsets, pd["k"], pd["n"], pd["step"], self_mode,
                                         nruns=7)
    span = pd["n"] - pd["k"]
    seq_of = np.searchsorted(g.offsets, rows[:, 1], side="right") - 1
    nq = npairs = post = nwin = 0
    for s in range(len(g.offsets) - 1):
        st, en = int(g.offsets[s]), int(g.offsets[s + 1])
        for i in range(st, en - pd["n"] + 1, pd["step"]):
            nwin += 1
            sel = (rows[:, 1] >= i) & (rows[:, 1] <= i + span)
            nq += int(sel.sum())
            hs = np.unique(rows[sel, 0])
            npairs += len(hs)
            pool = rows[seq_of == s] if self_mode == 2 else rows
            post += int(np.isin(pool[:, 0], hs).sum())
    assert got["windows"] == nwin and got["query_records"] == nq
    assert got["distinct_query_hashes"] == npairs and got["postings"] == post
    assert got["bytes"] == 4 * post + 8 * npairs + 8 * nq + 32 * 7


def test_counters_used_only_for_their_workload_shape_and_source(tmp_path, monkeypatch):
    """The per-unit ncu counters behind roofline.issue / roofline.traffic are
    used only for the workload and filter shape they were captured on, and
    only while the captured source file is unchanged."""
    import hashlib
    import json
    import bench
    src = tmp_path / "kernel.cu"
    src.write_text("// captured revision\n")
    entry = {"kernel": "filter family", "workload": "batch", "filter_shape": 11,
             "source": str(src), "sha256": hashlib.sha256(src.read_bytes()).hexdigest(),
             "unit": "hits", "warp_instructions_per_unit": 32.0, "dram_bytes_per_unit": 20.0}
    path = tmp_path / "counters.json"
    path.write_text(json.dumps({"entries": [entry]}))
    monkeypatch.setattr(bench, "COUNTERS", str(path))
    assert bench.counters_entry("filter family", "batch", 11)["warp_instructions_per_unit"] == 32.0
    assert bench.counters_entry("filter family", "batch", 3) is None
    assert bench.counters_entry("filter family", "human", 11) is None
    assert bench.counters_entry("refine family", "batch", 11) is None
    src.write_text("// changed revision\n")
    assert bench.counters_entry("filter family", "batch", 11) is None
    monkeypatch.setattr(bench, "COUNTERS", str(tmp_path / "missing.json"))
    assert bench.counters_entry("filter family", "batch", 11) is None
