"""Helpers shared by the GPU parity tests: run a stage through the C ABI and
convert its output to the oracle's row layout (test-side conversion only)."""
import numpy as np
import pytest

import oracle
from paper_1807_00205_gb300 import binding


def need_gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def run_rows(runs_t) -> np.ndarray:
    r = binding.struct_view(runs_t, binding.RUN_DTYPE)
    if len(r) == 0:
        return np.zeros((0, len(oracle.RUN_COLS)), dtype=np.int64)
    return np.stack([r[c].astype(np.int64) for c in oracle.RUN_COLS], axis=1)


def chain_rows(chains_t) -> np.ndarray:
    c = binding.struct_view(chains_t, binding.CHAIN_DTYPE)
    if len(c) == 0:
        return np.zeros((0, len(oracle.CHAIN_COLS)), dtype=np.int64)
    return np.stack([c[k].astype(np.int64) for k in oracle.CHAIN_COLS], axis=1)


def cand_rows_global(cands, offsets) -> np.ndarray:
    """Candidates (per-sequence coordinates) -> oracle layout (global)."""
    c = cands if isinstance(cands, np.ndarray) else binding.struct_view(cands, binding.CAND_DTYPE)
    if len(c) == 0:
        return np.zeros((0, len(oracle.CAND_COLS)), dtype=np.int64)
    off = np.asarray(offsets, dtype=np.int64)
    qs, ts = c["qseq"].astype(np.int64), c["tseq"].astype(np.int64)
    cols = {"qseq": qs, "q0": c["q0"] + off[qs], "q1": c["q1"] + off[qs], "tseq": ts,
            "t0": c["t0"] + off[ts], "t1": c["t1"] + off[ts], "o": c["o"],
            "score": c["score"], "nchains": c["nchains"]}
    return np.stack([np.asarray(cols[k], dtype=np.int64) for k in oracle.CAND_COLS], axis=1)


def rec_rows(rec_t) -> np.ndarray:
    return binding.records_to_rows(binding.to_numpy_records(rec_t))


def assert_rows_equal(got: np.ndarray, want: np.ndarray, what: str):
    assert got.shape == want.shape, f"{what}: shape {got.shape} != {want.shape}"
    if not np.array_equal(got, want):
        bad = np.nonzero(np.any(got != want, axis=1))[0]
        k = bad[0]
        raise AssertionError(f"{what}: {len(bad)} rows differ; first at {k}: "
                             f"got {got[k].tolist()} want {want[k].tolist()}")
