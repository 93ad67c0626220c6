"""Writes tests/golden/oracle_small.json: digests of the oracle's output on a
small seeded workload.  Calls only the oracle (and the input generator); run
it again only when the oracle's arithmetic changes for a reason the paper
gives."""
import hashlib
import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import numpy as np  # noqa: E402

import oracle  # noqa: E402
from paper_1807_00205_gb300 import synth  # noqa: E402


def digest(a: np.ndarray) -> str:
    return hashlib.sha256(np.ascontiguousarray(a, dtype=np.int64).tobytes()).hexdigest()


def workload():
    return synth.small_case(2024, lengths=(90_000, 35_000), n_sd=5, sd_lo=1500, sd_hi=6000,
                            id_lo=0.88, id_hi=0.995, mask_frac=0.2, n_gaps=True)


def compute():
    g = workload()
    r = oracle.selfsearch(g.seq, g.offsets, oracle.params())
    out = {}
    for key in ["recs", "index", "runs", "chains", "cands"]:
        out[key] = {"rows": int(len(r[key])), "sha256": digest(r[key])}
    out["offsets"] = {"rows": int(len(r["offsets"])), "sha256": digest(r["offsets"])}
    return out


if __name__ == "__main__":
    with open(os.path.join(HERE, "oracle_small.json"), "w") as f:
        json.dump(compute(), f, indent=1, sort_keys=True)
        f.write("\n")
