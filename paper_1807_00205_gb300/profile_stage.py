"""Runs the whole path a few times on a named workload, for profiler
captures of single kernels (e.g. `ncu -k regex:k_refine_batch -s 1 -c 1`).

    python -m paper_1807_00205_gb300.profile_stage [--workload chromosome|plain] [--repeat 2]
"""
import argparse
import os
import sys

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--workload", default="chromosome", choices=["chromosome", "plain"])
    ap.add_argument("--repeat", type=int, default=2)
    args = ap.parse_args()
    import torch
    from paper_1807_00205_gb300 import binding, synth
    g = synth.chromosome_100mbp() if args.workload == "chromosome" else synth.plain_2mbp()
    ctx = binding.Context(0)
    p = binding.params()
    d = torch.from_numpy(g.seq).cuda()
    out = None
    for _ in range(args.repeat):
        out = ctx.selfsearch(d, g.offsets, p)
    torch.cuda.synchronize()
    print("ok", out["nruns"], out["nchains"], out["ncands"], ctx.sedef_filter_stats())
    ctx.close()


if __name__ == "__main__":
    main()
