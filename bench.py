#!/usr/bin/env python
"""Throughput of the SEDEF seeding filter on one GB300 (or N replicas).

A step is one pass of the whole path over a device-resident input: pack,
sketch, index, filter (candidate lookup, sliding count, refine), chain and
merge, as one call of the C ABI (sedef_selfsearch).  The default workload is
the batch: 200 independent synthetic genomes of 1-20 Mbp (log-uniform, 1.43
Gbp in all; 41% GC, 30% soft-masked repeats, 50-500 planted duplications of
1-50 kbp at 75-99% identity), self-searched in one persistent pass
(self_mode 2), beside the plain form (one pass per genome).  Other
workloads: the 100 Mbp chromosome, the 2 Mbp plain genome, the 3.1 Gbp
human-scale assembly (self-search) and serving against its resident index.

Prints one JSON line (rank 0).  `value` is query Mbp/s of the whole job (all
ranks); `e2e` repeats the measurement through sedef_selfsearch_host with the
input in pinned host memory and the candidates copied back; `roofline`
relates the dominant kernel family's algorithmic bytes (or instructions) to
the measured peak; `cpu_baseline` times the CPU oracle on a bounded sample.

--impl reference times the CPU oracle (the reference arm of this build) on a
bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "query Mbp/s through sketch+Jaccard filter+chain (batched/served vs plain), p99 latency, HBM %"
WORKLOADS = {
    "batch": "batch of 200 independent genomes, 1-20 Mbp log-uniform (1.43 Gbp), 41% GC, 30% "
             "soft-masked repeats, 50-500 planted SDs of 1-50 kbp at 75-99% identity; one "
             "persistent pass (self_mode 2) vs one pass per genome",
    "chromosome": "chromosome-100Mbp self-search (41% GC, 40% soft-masked repeats, N-gaps, 2000 "
                  "planted SDs 1-200 kbp)",
    "plain": "plain-2Mbp self-search (i.i.d. ACGT, 20 planted SDs 1-20 kbp)",
    "human": "human-scale 3.1 Gbp self-search (24 chromosomes of 50-250 Mbp, 41% GC, 50% "
             "soft-masked repeats, N-gaps, 20000 planted SDs 1-300 kbp intra- and "
             "inter-chromosomal)",
}
FALLBACK_HBM_GBS = 6800.0
L2_FLUSH_BYTES = 256 << 20
COUNTERS = os.path.join(ROOT, "profiles", "roofline_counters.json")

# kernel families (trace stage labels) and the bound that holds for each
HBM_FAMILIES = ("pack", "sketch", "index", "filter")
ISSUE_FAMILIES = ("refine", "runsort", "chain", "merge")


class Workload:
    def __init__(self, name, seq, offsets, self_mode, genomes=None):
        self.name, self.seq, self.offsets, self.self_mode = name, seq, offsets, self_mode
        self.genomes = genomes

    @property
    def length(self) -> int:
        return int(self.offsets[-1])


def make_workload(name: str, max_genomes=None) -> Workload:
    from paper_1807_00205_gb300 import batch, synth
    if name == "batch":
        gs = synth.batch_genomes(max_genomes=max_genomes)
        seq, offs = batch.concatenate(gs)
        return Workload(name, seq, offs, 2, gs)
    g = {"chromosome": synth.chromosome_100mbp, "plain": synth.plain_2mbp,
         "human": synth.human_3gbp}[name]()
    return Workload(name, g.seq, g.offsets, 1)


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            d = json.load(f)
        hbm = d.get("hbm_gbs") or d.get("hbm_GBs") or d.get("hbm")
        if hbm:
            return float(hbm), "measured"
    return FALLBACK_HBM_GBS, "fallback"


class Clocks:
    """Samples SM clocks and throttle reasons during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device: int):
        self.device = device
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.device), f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}
        time.sleep(0.3)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as f:
            for line in f:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    sm.append(float(parts[1]))
                    smax.append(float(parts[2]))
                except ValueError:
                    continue
                for nm, v in zip(names, parts[5:9]):
                    if v.lower() == "active":
                        reasons.add(nm)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def aggregate_max_ms(ms: float, ws: int, device=None) -> float:
    """The slowest rank's time (all ranks call it; a no-op on one rank)."""
    if ws <= 1:
        return ms
    import torch
    import torch.distributed as dist
    t = torch.tensor([ms], dtype=torch.float64, device=device if device is not None else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def dist_info():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


# ------------------------------------------------------------ accounting --

def family_of(key: str) -> str:
    """Trace key "stage:kernel" -> kernel family (the stage label)."""
    return key.split(":", 1)[0] if ":" in key else "other"


def filter_algorithmic_bytes(rec, offsets, k, n, step, self_mode, nruns) -> dict:
    """The filter's algorithmic bytes for one pass, counted on the device:
    per query window, its query records (8 B each), one offset pair per
    distinct hash of W_Q (8 B) and every posting of those hashes (4 B: the
    position and strand a posting must carry; in self_mode 2 the postings
    of the window's own genome), plus the runs written (32 B each)."""
    import torch
    dev = rec.device
    r = rec.view(torch.int64)
    h = r >> 33
    pos = (r >> 1) & 0xFFFFFFFF
    off = torch.as_tensor(np.asarray(offsets, dtype=np.int64), device=dev)
    seq = torch.searchsorted(off, pos, right=True) - 1
    local = pos - off[seq]
    lens = off[1:] - off[:-1]
    nwin = torch.clamp((lens - n) // step + 1, min=0)
    wbase = torch.zeros(len(nwin) + 1, dtype=torch.int64, device=dev)
    wbase[1:] = torch.cumsum(nwin, 0)
    span = n - k
    w_lo = torch.clamp(torch.div(local - span + step - 1, step, rounding_mode="floor"), min=0)
    w_hi = torch.minimum(local // step, nwin[seq] - 1)
    keys, nq = [], 0
    for d in range(span // step + 2):
        w = w_lo + d
        ok = w <= w_hi
        nq += int(ok.sum())
        keys.append(((wbase[seq[ok]] + w[ok]) << 32) | h[ok])
    pairs = torch.unique(torch.cat(keys))
    del keys
    ph = pairs & 0xFFFFFFFF
    if self_mode == 2:
        wid = pairs >> 32
        wseq = torch.searchsorted(wbase, wid, right=True) - 1
        rk, rc = torch.unique((seq << 32) | h, return_counts=True)
        occ = rc[torch.searchsorted(rk, (wseq << 32) | ph)]
    else:
        occ = torch.bincount(h, minlength=1 << (2 * k))[ph]
    postings = int(occ.sum())
    return {"bytes": 4 * postings + 8 * int(pairs.numel()) + 8 * nq + 32 * int(nruns),
            "postings": postings, "distinct_query_hashes": int(pairs.numel()),
            "query_records": nq, "windows": int(wbase[-1])}


def algorithmic_bytes(N: int, nrec: int, k: int, filt: dict) -> dict:
    """Minimum bytes each HBM-bound family must move per pass: pack 1.5 B
    per base; sketch the packed input once (0.5 B per base) and 8 B per
    record written; index one read and one write of every record (the
    single-pass lower bound of a sort) and the 4^k + 1 offsets; filter as
    counted by filter_algorithmic_bytes."""
    return {"pack": int(1.5 * N), "sketch": int(0.5 * N + 8 * nrec),
            "index": 16 * nrec + 4 * ((1 << (2 * k)) + 1), "filter": filt["bytes"]}


def counters_entry(kernel: str, workload: str, variant: int):
    """Per-unit ncu counters of `kernel` captured on this workload with this
    filter shape, while its source file is unchanged; None otherwise."""
    if not os.path.exists(COUNTERS):
        return None
    with open(COUNTERS) as f:
        d = json.load(f)
    for e in d.get("entries", []):
        if e.get("kernel") != kernel or e.get("workload") != workload:
            continue
        if e.get("filter_shape") is not None and e["filter_shape"] != variant:
            continue
        src = os.path.join(ROOT, e["source"])
        if not os.path.exists(src):
            return None
        with open(src, "rb") as f:
            if hashlib.sha256(f.read()).hexdigest() != e["sha256"]:
                return None
        return e
    return None


# ---------------------------------------------------------- CPU baseline --

def oracle_selfsearch_rate(W: Workload, min_bases: int, threads: int):
    """The oracle self-searching a bounded sample of the workload: whole
    leading genomes of a batch (they are independent), or a prefix of one
    genome.  Returns (Mbp/s, seconds, bases, description)."""
    import oracle
    oracle.build()
    if W.genomes is not None:
        take, tot = [], 0
        for g in W.genomes:
            take.append(g)
            tot += g.length
            if tot >= min_bases:
                break
        from paper_1807_00205_gb300 import batch
        s, off = batch.concatenate(take)
        pd = oracle.params(self_mode=2)
        desc = f"self-search (self_mode 2) of the first {len(take)} genomes ({tot} bases)"
    else:
        X = min(min_bases, W.length)
        s, off = np.ascontiguousarray(W.seq[:X]), np.array([0, X], dtype=np.int64)
        pd = oracle.params()
        desc = f"self-search of the first {X} bases"
    t = time.perf_counter()
    oracle.selfsearch(s, off, pd, threads=threads)
    dt = time.perf_counter() - t
    bases = int(off[-1])
    return bases / dt / 1e6, dt, bases, desc


def cpu_baseline_line(W: Workload) -> dict:
    cores = os.cpu_count() or 1
    if W.name == "human":
        return cpu_baseline_windows(W, cores)
    v, dt, X, desc = oracle_selfsearch_rate(W, 30_000_000, cores)
    return {"value": v, "unit": "Mbp/s", "cores": cores, "kind": "oracle",
            "sample": f"{desc}, threads over windows, {dt:.1f} s wall"}


def cpu_baseline_windows(W: Workload, cores: int, nwin: int = 2000) -> dict:
    """Human scale: the oracle's sketch of the whole genome, then the filter
    over `nwin` evenly spaced query windows against the whole genome; Mbp/s
    counts query_step bases per window (each window stands for that much of
    the self-search)."""
    import oracle
    oracle.build()
    pd = oracle.params()
    t = time.perf_counter()
    recs = oracle.sketch(W.seq, W.offsets, pd, threads=cores)
    t_sk = time.perf_counter() - t
    wins = []
    for s in range(len(W.offsets) - 1):
        st, en = int(W.offsets[s]), int(W.offsets[s + 1])
        wins.extend(range(st, en - pd["n"] + 1, pd["step"]))
    wins = np.asarray(wins, dtype=np.int64)
    pick = wins[np.linspace(0, len(wins) - 1, nwin).astype(np.int64)]
    t = time.perf_counter()
    oracle.filter_runs(recs, W.offsets, recs, W.offsets, pd, windows=pick, threads=cores)
    t_f = time.perf_counter() - t
    per_win = t_f / nwin + t_sk / len(wins)
    return {"value": pd["step"] / per_win / 1e6, "unit": "Mbp/s", "cores": cores,
            "kind": "oracle",
            "sample": f"sketch of all {W.length} bases ({t_sk:.0f} s) and filter of {nwin} "
                      f"evenly spaced of {len(wins)} query windows ({t_f:.0f} s), extrapolated "
                      f"at {pd['step']} query bases per window; threads on all cores"}


def reference_arm(args):
    ws, rank, local = dist_info()
    if rank != 0:
        return
    if args.workload in ("serve", "human"):
        print(json.dumps({"impl": "reference", "unavailable":
                          "the CPU oracle cannot serve or self-search 3.1 Gbp within the bench's "
                          "time; its sampled rate is the cpu_baseline of --workload human"}))
        return
    cores = os.cpu_count() or 1
    W = make_workload(args.workload, max_genomes=12 if args.workload == "batch" else None)
    sample = 10_000_000
    for _ in range(args.warmup):
        oracle_selfsearch_rate(W, sample, cores)
    times, desc, bases = [], "", 0
    for _ in range(args.steps):
        _, dt, bases, desc = oracle_selfsearch_rate(W, sample, cores)
        times.append(dt)
    ms = 1000 * sum(times) / len(times)
    value = bases / (ms / 1000) / 1e6
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "Mbp/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u8",
        "data": "synthetic",
        "config": {"workload": WORKLOADS[args.workload], "sample": desc, "l2": "n/a (CPU)"},
        "cpu_baseline": {"value": value, "unit": "Mbp/s", "cores": cores, "kind": "oracle",
                         "sample": f"{desc} of the workload, threads over windows"},
        "e2e": {"value": value, "unit": "Mbp/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------- serving --

def serve_arm(args):
    """Resident index of the 3.1 Gbp human-scale workload (or the 100 Mbp
    chromosome); Poisson streams of query regions (10 kbp-5 Mbp, 0-25%
    mutation) at each rate, served by the continuously batching server and
    by the plain one-request-per-pass form."""
    import torch
    from paper_1807_00205_gb300 import binding, serve, synth
    ws, rank, local = dist_info()
    torch.cuda.set_device(local)
    g = {"human": synth.human_3gbp, "chromosome": synth.chromosome_100mbp}[args.serve_genome]()
    pool = synth.query_regions(g, 48)
    p = binding.params()
    ctx = binding.Context(local)
    index = serve.ResidentIndex(ctx, g.seq, g.offsets, p)
    results = []
    for rate in [float(x) for x in args.rates.split(",")]:
        row = {"rate": rate}
        for mode, workers, batching in [("served", 2, True), ("plain", 1, False)]:
            srv = serve.Server(index, p, workers=workers, batching=batching, device=local)
            srv.warm(pool[:8])
            srv.start()
            row[mode] = serve.run_load(srv, pool, rate, args.requests, seed=int(rate))
            srv.close()
        results.append(row)
    top = results[-1]
    name = "human" if args.serve_genome == "human" else "chromosome"
    line = {
        "metric": METRIC, "value": top["served"]["mbp_s"], "unit": "Mbp/s", "n_gpus": 1,
        "steps": args.requests, "warmup": 2, "ms_per_step": top["served"]["mean_ms"],
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u8",
        "data": "synthetic",
        "config": {"workload": f"serving: resident index of the {WORKLOADS[name]}; "
                               "Poisson query regions 10 kbp-5 Mbp log-uniform cut from it "
                               "with 0-25% mutation",
                   "served": "2 workers (own streams), continuous batching, admission by free HBM",
                   "plain": "1 worker, one request per pass"},
        "rates": results,
    }
    print(json.dumps(line), flush=True)
    ctx.close()


# -------------------------------------------- f1 extension, f2 chaining --

def measure_extension(ctx, out, W, p, d_seq, stream, max_seeds=2048, reps=2):
    """Section 3.2 (sedef_extend) and Section 3.3 (sedef_chain2) on an
    evenly spaced sample of at most max_seeds kept seeds of the pass, timed
    with CUDA events (best of `reps`).  Extending every kept seed of a large
    workload takes minutes: each seed of a duplication grows past it until
    the estimate falls, so the work grows with the square of the
    duplications' lengths."""
    import torch
    from paper_1807_00205_gb300 import binding
    runs = binding.struct_view(out["runs"], binding.RUN_DTYPE).copy()
    kept = np.nonzero(runs["keep"] == 1)[0]
    if len(kept) == 0:
        return None
    pick = kept[np.linspace(0, len(kept) - 1, min(max_seeds, len(kept))).astype(np.int64)]
    sel = np.zeros(len(runs), dtype=bool)
    sel[pick] = True
    runs["keep"] = np.where(sel, runs["keep"], 0)
    pa = binding.params_from_struct(p, min_unmasked=0)
    with torch.cuda.stream(stream):
        d_runs = torch.from_numpy(runs.view(np.uint8)).to(d_seq.device)
        ext = ctx.sedef_sketch(out["packed"], out["mask"], out["nbits"], W.offsets, pa)

    def timed(fn):
        best, res = None, None
        for _ in range(reps):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            with torch.cuda.stream(stream):
                e0.record(stream)
                res = fn()
                e1.record(stream)
            e1.synchronize()
            ms = e0.elapsed_time(e1)
            best = ms if best is None else min(best, ms)
        return best, res

    ems, (regions, nreg) = timed(lambda: ctx.sedef_extend(d_runs, len(runs), ext, W.offsets, ext,
                                                          W.offsets, p))
    cms, (sds, nsd) = timed(lambda: ctx.sedef_chain2(out["packed"], out["nbits"], W.length, regions,
                                                     nreg, p))
    reg = binding.struct_view(regions, binding.REGION_DTYPE)
    span = (reg["qb"].astype(np.int64) - reg["qa"]).sum()
    return {"seeds": int(nreg), "kept_seeds_in_pass": int(len(kept)),
            "sample": f"{int(nreg)} evenly spaced of {len(kept)} kept seeds",
            "extend_ms": ems, "extend_seeds_per_s": nreg / (ems / 1000),
            "region_bases": int(span), "mean_region_bases": float(span / max(nreg, 1)),
            "chain2_ms": cms, "chain2_regions_per_s": nreg / (cms / 1000),
            "chain2_query_mbp_s": span / (cms / 1000) / 1e6, "sds": int(nsd)}


# ------------------------------------------------------------- main arm --

def timed_steps(stream, flush, steps, warmup, fn):
    """Mean ms of `steps` calls of fn on `stream` (CUDA events, an L2 flush
    outside the events before each), after `warmup` untimed calls."""
    import torch
    with torch.cuda.stream(stream):
        for _ in range(warmup):
            fn()
            flush.fill_(1)
        ms = []
        for _ in range(steps):
            flush.fill_(1)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            fn()
            e1.record(stream)
            e1.synchronize()
            ms.append(e0.elapsed_time(e1))
    return sum(ms) / len(ms)


def run_workload(args):
    import torch
    from paper_1807_00205_gb300 import binding

    ws, rank, local = dist_info()
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    t0 = time.time()
    W = make_workload(args.workload, max_genomes=args.genomes)
    gen_s = time.time() - t0
    N = W.length
    p = binding.params(self_mode=W.self_mode)
    stream = torch.cuda.Stream(dev)
    ctx = binding.Context(local, stream=stream)
    with torch.cuda.stream(stream):
        d_seq = torch.from_numpy(W.seq).to(dev)
        flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.int32, device=dev)
    stream.synchronize()

    def barrier():
        if ws > 1:
            torch.distributed.barrier()

    # the filter's first-tier shape is autotuned once, then one pass stage by
    # stage keeps every intermediate for the accounting below (untimed)
    with torch.cuda.stream(stream):
        if args.variant is None:
            out = ctx.selfsearch(d_seq, W.offsets, p, autotune=True)
        else:
            ctx.sedef_filter_variant(args.variant)
        variant = ctx.sedef_filter_variant()[0]
        out = ctx.selfsearch(d_seq, W.offsets, p)
    fstats = ctx.sedef_filter_stats()

    def step():
        return ctx.sedef_selfsearch(d_seq, W.offsets, p)

    with torch.cuda.stream(stream):
        cands, ncands = step()  # sizes the context's buffers
    stream.synchronize()

    # ---- timed region: device-resident input, one C call per step
    barrier()
    torch.cuda.synchronize()
    clocks = Clocks(local)
    clocks.start()
    ctx.sedef_trace_report(reset=True)
    ctx.sedef_trace_enable(True)
    launches0 = binding.Context.sedef_launch_count()
    ms = timed_steps(stream, flush, args.steps, args.warmup, step)
    launches = (binding.Context.sedef_launch_count() - launches0) * args.steps // \
        (args.steps + args.warmup)
    ctx.sedef_trace_enable(False)
    trace = ctx.sedef_trace_report(reset=True)
    torch.cuda.synchronize()
    barrier()
    clk = clocks.stop()
    # the trace covers warm-up and timed steps alike: per-step figures divide
    # by their sum
    nsteps = args.steps + args.warmup
    ms = aggregate_max_ms(ms, ws, dev)
    value = ws * N / (ms / 1000) / 1e6

    # ---- plain form of the batch: one pass per genome (self_mode 1)
    plain = None
    if W.genomes is not None and not args.no_plain:
        pp = binding.params(self_mode=1)
        views = [d_seq[int(W.offsets[g]):int(W.offsets[g + 1])] for g in range(len(W.genomes))]
        offs1 = [np.array([0, int(W.offsets[g + 1] - W.offsets[g])], dtype=np.int64)
                 for g in range(len(W.genomes))]

        def plain_step():
            for v, o in zip(views, offs1):
                ctx.sedef_selfsearch(v, o, pp)

        l0 = binding.Context.sedef_launch_count()
        ms_p = timed_steps(stream, flush, args.steps, args.warmup, plain_step)
        lp = (binding.Context.sedef_launch_count() - l0) * args.steps // nsteps
        ms_p = aggregate_max_ms(ms_p, ws, dev)
        plain = {"value": ws * N / (ms_p / 1000) / 1e6, "unit": "Mbp/s", "ms_per_step": ms_p,
                 "mode": "one sedef_selfsearch call per genome (self_mode 1)",
                 "gpu_launches": int(lp), "batched_over_plain": ms_p / ms}

    # ---- the q-gram filter (Section 3.2) on the pass's kept seeds, timed alone
    with torch.cuda.stream(stream):
        qms = []
        for it in range(args.warmup + args.steps):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            _, qpass, npass = ctx.sedef_qgram(out["packed"], out["nbits"], N, out["runs"],
                                              out["nruns"], p, q=4, p_gap=0.005)
            e1.record(stream)
            e1.synchronize()
            if it >= args.warmup:
                qms.append(e0.elapsed_time(e1))
    kept = int((binding.struct_view(out["runs"], binding.RUN_DTYPE)["keep"] == 1).sum())
    qgram_info = {"q": 4, "p_gap": 0.005, "ms": sum(qms) / len(qms), "kept_seeds": kept,
                  "passed": int(npass), "bytes_per_seed": 2 * p.n // 4}
    # ---- the next steps of the method on a sample of the pass's seeds
    try:
        ext_info = None if args.no_extension else measure_extension(ctx, out, W, p, d_seq, stream)
    except binding.SedefError as e:
        ext_info = {"error": str(e)}

    # ---- the same pass as one captured graph (sedef_graph_*)
    graph_info = None
    try:
        if args.no_graph:
            raise RuntimeError("skipped (--no-graph)")
        with torch.cuda.stream(stream):
            caps = binding.caps_from_run(out, fstats)
            graph = ctx.selfsearch_graph(d_seq, W.offsets, p, caps=caps)

        def replay():
            graph.launch(stream)

        g_ms = timed_steps(stream, flush, args.steps, args.warmup, replay)
        graph.wait()
        graph_ms = aggregate_max_ms(g_ms, ws, dev)
        graph_info = {"value": ws * N / (graph_ms / 1000) / 1e6, "unit": "Mbp/s",
                      "ms_per_step": graph_ms, "kernel_nodes": graph.nodes,
                      "same_candidates": bool(graph.need["cands"] == int(ncands))}
        graph.close()
    except (binding.SedefError, RuntimeError) as e:
        graph_info = {"error": str(e)}

    # ---- end to end through the host-buffer entry point
    host_seq = torch.from_numpy(W.seq).pin_memory().numpy()
    e2e_times, nc_host = [], 0
    for it in range(0 if args.no_e2e else args.warmup + args.steps):
        barrier()
        t = time.perf_counter()
        hc = ctx.sedef_selfsearch_host(host_seq, W.offsets, p)
        dt = time.perf_counter() - t
        nc_host = len(hc)
        if it >= args.warmup:
            e2e_times.append(dt)
    e2e_ms = 1000 * sum(e2e_times) / len(e2e_times) if e2e_times else float("nan")
    e2e_ms = aggregate_max_ms(e2e_ms, ws, dev)

    if rank != 0:
        ctx.close()
        if ws > 1:
            torch.distributed.destroy_process_group()
        return

    # ---- per-family time, algorithmic bytes and the roofline
    peak, peak_kind = peaks()
    fam_ms = {}
    for key, (cnt, t) in trace.items():
        fam_ms[family_of(key)] = fam_ms.get(family_of(key), 0.0) + t / nsteps
    filt = filter_algorithmic_bytes(out["rec"], W.offsets, p.k, p.n, p.query_step, W.self_mode,
                                    out["nruns"])
    algo = algorithmic_bytes(N, int(out["rec"].numel()), p.k, filt)
    families = {}
    for f, t in sorted(fam_ms.items(), key=lambda kv: -kv[1]):
        e = {"ms_per_step": t, "share": t / ms}
        if f in algo and t > 0:
            gbs = algo[f] / (t / 1000) / 1e9
            e.update({"algorithmic_bytes": algo[f], "gbs": gbs, "frac_of_hbm": gbs / peak})
        families[f] = e
    dom = max(fam_ms.items(), key=lambda kv: kv[1])[0]
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    mhz = float(clk.get("sm_mhz") or clk.get("sm_max_mhz") or 2070.0)
    issue_peak = sms * 4 * mhz / 1000.0  # G warp instructions per second
    # per-unit ncu counters of the family (one capture on this workload and
    # filter shape, scaled by this pass's units: hits for the filter, runs
    # for the refine, bases for the streaming families)
    units = {"filter": int(fstats["hits"]), "refine": int(out["nruns"]),
             "runsort": int(out["nruns"]), "chain": int(out["nruns"]),
             "merge": int(out["nchains"]), "sketch": N, "pack": N, "index": N}.get(dom, 0)
    e = counters_entry(f"{dom} family", W.name, variant)
    issue = None
    traffic = None
    if e and units:
        inst = e["warp_instructions_per_unit"] * units
        a_i = inst / (fam_ms[dom] / 1000) / 1e9
        issue = {"achieved": a_i, "peak": issue_peak, "unit": "G warp-instructions/s",
                 "frac": a_i / issue_peak, "instructions_per_step": inst,
                 "peak_from": f"{sms} SMs x 4 schedulers x {mhz:.0f} MHz (median sampled)"}
        if e.get("dram_bytes_per_unit"):
            traffic = int(e["dram_bytes_per_unit"] * units)
    if dom in algo:
        a = algo[dom] / (fam_ms[dom] / 1000) / 1e9
        roof = {"kernel": f"{dom} family", "bound": "hbm", "achieved": a, "peak": peak,
                "unit": "GB/s", "frac": a / peak, "peak_source": peak_kind,
                "algorithmic_bytes_per_step": algo[dom], "ms_per_step": fam_ms[dom],
                "traffic": traffic, "issue": issue}
    else:
        # plain integer work bound by instruction issue: warp instructions
        # against 4 schedulers x SMs x the sampled SM clock
        roof = {"kernel": f"{dom} family", "bound": "alu", "peak": issue_peak,
                "unit": "G warp-instructions/s", "ms_per_step": fam_ms[dom],
                "achieved": issue["achieved"] if issue else None,
                "frac": issue["frac"] if issue else None, "traffic": traffic, "issue": issue}
    if e:
        roof["counters_from"] = e.get("profile")
        roof["counters_units"] = f"{units} {e.get('unit', 'units')}"
    kernels = {k: {"launches_per_step": c / nsteps, "ms_per_step": t / nsteps}
               for k, (c, t) in sorted(trace.items(), key=lambda kv: -kv[1][1])}
    if args.trace:
        print(json.dumps({"families": families, "kernels": kernels}, indent=1), file=sys.stderr)

    cpu = None
    if not args.no_cpu_baseline and ws == 1:
        cpu = cpu_baseline_line(W)

    line = {
        "metric": METRIC, "value": value, "unit": "Mbp/s", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "u8", "data": "synthetic",
        "config": {"workload": WORKLOADS[W.name], "genome_bases": N,
                   "sequences": len(W.offsets) - 1, "self_mode": W.self_mode, "k": p.k,
                   "w": p.w, "n": p.n, "query_step": p.query_step,
                   "parallelism": f"replicas x{ws}",
                   "l2": "inputs larger than L2 and a 256 MB L2 flush between steps",
                   "step": "one sedef_selfsearch call (pack ... merge) on the device-resident input",
                   "runs": int(out["nruns"]), "chains": int(out["nchains"]),
                   "candidates": int(ncands), "filter": fstats, "filter_accounting": filt,
                   "filter_shape": variant, "generation_s": gen_s},
        "plain": plain,
        "e2e": {"value": ws * N / (e2e_ms / 1000) / 1e6, "unit": "Mbp/s", "ms_per_step": e2e_ms,
                "h2d_bytes_per_step": int(N + 8 * len(W.offsets)),
                "d2h_bytes_per_step": int(nc_host * 40),
                "call": "sedef_selfsearch_host (page-locked host input read in place by the pack kernel over the host link, candidates copied back)"},
        "roofline": roof,
        "families": families,
        "cpu_baseline": cpu,
        "gpu_launches": int(launches),
        "clocks": clk,
        "graph": graph_info,
        "qgram": qgram_info,
        "extension_and_chain2": ext_info,
        "kernels": kernels,
    }
    print(json.dumps(line), flush=True)
    ctx.close()
    if ws > 1:
        torch.distributed.destroy_process_group()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="batch",
                    choices=["batch", "chromosome", "plain", "human", "serve"])
    ap.add_argument("--serve-genome", default="human", choices=["human", "chromosome"],
                    help="serving: the genome whose index stays resident")
    ap.add_argument("--rates", default="50,200,1000", help="serving: request rates per second")
    ap.add_argument("--requests", type=int, default=200, help="serving: requests per rate")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true", help="skip the host-buffer measurement")
    ap.add_argument("--no-graph", action="store_true", help="skip the captured-graph measurement")
    ap.add_argument("--no-plain", action="store_true", help="batch: skip the one-pass-per-genome form")
    ap.add_argument("--no-extension", action="store_true",
                    help="skip the extension / two-tier chaining measurement")
    ap.add_argument("--genomes", type=int, default=None,
                    help="batch: only the first N genomes of the batch (smaller runs, e.g. profiling)")
    ap.add_argument("--variant", type=int, default=None,
                    help="the filter's first-tier shape instead of autotuning it")
    ap.add_argument("--trace", action="store_true", help="print the per-kernel table to stderr")
    args = ap.parse_args()
    if args.impl == "reference":
        reference_arm(args)
    elif args.workload == "serve":
        serve_arm(args)
    else:
        run_workload(args)


if __name__ == "__main__":
    main()
